// FP32 production instantiations of the ESP kernels (P = 4 ... 12), plus the
// precision-independent scan and energy launchers.
#include <algorithm>

#define ESP_REAL float
#define ESP_P_MIN 4
#define ESP_NEAR_SHORT 10
#define ESP_P_MAX 12
// P = 4 ... 7 here, 8 ... 12 in esp_kern_f32_rest.cu (compiled in parallel)
#define ESP_P_CASES(FN, ...)                                              \
  ESP_P_CASE(4, FN, __VA_ARGS__) ESP_P_CASE(5, FN, __VA_ARGS__)           \
  ESP_P_CASE(6, FN, __VA_ARGS__) ESP_P_CASE(7, FN, __VA_ARGS__)
#include "esp_kern_impl.cuh"

namespace espk {

long long scan_tiles(long long n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan(const uint32_t* count, uint32_t* start, uint32_t* tile_sum, long long n,
                        cudaStream_t st) {
  const int tiles = (int)((n + kScanTile - 1) / kScanTile);
  if (tiles == 0) return cudaMemsetAsync(start, 0, sizeof(uint32_t), st);
  if (n <= kScanSmallMax) {
    k_scan_small<<<1, kScanThreads, 0, st>>>(count, start, n);
    return cudaGetLastError();
  }
  k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(count, start, tile_sum, n);
  k_scan_add<<<tiles, kScanThreads, 0, st>>>(start, tile_sum, n);
  return cudaGetLastError();
}

cudaError_t launch_energy(const SysDesc* sys, int nsys, const double* fourier, int n_fourier_blocks,
                          const double* partials, int n_chunks, const int* chunk_first,
                          const double* consts, double* out, double* user_energy, cudaStream_t st,
                          const double* vpart, const double* vloc, double* vout) {
  EnergyArgs ea;
  ea.nsys = nsys;
  ea.fourier = fourier;
  ea.n_fourier_blocks = n_fourier_blocks;
  ea.chunk_first = chunk_first;
  ea.consts = consts;
  ea.out = out;
  ea.user_energy = user_energy;
  ea.vpart = vpart;
  ea.vloc = vloc;
  ea.vout = vout;
  k_energy<<<nsys, 1024, 0, st>>>(sys, ea, partials, n_chunks);
  return cudaGetLastError();
}

}  // namespace espk
