// FP32 production instantiations of the ESP kernels (P = 4 ... 12), plus the
// precision-independent scan and energy launchers.
#include <algorithm>

#define ESP_REAL float
#define ESP_P_MIN 4
#define ESP_NEAR_SHORT 10
#define ESP_P_MAX 12
#define ESP_P_CASES(FN, ...)                                              \
  ESP_P_CASE(4, FN, __VA_ARGS__) ESP_P_CASE(5, FN, __VA_ARGS__)           \
  ESP_P_CASE(6, FN, __VA_ARGS__) ESP_P_CASE(7, FN, __VA_ARGS__)           \
  ESP_P_CASE(8, FN, __VA_ARGS__) ESP_P_CASE(9, FN, __VA_ARGS__)           \
  ESP_P_CASE(10, FN, __VA_ARGS__) ESP_P_CASE(11, FN, __VA_ARGS__)         \
  ESP_P_CASE(12, FN, __VA_ARGS__)
#include "esp_kern_impl.cuh"
#include "esp_near_cluster.cuh"

namespace espk {

template <>
cudaError_t Launch<float>::near_clusters(const SysDesc* sys, int nsys, long long n_cols,
                                         const uint32_t* start, const void* rel, void* nearres,
                                         const NearCoef<float>& nc, int terms, uint32_t* ccount,
                                         uint32_t* cstart, uint32_t* ctiles, int2* cmap, int2* catoms,
                                         long long cmap_cap, bool half, long long n_atoms, int stage,
                                         int* err, cudaStream_t st) {
  if (n_cols == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (!(stage & 1)) {
    // cluster lists
    const int cb = (int)((n_cols * 32 + 255) / 256);     // one warp per column
    k_col_clusters<<<cb, 256, 0, st>>>(sys, nsys, n_cols, start, ccount);
    e = launch_scan(ccount, cstart, ctiles, n_cols, st);
    if (e != cudaSuccess) return e;
    k_cluster_expand<<<cb, 256, 0, st>>>(sys, nsys, n_cols, ccount, cstart, start, cmap, catoms, cmap_cap, err);
    if (stage == 2) return cudaGetLastError();
  }
  decltype(&k_near_cluster<ESP_NEAR_SHORT, false>) kern = nullptr;
  if (terms == ESP_NEAR_SHORT) kern = half ? k_near_cluster<ESP_NEAR_SHORT, true> : k_near_cluster<ESP_NEAR_SHORT, false>;
  else if (terms == Deg<float>::nr) kern = half ? k_near_cluster<Deg<float>::nr, true> : k_near_cluster<Deg<float>::nr, false>;
  if (!kern) return cudaErrorInvalidValue;
  if (half) {
    // every result is accumulated with atomics
    e = cudaMemsetAsync(nearres, 0, (size_t)n_atoms * sizeof(float4), st);
    if (e != cudaSuccess) return e;
  }
  // persistent grid: as many blocks as fit on the device at once, each block
  // taking a contiguous run of clusters
  static int blocks_full = 0, blocks_half = 0;
  int& blocks = half ? blocks_half : blocks_full;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kClusterWarps * 32, 0);
    blocks = std::max(1, sms * std::max(1, per_sm));
  }
  const long long need = (cmap_cap + kClusterWarps - 1) / kClusterWarps;
  const int grid = (int)std::min<long long>(blocks, std::max<long long>(1, need));
  kern<<<grid, kClusterWarps * 32, 0, st>>>(sys, cmap, catoms, cstart + n_cols, (const float4*)rel, start,
                                           (float4*)nearres, nc, err);
  return cudaGetLastError();
}

long long scan_tiles(long long n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan(const uint32_t* count, uint32_t* start, uint32_t* tile_sum, long long n,
                        cudaStream_t st) {
  const int tiles = (int)((n + kScanTile - 1) / kScanTile);
  if (tiles == 0) return cudaMemsetAsync(start, 0, sizeof(uint32_t), st);
  k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(count, start, tile_sum, n);
  k_scan_totals<<<1, kScanThreads, 0, st>>>(tile_sum, tiles, start, n);
  k_scan_add<<<tiles, kScanThreads, 0, st>>>(start, tile_sum, n);
  return cudaGetLastError();
}

cudaError_t launch_energy(const SysDesc* sys, int nsys, const double* fourier, int n_fourier_blocks,
                          const double* partials, int n_chunks, const int* chunk_first,
                          const double* consts, double* out, double* user_energy, cudaStream_t st) {
  k_energy<<<nsys, 256, 0, st>>>(sys, fourier, n_fourier_blocks, partials, n_chunks, chunk_first,
                                 consts, out, user_energy);
  return cudaGetLastError();
}

}  // namespace espk
