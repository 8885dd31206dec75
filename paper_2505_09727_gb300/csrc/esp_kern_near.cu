// FP32 local part with one warp per cluster (see esp_near_cluster.cuh):
// launcher and instantiations for 8, 9, 10 and 12 polynomial terms.
#include <algorithm>

#include "esp_launch.h"
#include "esp_near_cluster.cuh"

namespace espk {

template <>
cudaError_t Launch<float>::near_clusters(const SysDesc* sys, int nsys, long long n_cols,
                                         const uint32_t* start, const void* rel, void* nearres,
                                         const NearCoef<float>& nc, int terms, uint32_t* ccount,
                                         uint32_t* cstart, uint32_t* ctiles, int2* cmap, int2* catoms,
                                         long long cmap_cap, bool half, long long n_atoms, int stage,
                                         int* err, cudaStream_t st, double* vloc) {
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
  if (vloc && !half) return cudaErrorNotSupported;         // the virial is formed in the half form
  decltype(&k_near_cluster<10, false>) kern = nullptr;
  switch (terms) {
    case 8: kern = vloc ? k_near_cluster<8, true, true> : half ? k_near_cluster<8, true> : k_near_cluster<8, false>; break;
    case 9: kern = vloc ? k_near_cluster<9, true, true> : half ? k_near_cluster<9, true> : k_near_cluster<9, false>; break;
    case 10: kern = vloc ? k_near_cluster<10, true, true> : half ? k_near_cluster<10, true> : k_near_cluster<10, false>; break;
    case 12: kern = vloc ? k_near_cluster<12, true, true> : half ? k_near_cluster<12, true> : k_near_cluster<12, false>; break;
    default: return cudaErrorInvalidValue;
  }
  if (half) {
    // every result is accumulated with atomics
    e = cudaMemsetAsync(nearres, 0, (size_t)n_atoms * sizeof(float4), st);
    if (e != cudaSuccess) return e;
  }
  // persistent grid: as many blocks as fit on the device at once, each block
  // taking a contiguous run of clusters
  static int blocks_full = 0, blocks_half = 0, blocks_vir = 0;
  int& blocks = vloc ? blocks_vir : half ? blocks_half : blocks_full;
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
                                           (float4*)nearres, nc, err, vloc);
  return cudaGetLastError();
}

}  // namespace espk
