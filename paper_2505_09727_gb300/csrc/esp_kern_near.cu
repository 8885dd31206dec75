// FP32 local part with one warp per cluster (see esp_near_cluster.cuh):
// launcher and instantiations for 8, 9, 10 and 12 polynomial terms.
#include <algorithm>

#include "esp_launch.h"
#include "esp_near_cluster.cuh"

namespace espk {

// The pair kernel with WARPS warps per block, on a persistent grid of as many
// blocks as fit on the device at once, each taking a contiguous run of
// clusters.
template <int WARPS>
static cudaError_t launch_near_cluster(const SysDesc* sys, long long n_cols, const uint32_t* start, const void* rel,
                                       void* nearres, const NearCoef<float>& nc, int terms, const uint32_t* cstart,
                                       const int2* cmap, const int2* catoms, long long cmap_cap, bool half, int* err,
                                       cudaStream_t st, double* vloc, int sms, bool tri) {
  decltype(&k_near_cluster<10, false, false, WARPS>) kern = nullptr;
  switch (terms) {
#define ESP_NC_CASE(T)                                                                       \
    case T:                                                                                  \
      kern = tri ? k_near_cluster<T, true, false, WARPS, true>                                \
           : vloc ? k_near_cluster<T, true, true, WARPS>                                      \
                  : half ? k_near_cluster<T, true, false, WARPS> : k_near_cluster<T, false, false, WARPS>; \
      break;
    ESP_NC_CASE(8)
    ESP_NC_CASE(9)
    ESP_NC_CASE(10)
    ESP_NC_CASE(12)
#undef ESP_NC_CASE
    default: return cudaErrorInvalidValue;
  }
  static int blocks[4] = {0, 0, 0, 0};              // per form: full, half, half + virial, triclinic
  int& nb = blocks[tri ? 3 : vloc ? 2 : half ? 1 : 0];
  if (nb == 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, 0);
    nb = std::max(1, sms * std::max(1, per_sm));
  }
  const long long need = (cmap_cap + WARPS - 1) / WARPS;
  const int grid = (int)std::min<long long>(nb, std::max<long long>(1, need));
  kern<<<grid, WARPS * 32, 0, st>>>(sys, cmap, catoms, cstart + n_cols, (const float4*)rel, start,
                                    (float4*)nearres, interleave(nc), err, vloc);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<float>::near_clusters(const SysDesc* sys, int nsys, long long n_cols,
                                         const uint32_t* start, const void* rel, void* nearres,
                                         const NearCoef<float>& nc, int terms, uint32_t* ccount,
                                         uint32_t* cstart, uint32_t* ctiles, int2* cmap, int2* catoms,
                                         long long cmap_cap, bool half, long long n_atoms, int stage,
                                         int* err, cudaStream_t st, double* vloc, bool tri) {
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
  if (tri && (vloc || !half)) return cudaErrorNotSupported; // triclinic: half form, no virial
  if (half) {
    // every result is accumulated with atomics
    e = cudaMemsetAsync(nearres, 0, (size_t)n_atoms * sizeof(float4), st);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the list's capacity decides the block shape: 16-warp blocks once every
  // SM gets at least 4 clusters per warp
  const bool large = cmap_cap >= (long long)sms * kClusterWarpsLarge * 4;
  return large ? launch_near_cluster<kClusterWarpsLarge>(sys, n_cols, start, rel, nearres, nc, terms, cstart, cmap,
                                                          catoms, cmap_cap, half, err, st, vloc, sms, tri)
               : launch_near_cluster<kClusterWarpsSmall>(sys, n_cols, start, rel, nearres, nc, terms, cstart, cmap,
                                                          catoms, cmap_cap, half, err, st, vloc, sms, tri);
}

}  // namespace espk
