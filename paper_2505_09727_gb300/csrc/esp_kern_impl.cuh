// Launcher bodies shared by the FP32 and FP64 instantiation units. Each unit
// defines ESP_REAL and the P range it compiles, then includes this file.
#pragma once
#include <algorithm>
#include "esp_kernels.cuh"
#include "esp_launch.h"

namespace espk {

namespace detail {

template <typename K>
static cudaError_t allow_smem(K kernel, size_t smem) {
  if (smem <= 32 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename real, typename In>
__global__ void __launch_bounds__(256) k_convert(const In* __restrict__ src, real* __restrict__ dst,
                                                 long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (real)src[i];
}

// CTAs per brick so that small grids of bricks still fill the device: at
// least two CTAs per SM in total, at most 16 per brick.
static int brick_splits(int n_work) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int want = 2 * sms;
  return std::max(1, std::min(16, (want + n_work - 1) / std::max(1, n_work)));
}

}  // namespace detail

#ifndef ESP_IMPL_REST
template <>
cudaError_t Launch<ESP_REAL>::ingest(const SysDesc* sys, const int2* chunks, int n_chunks,
                                     const void* xyz, bool xyz_is_double, void* coord,
                                     uint32_t* key, uint32_t* rank, uint32_t* count, int* err,
                                     cudaStream_t st) {
  using A = typename Types<ESP_REAL>::atom;
  if (n_chunks == 0) return cudaSuccess;
  if (xyz_is_double)
    k_ingest<ESP_REAL, double><<<n_chunks, kChunk, 0, st>>>(
        sys, chunks, (const double*)xyz, (A*)coord, key, rank, count, err);
  else
    k_ingest<ESP_REAL, float><<<n_chunks, kChunk, 0, st>>>(
        sys, chunks, (const float*)xyz, (A*)coord, key, rank, count, err);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<ESP_REAL>::scatter(const SysDesc* sys, const int2* chunks, int n_chunks,
                                      const void* coord, const uint32_t* key, const uint32_t* rank,
                                      const uint32_t* start, const ESP_REAL* q, void* atoms,
                                      void* rel, uint32_t* perm, cudaStream_t st) {
  using A = typename Types<ESP_REAL>::atom;
  using R = typename Types<ESP_REAL>::res;
  if (n_chunks == 0) return cudaSuccess;
  k_scatter<ESP_REAL, ESP_REAL><<<n_chunks, kChunk, 0, st>>>(sys, chunks, (const A*)coord, key, rank,
                                                             start, q, (A*)atoms, (R*)rel, perm);
  return cudaGetLastError();
}
#endif  // ESP_IMPL_REST

template <int P>
static cudaError_t spread_p(const SysDesc* sys, const int2* work, int n_work, size_t smem,
                            const void* atoms, const uint32_t* start, ESP_REAL* grids,
                            const SICoef<ESP_REAL>& si, int* err, cudaStream_t st) {
  using A = typename Types<ESP_REAL>::atom;
  if constexpr (sizeof(ESP_REAL) == 4) {
    // private tile per warp while up to 8 tiles fit in ~110 KB (two CTAs per
    // SM); otherwise one shared tile with shared-memory atomics
    const size_t stride = (smem / sizeof(float) + 31) & ~size_t(31);   // floats, bank-aligned
    const size_t per_warp = (stride + SpreadScratch<P>::kFloats) * sizeof(float);
    const int nwarps = (int)std::min<size_t>(8, (110u * 1024u) / per_warp);
    if (nwarps >= 2) {
      auto kw = k_spread_warps<P>;
      const size_t bytes = nwarps * per_warp;
      cudaError_t e = detail::allow_smem(kw, bytes);
      if (e != cudaSuccess) return e;
      const int splits = detail::brick_splits(n_work);
      kw<<<n_work * splits, 256, bytes, st>>>(sys, work, (const uint4*)atoms, start, (float*)grids, si, nwarps,
                                              (int)stride, splits, err);
      return cudaGetLastError();
    }
  }
  auto kern = k_spread<ESP_REAL, P>;
  cudaError_t e = detail::allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<n_work, 256, smem, st>>>(sys, work, (const A*)atoms, start, grids, si, err);
  return cudaGetLastError();
}

template <int P>
static cudaError_t gather_p(const SysDesc* sys, const int2* work, int n_work, size_t smem,
                            const void* atoms, const uint32_t* start, const ESP_REAL* grids,
                            const ESP_REAL* grids_ik, long long grid_total,
                            void* far, const SICoef<ESP_REAL>& si, int* err, cudaStream_t st) {
  using A = typename Types<ESP_REAL>::atom;
  using R = typename Types<ESP_REAL>::res;
  if (grids_ik) {
    // ik method: potential and three gradient tiles
    auto ki = k_gather_ik<ESP_REAL, P>;
    cudaError_t e = detail::allow_smem(ki, 4 * smem);
    if (e != cudaSuccess) return e;
    const int splits = detail::brick_splits(n_work);
    ki<<<n_work * splits, 256, 4 * smem, st>>>(sys, work, (const A*)atoms, start, grids, grids_ik, grid_total,
                                               (R*)far, si, splits, err);
    return cudaGetLastError();
  }
  auto kern = k_gather<ESP_REAL, P>;
  cudaError_t e = detail::allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int splits = detail::brick_splits(n_work);
  kern<<<n_work * splits, 256, smem, st>>>(sys, work, (const A*)atoms, start, grids, (R*)far, si, splits, err);
  return cudaGetLastError();
}

#define ESP_P_CASE(PP, FN, ...) \
  case PP: return FN<PP>(__VA_ARGS__);

// The stencil widths are split over two units compiled in parallel: the
// main unit's ESP_P_CASES, and the rest in a second unit (ESP_IMPL_REST)
// reached through spread_rest / gather_rest.
cudaError_t spread_rest(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem, const void* atoms,
                        const uint32_t* start, ESP_REAL* grids, const SICoef<ESP_REAL>& si, int* err,
                        cudaStream_t st);
cudaError_t gather_rest(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem, const void* atoms,
                        const uint32_t* start, const ESP_REAL* grids, const ESP_REAL* grids_ik, long long grid_total,
                        void* far, const SICoef<ESP_REAL>& si, int* err, cudaStream_t st);

#ifdef ESP_IMPL_REST

cudaError_t spread_rest(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem, const void* atoms,
                        const uint32_t* start, ESP_REAL* grids, const SICoef<ESP_REAL>& si, int* err,
                        cudaStream_t st) {
  switch (P) {
    ESP_P_CASES(spread_p, sys, work, n_work, smem, atoms, start, grids, si, err, st)
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gather_rest(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem, const void* atoms,
                        const uint32_t* start, const ESP_REAL* grids, const ESP_REAL* grids_ik, long long grid_total,
                        void* far, const SICoef<ESP_REAL>& si, int* err, cudaStream_t st) {
  switch (P) {
    ESP_P_CASES(gather_p, sys, work, n_work, smem, atoms, start, grids, grids_ik, grid_total, far, si, err, st)
    default: return cudaErrorInvalidValue;
  }
}

#else

template <>
cudaError_t Launch<ESP_REAL>::spread(int P, const SysDesc* sys, const int2* work, int n_work,
                                     size_t smem, const void* atoms, const uint32_t* start,
                                     ESP_REAL* grids, const SICoef<ESP_REAL>& si, int* err,
                                     cudaStream_t st) {
  if (n_work == 0) return cudaSuccess;
  switch (P) {
    ESP_P_CASES(spread_p, sys, work, n_work, smem, atoms, start, grids, si, err, st)
    default: return spread_rest(P, sys, work, n_work, smem, atoms, start, grids, si, err, st);
  }
}

template <>
cudaError_t Launch<ESP_REAL>::gather(int P, const SysDesc* sys, const int2* work, int n_work,
                                     size_t smem, const void* atoms, const uint32_t* start,
                                     const ESP_REAL* grids, const ESP_REAL* grids_ik, long long grid_total,
                                     void* far, const SICoef<ESP_REAL>& si, int* err, cudaStream_t st) {
  if (n_work == 0) return cudaSuccess;
  switch (P) {
    ESP_P_CASES(gather_p, sys, work, n_work, smem, atoms, start, grids, grids_ik, grid_total, far, si, err, st)
    default: return gather_rest(P, sys, work, n_work, smem, atoms, start, grids, grids_ik, grid_total, far, si,
                                err, st);
  }
}

template <>
bool Launch<ESP_REAL>::supports_P(int P) { return P >= ESP_P_MIN && P <= ESP_P_MAX; }

template <>
cudaError_t Launch<ESP_REAL>::scale(const SysDesc* sys, int nsys, int nblk, void* spec,
                                    const ESP_REAL* tabs, double* partials, void* spec_ik,
                                    long long spec_total, double* vpart, cudaStream_t st) {
  using C = typename Types<ESP_REAL>::cplx;
  dim3 grid(nblk, nsys);
  k_scale<ESP_REAL><<<grid, 256, 0, st>>>(sys, (C*)spec, tabs, partials, (C*)spec_ik, spec_total, vpart);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<ESP_REAL>::near(const SysDesc* sys, const int2* chunks, int n_chunks,
                                   const void* atoms, const void* rel, const uint32_t* start,
                                   void* nearres, const NearCoef<ESP_REAL>& nc, int terms,
                                   bool queued, cudaStream_t st, double* vloc) {
  using A = typename Types<ESP_REAL>::atom;
  using R = typename Types<ESP_REAL>::res;
  if (n_chunks == 0) return cudaSuccess;
  if (vloc && queued) return cudaErrorNotSupported;     // the virial is formed in the inline form
  decltype(&k_near<ESP_REAL, ESP_NEAR_SHORT, true>) kern = nullptr;
  // fewer terms run on the shorter instance: the unused coefficients are zero
  if (terms <= ESP_NEAR_SHORT)
    kern = vloc ? k_near<ESP_REAL, ESP_NEAR_SHORT, false, true>
                : queued ? k_near<ESP_REAL, ESP_NEAR_SHORT, true> : k_near<ESP_REAL, ESP_NEAR_SHORT, false>;
  else if (terms == Deg<ESP_REAL>::nr)
    kern = vloc ? k_near<ESP_REAL, Deg<ESP_REAL>::nr, false, true>
                : queued ? k_near<ESP_REAL, Deg<ESP_REAL>::nr, true> : k_near<ESP_REAL, Deg<ESP_REAL>::nr, false>;
  if (!kern) return cudaErrorInvalidValue;
  const size_t smem = queued ? kNearQueueBytes : 0;
  cudaError_t e = detail::allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<n_chunks, kChunk, smem, st>>>(sys, chunks, (const A*)atoms, (const R*)rel, start, (R*)nearres, nc, vloc);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<ESP_REAL>::finalize(const SysDesc* sys, const int2* chunks, int n_chunks,
                                       const void* atoms, const uint32_t* perm, const void* far,
                                       const void* nearres, void* forces, void* pot,
                                       bool out_double, double* partials, cudaStream_t st,
                                       const EnergyArgs& ea) {
  using A = typename Types<ESP_REAL>::atom;
  using R = typename Types<ESP_REAL>::res;
  if (n_chunks == 0) return cudaSuccess;
  if (out_double)
    k_finalize<ESP_REAL, double><<<n_chunks, kChunk, 0, st>>>(
        sys, chunks, (const A*)atoms, perm, (const R*)far, (const R*)nearres, (double*)forces,
        (double*)pot, partials, n_chunks, ea);
  else
    k_finalize<ESP_REAL, float><<<n_chunks, kChunk, 0, st>>>(
        sys, chunks, (const A*)atoms, perm, (const R*)far, (const R*)nearres, (float*)forces,
        (float*)pot, partials, n_chunks, ea);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<ESP_REAL>::exclusions(const SysDesc* sys, const int2* pairs, long long n_pairs,
                                         const uint32_t* perm, uint32_t* inv, long long n_atoms, const void* atoms,
                                         void* nearres, cudaStream_t st) {
  using A = typename Types<ESP_REAL>::atom;
  using R = typename Types<ESP_REAL>::res;
  if (n_pairs == 0 || n_atoms == 0) return cudaSuccess;
  k_inverse_perm<<<(int)((n_atoms + 255) / 256), 256, 0, st>>>(perm, inv, n_atoms);
  k_exclusions<ESP_REAL><<<(int)((n_pairs + 255) / 256), 256, 0, st>>>(sys, pairs, n_pairs, inv, (const A*)atoms,
                                                                       (R*)nearres);
  return cudaGetLastError();
}

template <>
cudaError_t Launch<ESP_REAL>::convert_charges(const void* src, bool src_double, ESP_REAL* dst,
                                              long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (src_double)
    detail::k_convert<ESP_REAL, double><<<blocks, 256, 0, st>>>((const double*)src, dst, n);
  else
    detail::k_convert<ESP_REAL, float><<<blocks, 256, 0, st>>>((const float*)src, dst, n);
  return cudaGetLastError();
}

template <>
size_t Launch<ESP_REAL>::atom_bytes() { return sizeof(typename Types<ESP_REAL>::atom); }
template <>
size_t Launch<ESP_REAL>::res_bytes() { return sizeof(typename Types<ESP_REAL>::res); }

#endif  // ESP_IMPL_REST

}  // namespace espk
