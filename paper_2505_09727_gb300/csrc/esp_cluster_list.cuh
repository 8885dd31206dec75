// Cluster lists of the FP32 local part: per cell-list column the number of
// i-clusters (up to kClusterAtoms consecutive atoms of the column in z
// order), and per cluster its (system, column) and its atoms. Built once per
// step from the counting sort's cell offsets alone.
#pragma once
#include "esp_kernels.cuh"

namespace espk {

constexpr int kClusterAtoms = kClusterAtomsHost;

__device__ __forceinline__ int system_of_column(const SysDesc* __restrict__ sys, int nsys, long long g) {
  int lo = 0, hi = nsys - 1;                      // last system with col0 <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sys[mid].col0 <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One warp per pooled column (lanes over the column's bricks).
// Cluster count per column: ceil(atoms in the column / kClusterAtoms).
static __global__ void __launch_bounds__(256) k_col_clusters(
    const SysDesc* __restrict__ sys, int nsys, long long n_cols, const uint32_t* __restrict__ start,
    uint32_t* __restrict__ ccount) {
  const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_cols) return;
  const SysDesc& S = sys[system_of_column(sys, nsys, g)];
  const int c = (int)(g - S.col0);
  const int cx = c / S.n_c, cy = c - cx * S.n_c;
  const uint32_t* st = start + S.cell0;
  uint32_t total = 0;
  for (int bz = lane; bz < S.nb; bz += 32) {
    const long long k0 = cell_key(S, cx, cy, bz * S.bc);
    total += st[(k0 + S.bc) * kSub] - st[k0 * kSub];
  }
  total = __reduce_add_sync(0xffffffffu, total);
  if (lane == 0) ccount[g] = (total + kClusterAtoms - 1) / kClusterAtoms;
}

// Cluster list: cmap[q] = (system, column) and catoms[q][t] = (atom index,
// brick z index) of the t-th atom of cluster q = cstart[column] + k
// (index -1 in the empty slots of a column's last cluster).
static __global__ void __launch_bounds__(256) k_cluster_expand(
    const SysDesc* __restrict__ sys, int nsys, long long n_cols, const uint32_t* __restrict__ ccount,
    const uint32_t* __restrict__ cstart, const uint32_t* __restrict__ start, int2* __restrict__ cmap,
    int2* __restrict__ catoms, long long capacity, int* __restrict__ err) {
  const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_cols) return;
  const int s = system_of_column(sys, nsys, g);
  const SysDesc& S = sys[s];
  const int c = (int)(g - S.col0);
  const int cx = c / S.n_c, cy = c - cx * S.n_c;
  const uint32_t n = ccount[g], b = cstart[g];
  if ((long long)b + n > capacity) {
    if (lane == 0) atomicOr(err, 4);
    return;
  }
  for (uint32_t k = lane; k < n; k += 32) cmap[b + k] = make_int2(s, c);
  const uint32_t* st = start + S.cell0;
  const long long slots = (long long)n * kClusterAtoms;
  int2* out = catoms + (long long)b * kClusterAtoms;
  long long p = 0;                                  // position of the group's first atom
  for (int bz0 = 0; bz0 < S.nb; bz0 += 32) {
    // lane k reads brick bz0 + k's atom range; a warp scan places them
    const int bz = bz0 + lane;
    uint32_t j0 = 0, cnt = 0;
    if (bz < S.nb) {
      const long long k0 = cell_key(S, cx, cy, bz * S.bc);
      j0 = st[k0 * kSub];
      cnt = st[(k0 + S.bc) * kSub] - j0;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t excl = incl - cnt;
    const int nbz = min(32, S.nb - bz0);
    for (int k = 0; k < nbz; ++k) {
      const uint32_t bj0 = __shfl_sync(0xffffffffu, j0, k);
      const uint32_t bcnt = __shfl_sync(0xffffffffu, cnt, k);
      const long long bpos = p + __shfl_sync(0xffffffffu, excl, k);
      for (uint32_t j = lane; j < bcnt; j += 32)
        if (bpos + j < slots) out[bpos + j] = make_int2((int)(bj0 + j), bz0 + k);
    }
    p += __shfl_sync(0xffffffffu, incl, 31);
  }
  for (long long q = p + lane; q < slots; q += 32) out[q] = make_int2(-1, 0);
}

}  // namespace espk
