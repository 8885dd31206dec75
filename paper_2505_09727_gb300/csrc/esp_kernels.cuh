// Kernel templates of the ESP pipeline (see esp_device.cuh for the overview).
// Instantiated for FP32 (production) in esp_kern_f32.cu and FP64 (plain mode)
// in esp_kern_f64.cu.
#pragma once
#include <climits>

#include "esp_device.cuh"

namespace espk {

constexpr double kFourPi = 12.566370614359172953850573533118;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// 32-byte aligned FP64 quadruple (one 256-bit access per atom / result).
struct __align__(32) dquad { double x, y, z, w; };
__host__ __device__ inline dquad make_dquad(double x, double y, double z, double w) {
  dquad d; d.x = x; d.y = y; d.z = z; d.w = w; return d;
}

template <typename real> struct Types;
template <> struct Types<float> {
  using atom = uint4;      // (ux, uy, uz) fixed point, w = charge bits
  using res = float4;      // (u, a, b, c)
  using cplx = float2;
};
template <> struct Types<double> {
  using atom = dquad;      // (x, y, z) wrapped, w = charge
  using res = dquad;
  using cplx = double2;
};

template <typename real> __device__ inline typename Types<real>::cplx make_cplx(real re, real im) {
  typename Types<real>::cplx c;
  c.x = re;
  c.y = im;
  return c;
}

__device__ inline float atom_q(const uint4& a) { return __uint_as_float(a.w); }
__device__ inline double atom_q(const dquad& a) { return a.w; }

// ------------------------------------------------------------ cell geometry
// Cells are numbered brick by brick; inside a brick z runs fastest, so the
// cells of one column of a brick are consecutive.
__device__ inline int cell_key(const SysDesc& S, int cx, int cy, int cz) {
  const int bc = S.bc, nb = S.nb;
  const int bx = cx / bc, by = cy / bc, bz = cz / bc;
  const int lx = cx - bx * bc, ly = cy - by * bc, lz = cz - bz * bc;
  return ((bz * nb + by) * nb + bx) * (bc * bc * bc) + (lx * bc + ly) * bc + lz;
}

__device__ inline void atom_cell(const SysDesc& S, const uint4& a, int& cx, int& cy, int& cz) {
  cx = (int)(((uint64_t)a.x * (uint64_t)S.n_c) >> 32);
  cy = (int)(((uint64_t)a.y * (uint64_t)S.n_c) >> 32);
  cz = (int)(((uint64_t)a.z * (uint64_t)S.n_c) >> 32);
}

__device__ inline int cell_f64(double x, const SysDesc& S) {
  int c = (int)(x * S.inv_L * S.n_c);
  return c < 0 ? 0 : (c >= S.n_c ? S.n_c - 1 : c);
}

__device__ inline void atom_cell(const SysDesc& S, const dquad& a, int& cx, int& cy, int& cz) {
  cx = cell_f64(a.x, S);
  cy = cell_f64(a.y, S);
  cz = cell_f64(a.z, S);
}

// Tile origin of brick coordinate cb (cells cb*bc ...) along one axis.
__device__ inline int tile_origin(const SysDesc& S, int cbrick, int P, float) {
  return tile_origin_fixed(cbrick * S.bc, S.n_c, S.n_f, P);
}
__device__ inline int tile_origin(const SysDesc& S, int cbrick, int P, double) {
  double d;
  double x = (double)(cbrick * S.bc) * S.L / S.n_c;
  return stencil_origin_f64(x, S.L, S.n_f, P, d) - 1;   // one-point margin for FP64 rounding
}

// Stencil of one coordinate: origin l0 and y = 2 delta - 1.
__device__ inline int stencil(const SysDesc& S, uint32_t u, int P, float& y) {
  int l0; int64_t r;
  stencil_fixed(u, S.n_f, P, l0, r);
  y = (float)(r - (1LL << 31)) * 4.656612873077392578125e-10f;   // 2^-31
  return l0;
}
__device__ inline int stencil(const SysDesc& S, double x, int P, double& y) {
  double delta;
  int l0 = stencil_origin_f64(x, S.L, S.n_f, P, delta);
  y = 2.0 * delta - 1.0;
  return l0;
}

// P SI weights (and optionally derivatives d phi / dt) at y.
template <typename real, int P, bool DERIV>
__device__ __forceinline__ void si_weights(const SICoef<real>& si, real y, real* w, real* dw) {
  constexpr int NC = Deg<real>::si;
#pragma unroll
  for (int a = 0; a < P; ++a) {
    real v = si.c[a][NC - 1];
    real d = real(0);
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) {
      if (DERIV) d = d * y + v;
      v = v * y + si.c[a][k];
    }
    w[a] = v;
    if (DERIV) dw[a] = real(2) * d;    // d/dt = d/d delta = 2 d/dy
  }
}

// Weight (and derivative) of one stencil point a (runtime, block-uniform).
template <typename real, bool DERIV>
__device__ __forceinline__ void si_weight_one(const SICoef<real>& si, int a, real y, real& w, real& dw) {
  constexpr int NC = Deg<real>::si;
  real v = si.c[a][NC - 1];
  real d = real(0);
#pragma unroll
  for (int k = NC - 2; k >= 0; --k) {
    if (DERIV) d = d * y + v;
    v = v * y + si.c[a][k];
  }
  w = v;
  if (DERIV) dw = real(2) * d;
}

// Wide stencils keep the outer (z) loop rolled to bound code size.
template <int P> struct Unroll { static constexpr int outer = P <= 8 ? P : 1; };

// ================================================================ kernels
// A0: wrap, convert, key, rank. One thread per atom of a chunk.
template <typename real, typename In>
__global__ void __launch_bounds__(kChunk) k_ingest(
    const SysDesc* __restrict__ sys, const int2* __restrict__ chunks, const In* __restrict__ xyz,
    typename Types<real>::atom* __restrict__ coord, uint32_t* __restrict__ key,
    uint32_t* __restrict__ rank, uint32_t* __restrict__ count, int* __restrict__ err) {
  const int2 ch = chunks[blockIdx.x];
  const SysDesc& S = sys[ch.x];
  const int local = ch.y + threadIdx.x;
  if (local >= S.n_atoms) return;
  const long long i = S.atom0 + local;
  double p[3];
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p[a] = (double)xyz[3 * i + a];
    // finite = exponent field not all ones (integer test, no FP64 compare)
    finite &= ((__double_as_longlong(p[a]) >> 52) & 0x7ff) != 0x7ff;
  }
  if (!finite) {
    atomicOr(err, 1);
    p[0] = p[1] = p[2] = 0.0;
  }
  int c[3];
  int slab;
  typename Types<real>::atom out;
  if constexpr (sizeof(real) == 4) {
    uint32_t u[3];
    if (S.tri) {
      // triclinic cell: u = floor(s 2^32) mod 2^32 of the fractional
      // coordinates s = H^-1 r (H^-1 upper triangular)
      const double* t = S.tfix;
      const double sv[3] = {fma(p[0], t[0], fma(p[1], t[1], p[2] * t[2])), fma(p[1], t[3], p[2] * t[4]),
                            p[2] * t[5]};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        long long v = __double2ll_rd(sv[a]);
        if (v == LLONG_MAX || v == LLONG_MIN) {   // saturated: |s| beyond 2^31
          double f = sv[a] * 2.3283064365386962890625e-10;
          f -= floor(f);
          v = (long long)(f * 4294967296.0);
        }
        u[a] = (uint32_t)(unsigned long long)v;
        c[a] = (int)(((uint64_t)u[a] * (uint64_t)S.n_c) >> 32);
      }
    } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // u = floor(x 2^32 / L) mod 2^32 (the periodic wrap is the mod), in
      // integer arithmetic: exact for every finite x
      u[a] = fixed_from_double(p[a], S.fix_m, S.fix_e);
      c[a] = (int)(((uint64_t)u[a] * (uint64_t)S.n_c) >> 32);
    }
    }
    // slab: fractional position inside the z cell, in kSub parts
    const uint32_t zfrac = (uint32_t)((uint64_t)u[2] * (uint64_t)S.n_c);
    slab = (int)(((uint64_t)zfrac * kSub) >> 32);
    out = make_uint4(u[0], u[1], u[2], 0u);
  } else {
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double x = p[a];
      if (!(x >= 0.0 && x < S.L)) {
        x = x - S.L * floor(x / S.L);
        if (!(x < S.L) || x < 0.0) x = 0.0;
      }
      w[a] = x;
      c[a] = cell_f64(x, S);
    }
    slab = (int)((w[2] - c[2] * S.w) / S.w * kSub);
    slab = slab < 0 ? 0 : (slab >= kSub ? kSub - 1 : slab);
    out = make_dquad(w[0], w[1], w[2], 0.0);
  }
  const uint32_t k = (uint32_t)(cell_key(S, c[0], c[1], c[2]) * kSub + slab);
  coord[i] = out;
  key[i] = k;
  // warp-aggregated: lanes with the same slab key take consecutive ranks from
  // one atomic (input order is often spatially coherent, so keys repeat)
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, k);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&count[S.cell0 + k], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  rank[i] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// A1a: exclusive scan of the pooled cell-list counts in two passes: each
// block scans kScanTile entries and records its total; then every block adds
// the sum of the totals before it. start[n] receives the grand total.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t x = wsum[lane];
    uint32_t xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    wsum[lane] = xi - x;
    if (lane == 31) wsum[32] = xi;
  }
  __syncthreads();
  const uint32_t r = wsum[wid] + incl - v;
  if (total) *total = wsum[32];
  __syncthreads();
  return r;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_tiles(
    const uint32_t* __restrict__ count, uint32_t* __restrict__ start, uint32_t* __restrict__ tile_sum,
    long long n) {
  __shared__ uint32_t wsum[33];
  const long long b = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (b + k < n) ? count[b + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, wsum, &total);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (b + k < n) start[b + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// Whole scan in one CTA for short arrays (one launch instead of three): each
// thread sums a contiguous run of entries, the CTA scans the run sums, and
// each thread writes its run.
constexpr long long kScanSmallMax = (long long)kScanThreads * 16;

static __global__ void __launch_bounds__(kScanThreads) k_scan_small(
    const uint32_t* __restrict__ count, uint32_t* __restrict__ start, long long n) {
  __shared__ uint32_t wsum[33];
  const long long per = (n + kScanThreads - 1) / kScanThreads;
  const long long b = per * threadIdx.x;
  const long long e = b + per < n ? b + per : n;
  uint32_t s = 0;
  for (long long j = b; j < e; ++j) s += count[j];
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, wsum, &total);
  for (long long j = b; j < e; ++j) {
    const uint32_t t = count[j];
    start[j] = run;
    run += t;
  }
  if (threadIdx.x == 0) start[n] = total;
}

// Sum of v over the CTA (every thread gets it); wsum holds 32 words.
__device__ inline uint32_t block_sum_u32(uint32_t v, uint32_t* wsum) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();                                  // wsum is free again
  if (lane == 0) wsum[wid] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
  return t;
}

// Second pass: each tile adds the sum of the tile totals before it (a CTA
// reduction over the totals); the last tile also writes the grand total to
// start[n].
static __global__ void __launch_bounds__(kScanThreads) k_scan_add(
    uint32_t* __restrict__ start, const uint32_t* __restrict__ tile_sum, long long n) {
  __shared__ uint32_t wsum[32];
  const int tb = (int)blockIdx.x;
  uint32_t before = 0, through = 0;
  for (int j = threadIdx.x; j <= tb; j += blockDim.x) {
    const uint32_t t = tile_sum[j];
    through += t;
    if (j < tb) before += t;
  }
  const uint32_t off = block_sum_u32(before, wsum);
  if (tb == (int)gridDim.x - 1) {
    const uint32_t tot = block_sum_u32(through, wsum);
    if (threadIdx.x == 0) start[n] = tot;
  }
  const long long b = (long long)tb * kScanTile + (long long)threadIdx.x * kScanPer;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (b + k < n) start[b + k] += off;
}

// A1b: counting-sort scatter. perm[sorted] = pooled caller index.
// Position of a coordinate relative to the lower face of its cell (x, y) or
// of its brick (z: the cells of a brick column share one z frame).
__device__ inline float cell_relative(const SysDesc& S, uint32_t u) {
  const uint32_t frac = (uint32_t)((uint64_t)u * (uint64_t)S.n_c);   // fraction of the cell
  return (float)frac * S.w32f;                                        // < w: two FP32 roundings
}
__device__ inline float brick_relative(const SysDesc& S, uint32_t u) {
  const uint64_t t = (uint64_t)u * (uint64_t)S.n_c;                   // 32.32 cell coordinate
  const uint32_t c = (uint32_t)(t >> 32);
  // position in the brick as an exact 35-bit fixed-point integer, one FP64
  // product and one rounding to FP32 (z spans several cells)
  const uint64_t in_brick = ((uint64_t)(c % (uint32_t)S.bc) << 32) | (uint32_t)t;
  return (float)((double)in_brick * S.w32);
}
// Triclinic cell: the position relative to the brick corner H (cx, cy,
// bz bc) / n_c in Cartesian coordinates, H applied in FP64 to the exact
// fixed-point fractions inside the cell (x, y) and the brick (z).
__device__ inline float4 tri_relative(const SysDesc& S, uint4 a) {
  const double f = 2.3283064365386962890625e-10;
  const double fx = (double)(uint32_t)((uint64_t)a.x * (uint64_t)S.n_c) * f;
  const double fy = (double)(uint32_t)((uint64_t)a.y * (uint64_t)S.n_c) * f;
  const uint64_t t = (uint64_t)a.z * (uint64_t)S.n_c;
  const uint32_t c = (uint32_t)(t >> 32);
  const double fz = (double)(((uint64_t)(c % (uint32_t)S.bc) << 32) | (uint32_t)t) * f;
  const double* e = S.tcell;     // a_x, b_x, b_y, c_x, c_y, c_z over n_c
  return make_float4((float)fma(fx, e[0], fma(fy, e[1], fz * e[3])), (float)fma(fy, e[2], fz * e[4]),
                     (float)(fz * e[5]), 0.f);
}
__device__ inline double brick_relative(const SysDesc&, double x) { return x; }
// FP64 mode keeps absolute wrapped coordinates in the pair records, so pair
// differences are the same FP64 subtractions as a plain minimum-image sum.
__device__ inline double cell_relative(const SysDesc&, double x) { return x; }

template <typename real, typename Q>
__global__ void __launch_bounds__(kChunk) k_scatter(
    const SysDesc* __restrict__ sys, const int2* __restrict__ chunks,
    const typename Types<real>::atom* __restrict__ coord, const uint32_t* __restrict__ key,
    const uint32_t* __restrict__ rank, const uint32_t* __restrict__ start, const Q* __restrict__ q,
    typename Types<real>::atom* __restrict__ atoms, typename Types<real>::res* __restrict__ rel,
    uint32_t* __restrict__ perm) {
  const int2 ch = chunks[blockIdx.x];
  const SysDesc& S = sys[ch.x];
  const int local = ch.y + threadIdx.x;
  if (local >= S.n_atoms) return;
  const long long i = S.atom0 + local;
  const uint32_t dst = start[S.cell0 + key[i]] + rank[i];
  typename Types<real>::atom a = coord[i];
  typename Types<real>::res r;
  if constexpr (sizeof(real) == 4) {
    if (S.tri) {
      r = tri_relative(S, a);
    } else {
      r.x = cell_relative(S, a.x);
      r.y = cell_relative(S, a.y);
      r.z = brick_relative(S, a.z);
    }
  } else {
    r.x = cell_relative(S, a.x);
    r.y = cell_relative(S, a.y);
    r.z = brick_relative(S, a.z);
  }
  r.w = (real)q[i];
  if constexpr (sizeof(real) == 4) a.w = __float_as_uint((float)q[i]);
  else a.w = (double)q[i];
  atoms[dst] = a;
  rel[dst] = r;
  perm[dst] = (uint32_t)i;
}

// A2: spread (Eq. spread). One CTA per (system, brick).
template <typename real, int P>
__global__ void __launch_bounds__(256) k_spread(
    const SysDesc* __restrict__ sys, const int2* __restrict__ work,
    const typename Types<real>::atom* __restrict__ atoms, const uint32_t* __restrict__ start,
    real* __restrict__ grids, const SICoef<real> si, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* tile = reinterpret_cast<real*>(smem_raw);
  const int2 wk = work[blockIdx.x];
  const SysDesc& S = sys[wk.x];
  const int nb = S.nb, T = S.T, n_f = S.n_f, bc = S.bc;
  const int b = wk.y;
  const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
  const int ox = tile_origin(S, bx, P, real()), oy = tile_origin(S, by, P, real()),
            oz = tile_origin(S, bz, P, real());
  const int PY = S.tpy, PZ = S.tpz;
  for (int j = threadIdx.x; j < PZ * T; j += blockDim.x) tile[j] = real(0);
  __syncthreads();
  const long long k0 = S.cell0 + (long long)b * bc * bc * bc * kSub;
  const uint32_t a_begin = start[k0], a_end = start[k0 + bc * bc * bc * kSub];
  for (uint32_t i = a_begin + threadIdx.x; i < a_end; i += blockDim.x) {
    const typename Types<real>::atom at = atoms[i];
    real yx, yy, yz;
    const int lx = stencil(S, at.x, P, yx) - ox;
    const int ly = stencil(S, at.y, P, yy) - oy;
    const int lz = stencil(S, at.z, P, yz) - oz;
    if (lx < 0 || ly < 0 || lz < 0 || lx > T - P || ly > T - P || lz > T - P) {
      atomicOr(err, 2);
      continue;
    }
    real wx[P], wy[P];
    si_weights<real, P, false>(si, yx, wx, nullptr);
    si_weights<real, P, false>(si, yy, wy, nullptr);
    const real q = (real)atom_q(at);
#pragma unroll (Unroll<P>::outer)
    for (int c = 0; c < P; ++c) {
      real wzc, unused;
      si_weight_one<real, false>(si, c, yz, wzc, unused);
      const real qz = q * wzc;
#pragma unroll
      for (int bb = 0; bb < P; ++bb) {
        const real qzy = qz * wy[bb];
        real* row = tile + (lz + c) * PZ + (ly + bb) * PY + lx;
#pragma unroll
        for (int a = 0; a < P; ++a) atomicAdd(row + a, qzy * wx[a]);
      }
    }
  }
  __syncthreads();
  real* grid = grids + S.grid0;
  for (int jyx = threadIdx.x; jyx < T * T; jyx += blockDim.x) {
    const int jy = jyx / T, jx = jyx - jy * T;
    const long long gyx = (long long)wrap_near(oy + jy, n_f) * n_f + wrap_near(ox + jx, n_f);
    for (int jz = 0; jz < T; ++jz) {
      const real v = tile[jz * PZ + jy * PY + jx];
      if (v != real(0)) atomicAdd(grid + (long long)wrap_near(oz + jz, n_f) * n_f * n_f + gyx, v);
    }
  }
}

// A2 (FP32): spread with one private tile per warp and no atomics inside the
// block. Every warp of the brick's CTAs takes an equal contiguous share of
// the brick's atoms, in chunks of 32: lane l evaluates the 3P one-dimensional
// weights of the chunk's atom l (charge folded into the z weights) and its
// tile offset into the warp's scratch; then the chunk's atoms follow each
// other, every lane taking whole stencil rows (b, c) of the atom (the rows
// beyond the last full pass of 32, when their points fit one pass, one point
// per lane). The points of one atom are distinct, so plain read-add-write
// needs no atomics, and the padded tile pitches put the rows of one atom on
// distinct banks. The private tiles are summed point by point and flushed to
// the grid with global atomics (bricks overlap by P - 1 points).
template <int P>
struct SpreadScratch {
  static constexpr int kW = 3 * P | 1;            // weights per atom; odd: lane stores hit distinct banks
  static constexpr int kFloats = 32 * kW + 32;    // weights of 32 atoms + their tile offsets
};

template <int P>
__global__ void __launch_bounds__(256) k_spread_warps(
    const SysDesc* __restrict__ sys, const int2* __restrict__ work, const uint4* __restrict__ atoms,
    const uint32_t* __restrict__ start, float* __restrict__ grids, const SICoef<float> si, int nwarps,
    int tile_stride, int splits, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kW = SpreadScratch<P>::kW;
  float* tiles = reinterpret_cast<float*>(smem_raw);                 // [nwarps][tile_stride]
  const int2 wk = work[blockIdx.x / splits];
  const int split = blockIdx.x % splits;
  const SysDesc& S = sys[wk.x];
  const int nb = S.nb, T = S.T, n_f = S.n_f, bc = S.bc;
  const int b = wk.y;
  const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
  const int ox = tile_origin(S, bx, P, 0.f), oy = tile_origin(S, by, P, 0.f), oz = tile_origin(S, bz, P, 0.f);
  const int T2 = T * T, PY = S.tpy, PZ = S.tpz;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < nwarps * tile_stride; j += blockDim.x) tiles[j] = 0.f;
  __syncthreads();
  const long long k0 = S.cell0 + (long long)b * bc * bc * bc * kSub;
  const uint32_t a_begin = start[k0], a_end = start[k0 + bc * bc * bc * kSub];
  if (wid < nwarps) {
    float* tile = tiles + (size_t)wid * tile_stride;
    float* wts = tiles + (size_t)nwarps * tile_stride + (size_t)wid * SpreadScratch<P>::kFloats;
    int* offs = reinterpret_cast<int*>(wts + 32 * kW);
    constexpr int kRows = P * P;
    // rows left after the full passes of 32; when their points fit one pass
    // (P = 6: 4 rows, 24 points) they go one point per lane instead of a
    // row pass with few lanes busy
    constexpr int kLeftRows = kRows % 32;
    constexpr bool kPointTail = kRows > 32 && kLeftRows > 0 && kLeftRows * P <= 32;
    constexpr int kPass = kPointTail ? kRows / 32 : (kRows + 31) / 32;
    int row_off[kPass], wy_at[kPass], wz_at[kPass];
#pragma unroll
    for (int k = 0; k < kPass; ++k) {
      const int r = min(lane + 32 * k, kRows - 1);
      row_off[k] = (r / P) * PZ + (r % P) * PY;
      wy_at[k] = P + r % P;
      wz_at[k] = 2 * P + r / P;
    }
    int pt_off = 0, pt_wx = 0, pt_wy = 0, pt_wz = 0;   // kPointTail: this lane's point
    if constexpr (kPointTail) {
      const int pnt = min(lane, kLeftRows * P - 1);
      const int r = kRows - kLeftRows + pnt / P;
      pt_wx = pnt % P;
      pt_off = (r / P) * PZ + (r % P) * PY + pt_wx;
      pt_wy = P + r % P;
      pt_wz = 2 * P + r / P;
    }
    // the brick's atoms in equal contiguous shares, one per warp of its CTAs
    const int n_here = (int)(a_end - a_begin);
    const int parts = nwarps * splits, part = split * nwarps + wid;
    const int p_lo = (int)((long long)n_here * part / parts);
    const int p_hi = (int)((long long)n_here * (part + 1) / parts);
    for (int a0 = p_lo; a0 < p_hi; a0 += 32) {
      const int cnt = min(32, p_hi - a0);
      bool sok = false;
      if (lane < cnt) {
        const uint4 at = atoms[a_begin + a0 + lane];
        float yx, yy, yz;
        const int lx = stencil(S, at.x, P, yx) - ox;
        const int ly = stencil(S, at.y, P, yy) - oy;
        const int lz = stencil(S, at.z, P, yz) - oz;
        sok = !(lx < 0 || ly < 0 || lz < 0 || lx > T - P || ly > T - P || lz > T - P);
        if (!sok) atomicOr(err, 2);
        float w[3 * P];
        si_weights<float, P, false>(si, yx, w, nullptr);
        si_weights<float, P, false>(si, yy, w + P, nullptr);
        si_weights<float, P, false>(si, yz, w + 2 * P, nullptr);
        const float q = __uint_as_float(at.w);
        float* mine = wts + lane * kW;
#pragma unroll
        for (int k = 0; k < 2 * P; ++k) mine[k] = w[k];
#pragma unroll
        for (int k = 2 * P; k < 3 * P; ++k) mine[k] = q * w[k];
        offs[lane] = sok ? lz * PZ + ly * PY + lx : -1;
      }
      __syncwarp();
      for (int t = 0; t < cnt; ++t) {
        const int off = offs[t];
        if (off < 0) continue;                   // warp-uniform
        const float* wt = wts + t * kW;
        float wx[P];
#pragma unroll
        for (int a = 0; a < P; ++a) wx[a] = wt[a];
#pragma unroll
        for (int k = 0; k < kPass; ++k) {
          if (lane + 32 * k < kRows) {
            const float wyz = wt[wy_at[k]] * wt[wz_at[k]];
            float* row = tile + off + row_off[k];
#pragma unroll
            for (int a = 0; a < P; ++a) row[a] = fmaf(wyz, wx[a], row[a]);
          }
        }
        if constexpr (kPointTail) {
          // the same product and rounding as the row form
          if (lane < kLeftRows * P) {
            float* pt = tile + off + pt_off;
            *pt = fmaf(wt[pt_wy] * wt[pt_wz], wt[pt_wx], *pt);
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // flush: a thread keeps one (y, x) column of the tile and walks it in z
  float* grid = grids + S.grid0;
  for (int jyx = threadIdx.x; jyx < T2; jyx += blockDim.x) {
    const int jy = jyx / T, jx = jyx - jy * T;
    const long long gyx = (long long)wrap_near(oy + jy, n_f) * n_f + wrap_near(ox + jx, n_f);
    int jt = jy * PY + jx;
    for (int jz = 0; jz < T; ++jz, jt += PZ) {
      float v = 0.f;
      for (int k = 0; k < nwarps; ++k) v += tiles[(size_t)k * tile_stride + jt];
      if (v != 0.f) atomicAdd(grid + (long long)wrap_near(oz + jz, n_f) * n_f * n_f + gyx, v);
    }
  }
}

// Knuth's TwoSum: hi + lo += t with the rounding error of the sum kept in lo.
__device__ __forceinline__ void acc_two_sum(float& hi, float& lo, float t) {
  const float s = hi + t;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (t - bp);
  hi = s;
}

// A4: influence scale fused with the spectral energy (Eq. pk). Grid-stride
// over the half spectrum [kz][ky][kx], kx in [0, n_f/2]; blockIdx.y = system.
template <typename real>
__global__ void __launch_bounds__(256) k_scale(
    const SysDesc* __restrict__ sys, typename Types<real>::cplx* __restrict__ spec,
    const real* __restrict__ tabs, double* __restrict__ partials,
    typename Types<real>::cplx* __restrict__ spec_ik, long long spec_total, double* __restrict__ vpart) {
  __shared__ double red[32];
  const SysDesc& S = sys[blockIdx.y];
  const int n = S.n_f, nh = n / 2 + 1, half = n / 2;
  const long long total = (long long)n * n * nh;
  typename Types<real>::cplx* sp = spec + S.spec0;
  const real* G = tabs + S.tab0;
  const real* W = G + S.gsize;
  const real* H = W + (half + 1);                 // virial table: p'_k over the window factors
  double e = 0.0;                                 // FP64 plans
  float e_hi = 0.f, e_lo = 0.f;                   // FP32 plans: error-free (hi, lo) sum
  double vir[6] = {0, 0, 0, 0, 0, 0};             // xx, yy, zz, xy, xz, yz
  // one mode; kx, kyi, kzi its half-spectrum indices
  auto mode = [&](long long idx, int kx, int kyi, int kzi) {
    const int ky = kyi < half ? kyi : kyi - n;
    const int kz = kzi < half ? kzi : kzi - n;
    const int m = kx * kx + ky * ky + kz * kz;
    // cube: G over |k|^2; triclinic cell: G over the half spectrum itself
    const long long gi = S.tri ? idx : (long long)m;
    const real p = __ldg(G + gi) * __ldg(W + kx) * __ldg(W + abs(ky)) * __ldg(W + abs(kz));
    typename Types<real>::cplx v = sp[idx];
    const bool edge = kx == 0 || kx == half;
    if constexpr (sizeof(real) == 4) {
      acc_two_sum(e_hi, e_lo, (edge ? 1.f : 2.f) * p * fmaf(v.x, v.x, v.y * v.y));
    } else {
      e += (edge ? 1.0 : 2.0) * (double)p * ((double)v.x * v.x + (double)v.y * v.y);
    }
    if (vpart && m > 0) {
      const double wgt = edge ? 1.0 : 2.0;
      // virial of the mode: 1/2 |bh|^2 W W W [G delta + H k k^T / |k|^2]
      const double a = 0.5 * wgt * (double)(__ldg(W + kx) * __ldg(W + abs(ky)) * __ldg(W + abs(kz))) *
                       ((double)v.x * v.x + (double)v.y * v.y);
      const double g = a * (double)__ldg(G + m), hm = a * (double)__ldg(H + m) / m;
      // a Nyquist index stands for both aliases +-n_f/2. The exact
      // -dE/d eps pairs the mode with the representative of -k, whose
      // Nyquist components flip together: an off-diagonal product is zero
      // when exactly one of its two components is Nyquist and k_a k_b (with
      // both at -n_f/2) when both are
      const bool even = (n & 1) == 0;
      const bool nx = even && kx == half, ny = even && kyi == half, nz = even && kzi == half;
      const int ax = nx ? -half : kx;               // ky, kz are already -n_f/2 there
      vir[0] += g + hm * kx * kx;
      vir[1] += g + hm * ky * ky;
      vir[2] += g + hm * kz * kz;
      vir[3] += nx != ny ? 0.0 : hm * ax * ky;
      vir[4] += nx != nz ? 0.0 : hm * ax * kz;
      vir[5] += ny != nz ? 0.0 : hm * ky * kz;
    }
    v.x *= p;
    v.y *= p;
    sp[idx] = v;
    if (spec_ik) {
      // ik method: the inverse transform is sum_k c_k exp(+2 pi i k.l/n_f),
      // so d/dx_a multiplies c_k by +2 pi i k_a / L; the Nyquist component
      // of the differentiated axis is zero (no real grid function)
      const real s = real(kTwoPi / S.L);
      const real sx = kx == half ? real(0) : s * kx;
      const real sy = kyi == half ? real(0) : s * ky;
      const real sz = kzi == half ? real(0) : s * kz;
      typename Types<real>::cplx* o = spec_ik + S.spec0 + idx;
      o[0] = make_cplx<real>(-v.y * sx, v.x * sx);
      o[spec_total] = make_cplx<real>(-v.y * sy, v.x * sy);
      o[2 * spec_total] = make_cplx<real>(-v.y * sz, v.x * sz);
    }
  };
  if (total < (1ll << 31)) {
    // 32-bit index arithmetic (64-bit division is slow)
    const uint32_t t32 = (uint32_t)total, unh = (uint32_t)nh, un = (uint32_t)n;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < t32; idx += gridDim.x * blockDim.x) {
      const uint32_t r = idx / unh;
      const uint32_t kzi = r / un;
      mode(idx, (int)(idx - r * unh), (int)(r - kzi * un), (int)kzi);
    }
  } else {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
      const long long r = idx / nh;
      mode(idx, (int)(idx % nh), (int)(r % n), (int)(r / n));
    }
  }
  if constexpr (sizeof(real) == 4) e = f32_to_f64(e_hi) + f32_to_f64(e_lo);
  e = block_sum(e, red);
  if (threadIdx.x == 0) partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = 0.5 * e;
  if (vpart) {
    for (int c = 0; c < 6; ++c) {
      const double t = block_sum(vir[c], red);
      if (threadIdx.x == 0) vpart[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 6 + c] = t;
    }
  }
}

// The T^3 tile of a brick (origin ox, oy, oz, periodic) from the grid into
// shared memory: one element per thread and step, four loads in flight per
// thread (the element index split by FP32 reciprocals, exact for these
// sizes: the quotients stay 1e-4 away from integers and below 2^24).
template <typename real>
__device__ __forceinline__ void load_tile(real* __restrict__ tile, const real* __restrict__ grid, int T, int PY,
                                          int PZ, int ox, int oy, int oz, int n_f) {
  const int T2 = T * T, T3 = T2 * T;
  const float inv_T = 1.f / (float)T, inv_T2 = 1.f / (float)T2;
  const long long plane = (long long)n_f * n_f;
#pragma unroll 4
  for (int e = threadIdx.x; e < T3; e += blockDim.x) {
    const int jz = __float2int_rd(((float)e + 0.5f) * inv_T2);
    const int r = e - jz * T2;
    const int jy = __float2int_rd(((float)r + 0.5f) * inv_T);
    const int jx = r - jy * T;
    tile[jz * PZ + jy * PY + jx] = __ldg(grid + (long long)wrap_near(oz + jz, n_f) * plane +
                                         (long long)wrap_near(oy + jy, n_f) * n_f + wrap_near(ox + jx, n_f));
  }
}

// A6 (ik method): gather the potential and the three gradient grids with the
// SI weights alone; the gradients are already derivatives in physical units.
template <typename real, int P>
__global__ void __launch_bounds__(256) k_gather_ik(
    const SysDesc* __restrict__ sys, const int2* __restrict__ work,
    const typename Types<real>::atom* __restrict__ atoms, const uint32_t* __restrict__ start,
    const real* __restrict__ grids, const real* __restrict__ grids_ik, long long grid_total,
    typename Types<real>::res* __restrict__ far, const SICoef<real> si, int splits, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 wk = work[blockIdx.x / splits];
  const int split = blockIdx.x % splits;
  const SysDesc& S = sys[wk.x];
  const int nb = S.nb, T = S.T, n_f = S.n_f, bc = S.bc;
  const int b = wk.y;
  const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
  const int ox = tile_origin(S, bx, P, real()), oy = tile_origin(S, by, P, real()),
            oz = tile_origin(S, bz, P, real());
  const int PY = S.tpy, PZ = S.tpz;
  const int tsz = PZ * T;                                   // elements of one tile
  real* tile = reinterpret_cast<real*>(smem_raw);           // [4][tsz]: u, du/dx, du/dy, du/dz
  for (int g = 0; g < 4; ++g) {
    const real* grid = (g == 0 ? grids : grids_ik + (g - 1) * grid_total) + S.grid0;
    load_tile(tile + g * tsz, grid, T, PY, PZ, ox, oy, oz, n_f);
  }
  __syncthreads();
  const long long k0 = S.cell0 + (long long)b * bc * bc * bc * kSub;
  const uint32_t a_begin = start[k0], a_end = start[k0 + bc * bc * bc * kSub];
  for (uint32_t i = a_begin + split * blockDim.x + threadIdx.x; i < a_end; i += blockDim.x * splits) {
    const typename Types<real>::atom at = atoms[i];
    real yx, yy, yz;
    const int lx = stencil(S, at.x, P, yx) - ox;
    const int ly = stencil(S, at.y, P, yy) - oy;
    const int lz = stencil(S, at.z, P, yz) - oz;
    typename Types<real>::res out;
    if (lx < 0 || ly < 0 || lz < 0 || lx > T - P || ly > T - P || lz > T - P) {
      atomicOr(err, 2);
      out.x = out.y = out.z = out.w = real(0);
      far[i] = out;
      continue;
    }
    real wx[P], wy[P];
    si_weights<real, P, false>(si, yx, wx, nullptr);
    si_weights<real, P, false>(si, yy, wy, nullptr);
    real acc[4] = {0, 0, 0, 0};
#pragma unroll (Unroll<P>::outer)
    for (int c = 0; c < P; ++c) {
      real wzc, unused;
      si_weight_one<real, false>(si, c, yz, wzc, unused);
      real accc[4] = {0, 0, 0, 0};
#pragma unroll
      for (int bb = 0; bb < P; ++bb) {
        const int row = (lz + c) * PZ + (ly + bb) * PY + lx;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const real* r = tile + g * tsz + row;
          real sx = 0;
#pragma unroll
          for (int a = 0; a < P; ++a) sx += wx[a] * r[a];
          accc[g] += wy[bb] * sx;
        }
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) acc[g] += wzc * accc[g];
    }
    out.x = acc[0];
    out.y = acc[1];
    out.z = acc[2];
    out.w = acc[3];
    far[i] = out;
  }
}

// A6: gather (Eq. interp) with analytic-derivative forces.
template <typename real, int P>
__global__ void __launch_bounds__(256) k_gather(
    const SysDesc* __restrict__ sys, const int2* __restrict__ work,
    const typename Types<real>::atom* __restrict__ atoms, const uint32_t* __restrict__ start,
    const real* __restrict__ grids, typename Types<real>::res* __restrict__ far,
    const SICoef<real> si, int splits, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* tile = reinterpret_cast<real*>(smem_raw);
  const int2 wk = work[blockIdx.x / splits];
  const int split = blockIdx.x % splits;
  const SysDesc& S = sys[wk.x];
  const int nb = S.nb, T = S.T, n_f = S.n_f, bc = S.bc;
  const int b = wk.y;
  const int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
  const int ox = tile_origin(S, bx, P, real()), oy = tile_origin(S, by, P, real()),
            oz = tile_origin(S, bz, P, real());
  const int PY = S.tpy, PZ = S.tpz;
  const real* grid = grids + S.grid0;
  load_tile(tile, grid, T, PY, PZ, ox, oy, oz, n_f);
  __syncthreads();
  const long long k0 = S.cell0 + (long long)b * bc * bc * bc * kSub;
  const uint32_t a_begin = start[k0], a_end = start[k0 + bc * bc * bc * kSub];
  const real inv_h = (real)S.inv_h;
  for (uint32_t i = a_begin + split * blockDim.x + threadIdx.x; i < a_end; i += blockDim.x * splits) {
    const typename Types<real>::atom at = atoms[i];
    real yx, yy, yz;
    const int lx = stencil(S, at.x, P, yx) - ox;
    const int ly = stencil(S, at.y, P, yy) - oy;
    const int lz = stencil(S, at.z, P, yz) - oz;
    typename Types<real>::res out;
    if (lx < 0 || ly < 0 || lz < 0 || lx > T - P || ly > T - P || lz > T - P) {
      atomicOr(err, 2);
      out.x = out.y = out.z = out.w = real(0);
      far[i] = out;
      continue;
    }
    real wx[P], wy[P], dx[P], dy[P];
    si_weights<real, P, true>(si, yx, wx, dx);
    si_weights<real, P, true>(si, yy, wy, dy);
    real u = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll (Unroll<P>::outer)
    for (int c = 0; c < P; ++c) {
      real wzc, dzc;
      si_weight_one<real, true>(si, c, yz, wzc, dzc);
      real uc = 0, gxc = 0, gyc = 0;
#pragma unroll
      for (int bb = 0; bb < P; ++bb) {
        const real* row = tile + (lz + c) * PZ + (ly + bb) * PY + lx;
        real s0 = 0, s1 = 0;
#pragma unroll
        for (int a = 0; a < P; ++a) {
          const real v = row[a];
          s0 += wx[a] * v;
          s1 += dx[a] * v;
        }
        uc += wy[bb] * s0;
        gyc += dy[bb] * s0;
        gxc += wy[bb] * s1;
      }
      u += wzc * uc;
      gz += dzc * uc;
      gx += wzc * gxc;
      gy += wzc * gyc;
    }
    out.x = u;
    if (sizeof(real) == 4 && S.tri) {
      // triclinic cell: grad_r = n_f H^-T grad_t (H^-T lower triangular)
      const float* m = S.tgrad;
      out.y = gx * (real)m[0];
      out.z = gx * (real)m[1] + gy * (real)m[2];
      out.w = gx * (real)m[3] + gy * (real)m[4] + gz * (real)m[5];
    } else {
      out.y = gx * inv_h;
      out.z = gy * inv_h;
      out.w = gz * inv_h;
    }
    far[i] = out;
  }
}

// A7: local part (Eq. localpart). One thread per sorted atom i, in two
// phases that alternate at warp-uniform points:
//  scan   the atoms within r_c of i lie in the (2R+1)^2 columns of cells
//         around its cell (edge w >= r_c/R). Per neighbouring column the
//         lane computes the xy gap; a column no closer than r_c is skipped,
//         otherwise the z window of the cutoff sphere over the column is read
//         as one contiguous key range per brick it crosses (cells of a brick
//         column are consecutive, split into kSub z slabs). Each candidate is
//         tested with cheap cell-relative coordinates (FP32; absolute with
//         image shifts in FP64) and, if r < r_c, its index is queued.
//  pairs  when some lane's queue fills, every lane evaluates its queued pairs
//         with the minimum-image difference of the fixed-point coordinates
//         (int32 wrap; FP64: r - L rint(r/L)), so the pair work runs only for
//         pairs inside the cutoff and with most lanes busy.
template <typename real, int NC>
__device__ __forceinline__ real horner(const real* c, real y) {
  real v = c[NC - 1];
#pragma unroll
  for (int k = NC - 2; k >= 0; --k) v = v * y + c[k];
  return v;
}

__device__ inline float rsqrt_real(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_real(double x) { return 1.0 / sqrt(x); }
__device__ inline float sqrt_real(float x) { return sqrtf(x); }
__device__ inline double sqrt_real(double x) { return sqrt(x); }

constexpr int kMaxCellsAxis = 512;
constexpr int kMaxReach = 4;
constexpr int kTabPad = kMaxReach + 1;            // unwrapped cell indices -kTabPad ... n_c + kTabPad - 1
constexpr int kNearWarps = kChunk / 32;
constexpr int kQueueCap = 24;                      // pairs buffered per lane (queued variant)
constexpr int kQueueFlush = 12;                    // flush when a lane holds this many
constexpr size_t kNearQueueBytes = (size_t)kNearWarps * kQueueCap * 32 * sizeof(uint32_t);

struct NearTabs {
  int key[3][kMaxCellsAxis];                       // key parts per axis (brick-major, z fastest in brick)
  short wrap[kMaxCellsAxis + 2 * kTabPad];         // wrapped index of an unwrapped cell index
  short image[kMaxCellsAxis + 2 * kTabPad];        // periodic image of an unwrapped cell index
  short bend[kMaxCellsAxis + 2 * kTabPad];         // last unwrapped index in the same brick (z)
};

template <typename real>
__device__ __forceinline__ void pair_geometry(const SysDesc& S, const typename Types<real>::atom& ai,
                                              const typename Types<real>::atom& aj, real& dx, real& dy,
                                              real& dz) {
  if constexpr (sizeof(real) == 4) {
    const float sc = (float)S.fix_scale;
    dx = (float)(int)(ai.x - aj.x) * sc;         // int32 wrap = minimum image
    dy = (float)(int)(ai.y - aj.y) * sc;
    dz = (float)(int)(ai.z - aj.z) * sc;
  } else {
    dx = ai.x - aj.x; dx -= S.L * rint(dx * S.inv_L);
    dy = ai.y - aj.y; dy -= S.L * rint(dy * S.inv_L);
    dz = ai.z - aj.z; dz -= S.L * rint(dz * S.inv_L);
  }
}

template <typename real, int NC>
__device__ __forceinline__ void near_flush(const SysDesc& S, const typename Types<real>::atom& ai,
                                           const typename Types<real>::atom* __restrict__ atoms,
                                           const uint32_t* q, int cnt, const NearCoef<real>& nc,
                                           real rc2, real inv_rc, real inv_rc2x2, real inv_rc3,
                                           real& pot, real& fx, real& fy, real& fz) {
  const int m = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
  for (int k = 0; k < m; ++k) {
    if (k < cnt) {
      const uint32_t j = q[k * 32];
      const typename Types<real>::atom aj = atoms[j];
      real dx, dy, dz;
      pair_geometry<real>(S, ai, aj, dx, dy, dz);
      const real r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rc2 && r2 > real(0)) {
        const real rinv = rsqrt_real(r2);
        const real y = r2 * inv_rc2x2 - real(1);
        const real h = horner<real, NC>(nc.h, y);
        const real kk = horner<real, NC>(nc.k, y);
        const real qj = (real)atom_q(aj);
        pot += qj * (rinv - h * inv_rc);
        const real fs = qj * (rinv * rinv * rinv + kk * inv_rc3);
        fx += fs * dx;
        fy += fs * dy;
        fz += fs * dz;
      }
    }
  }
}

// VIR (inline form only): also the local virial, per atom 1/2 q_i sum_j
// fs_ij d d^T (every pair is met from both sides), summed over the warp and
// added to vloc[6 * system + c] with FP64 atomics.
template <typename real, int NC, bool QUEUE, bool VIR = false>
__global__ void __launch_bounds__(kChunk) k_near(
    const SysDesc* __restrict__ sys, const int2* __restrict__ chunks,
    const typename Types<real>::atom* __restrict__ atoms,
    const typename Types<real>::res* __restrict__ rel, const uint32_t* __restrict__ start,
    typename Types<real>::res* __restrict__ nearres, const NearCoef<real> nc,
    double* __restrict__ vloc = nullptr) {
  static_assert(!(QUEUE && VIR), "the virial is formed in the inline form");
  __shared__ NearTabs tabs;
  extern __shared__ __align__(16) uint32_t queue_mem[];   // [warp][kQueueCap][32]
  const int2 ch = chunks[blockIdx.x];
  const SysDesc& S = sys[ch.x];
  const int n_c = S.n_c, bc = S.bc, nb = S.nb, R = S.reach;
  for (int c = threadIdx.x; c < n_c; c += blockDim.x) {
    const int bq = c / bc, l = c - bq * bc;
    tabs.key[0][c] = bq * bc * bc * bc + l * bc * bc;
    tabs.key[1][c] = bq * nb * bc * bc * bc + l * bc;
    tabs.key[2][c] = bq * nb * nb * bc * bc * bc + l;
  }
  for (int u = threadIdx.x; u < n_c + 2 * kTabPad; u += blockDim.x) {
    const int zc = u - kTabPad;
    const int zz = ((zc % n_c) + n_c) % n_c;
    tabs.wrap[u] = (short)zz;
    tabs.image[u] = (short)((zc - zz) / n_c);
    tabs.bend[u] = (short)(zc + (bc - 1 - zz % bc));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t* q = queue_mem + (size_t)(threadIdx.x >> 5) * kQueueCap * 32 + lane;
  const int local = ch.y + threadIdx.x;
  const bool valid = local < S.n_atoms;
  const long long i = S.atom0 + (valid ? local : 0);
  const typename Types<real>::atom ai = atoms[i];
  int cx, cy, cz;
  atom_cell(S, ai, cx, cy, cz);
  const typename Types<real>::res ra = rel[i];
  const real w = (real)S.w;
  const real Lbox = (real)S.L;
  real xi, yi, zi;                                  // i relative to its own cell
  if constexpr (sizeof(real) == 8) {
    xi = ra.x - cx * S.w;
    yi = ra.y - cy * S.w;
    zi = ra.z - cz * S.w;
  } else {
    xi = ra.x;
    yi = ra.y;
    zi = ra.z - (real)(cz % bc) * w;
  }
  const real rc2 = (real)S.rc2, inv_rc = (real)S.inv_rc;
  const real inv_rc2x2 = real(2) * (real)S.inv_rc2, inv_rc3 = (real)S.inv_rc3;
  const real slab_per_len = real(kSub) / w;
  const real margin = real(1e-4) * w;          // guards the slab and column tests against rounding
  const real cull2 = rc2 + real(2) * margin * (real)S.r_c;
  const int slab_min = -R * kSub, slab_max = (R + 1) * kSub - 1;
  const uint32_t* st = start + S.cell0;
  real pot = 0, fx = 0, fy = 0, fz = 0;
  real vir[6] = {0, 0, 0, 0, 0, 0};
  int cnt = 0;
  for (int oy = -R; oy <= R; ++oy) {
    const int uy = cy + oy + kTabPad;
    const int yy = tabs.wrap[uy];
    const real gy = oy > 0 ? oy * w - yi : (oy < 0 ? yi - (oy + 1) * w : real(0));
    real sy;
    if constexpr (sizeof(real) == 8) sy = ra.y - Lbox * (real)tabs.image[uy];
    else sy = yi - oy * w;
    for (int ox = -R; ox <= R; ++ox) {
      const real gx = ox > 0 ? ox * w - xi : (ox < 0 ? xi - (ox + 1) * w : real(0));
      const real d2 = gx * gx + gy * gy;
      if (valid && d2 < cull2) {
        const real hz = sqrt_real(rc2 - (d2 < rc2 ? d2 : rc2)) + margin;
        const int ux = cx + ox + kTabPad;
        const int xx = tabs.wrap[ux];
        real sx;
        if constexpr (sizeof(real) == 8) sx = ra.x - Lbox * (real)tabs.image[ux];
        else sx = xi - ox * w;
        const int kxy = tabs.key[0][xx] + tabs.key[1][yy];
        int s_lo = (int)floor((zi - hz) * slab_per_len);
        int s_hi = (int)floor((zi + hz) * slab_per_len);
        s_lo = s_lo < slab_min ? slab_min : s_lo;
        s_hi = s_hi > slab_max ? slab_max : s_hi;
        const int oz_first = s_lo >> 2, oz_last = s_hi >> 2;     // kSub = 4
        for (int oz = oz_first; oz <= oz_last;) {
          const int uz = cz + oz + kTabPad;
          const int zz = tabs.wrap[uz];
          const int seg_last = min(oz_last, (int)tabs.bend[uz] - cz);
          const int sl_first = oz == oz_first ? s_lo - oz * kSub : 0;
          const int sl_last = seg_last == oz_last ? s_hi - seg_last * kSub : kSub - 1;
          const int k0 = kxy + tabs.key[2][zz];
          const uint32_t jb = st[(long long)k0 * kSub + sl_first];
          const uint32_t je = st[(long long)(k0 + seg_last - oz) * kSub + sl_last + 1];
          real sz;
          if constexpr (sizeof(real) == 8) sz = ra.z - Lbox * (real)tabs.image[uz];
          else sz = zi - (real)(oz - zz % bc) * w;            // frame of this brick column
          for (uint32_t j = jb; j < je; ++j) {
            const typename Types<real>::res rj = rel[j];
            const real dx = sx - rj.x, dy = sy - rj.y, dz = sz - rj.z;
            const real r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2 && r2 > real(0)) {
              if (!QUEUE) {
                // inline variant: evaluate the pair in the scan (masked lanes idle)
                const real rinv = rsqrt_real(r2);
                const real y = r2 * inv_rc2x2 - real(1);
                const real qj = rj.w;
                pot += qj * (rinv - horner<real, NC>(nc.h, y) * inv_rc);
                const real fs = qj * (rinv * rinv * rinv + horner<real, NC>(nc.k, y) * inv_rc3);
                fx += fs * dx;
                fy += fs * dy;
                fz += fs * dz;
                if constexpr (VIR) {
                  vir[0] += fs * dx * dx;
                  vir[1] += fs * dy * dy;
                  vir[2] += fs * dz * dz;
                  vir[3] += fs * dx * dy;
                  vir[4] += fs * dx * dz;
                  vir[5] += fs * dy * dz;
                }
              } else if (cnt < kQueueCap) {
                q[cnt * 32] = j;
                ++cnt;
              } else {
                // rare overflow: evaluate this pair at once
                const typename Types<real>::atom aj = atoms[j];
                real ex, ey, ez;
                pair_geometry<real>(S, ai, aj, ex, ey, ez);
                const real e2 = ex * ex + ey * ey + ez * ez;
                const real rinv = rsqrt_real(e2);
                const real y = e2 * inv_rc2x2 - real(1);
                const real qj = (real)atom_q(aj);
                pot += qj * (rinv - horner<real, NC>(nc.h, y) * inv_rc);
                const real fs = qj * (rinv * rinv * rinv + horner<real, NC>(nc.k, y) * inv_rc3);
                fx += fs * ex;
                fy += fs * ey;
                fz += fs * ez;
              }
            }
          }
          oz = seg_last + 1;
        }
      }
      if (QUEUE && __any_sync(0xffffffffu, cnt >= kQueueFlush)) {
        near_flush<real, NC>(S, ai, atoms, q, cnt, nc, rc2, inv_rc, inv_rc2x2, inv_rc3, pot, fx, fy, fz);
        cnt = 0;
      }
    }
  }
  if (QUEUE)
    near_flush<real, NC>(S, ai, atoms, q, cnt, nc, rc2, inv_rc, inv_rc2x2, inv_rc3, pot, fx, fy, fz);
  if constexpr (VIR) {
    const double w = valid ? 0.5 * (double)ra.w / kFourPi : 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double t = w * (double)vir[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) atomicAdd(vloc + 6 * ch.x + c, t);
    }
  }
  if (!valid) return;
  const real qi = ra.w;
  const real k4 = real(1.0 / kFourPi);
  typename Types<real>::res out;
  out.x = pot * k4;
  out.y = qi * fx * k4;
  out.z = qi * fy * k4;
  out.w = qi * fz * k4;
  nearres[i] = out;
}

template <typename Out> __device__ __forceinline__ Out out_cast(float v) {
  if constexpr (sizeof(Out) == 8) return f32_to_f64(v);
  else return (Out)v;
}

static __device__ void energy_of_system(int s, const SysDesc* __restrict__ sys, const EnergyArgs& ea,
                                        const double* __restrict__ partials, int n_chunks, double* red);

// A8: per-atom totals in the caller's order and energy partials; with
// ea.ticket set, the last CTA to finish (a ticket taken after its partials
// are written and fenced) also combines every system's energy.
// partials layout: [near chunk partials][gather chunk partials].
// (hi, lo) += (bh, bl) with the rounding error of hi + bh kept in lo
// (Knuth's TwoSum; exact for FP32 round-to-nearest without reassociation).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (bh - bp);
  hi = s;
  lo = lo + bl + err;
}

template <typename real, typename Out>
__global__ void __launch_bounds__(kChunk) k_finalize(
    const SysDesc* __restrict__ sys, const int2* __restrict__ chunks,
    const typename Types<real>::atom* __restrict__ atoms, const uint32_t* __restrict__ perm,
    const typename Types<real>::res* __restrict__ far, const typename Types<real>::res* __restrict__ nearres,
    Out* __restrict__ forces, Out* __restrict__ pot, double* __restrict__ partials, int n_chunks,
    const EnergyArgs ea) {
  __shared__ double red[32];
  __shared__ unsigned last_cta;
  const int2 ch = chunks[blockIdx.x];
  const SysDesc& S = sys[ch.x];
  const int local = ch.y + threadIdx.x;
  if constexpr (sizeof(real) == 4) {
    // FP32 mode: the far and near parts are FP32 sums, so their combination
    // stays in FP32 (FP64 arithmetic is scarce on this GPU); the energy
    // terms are summed without loss over the warp as FP32 (hi, lo) pairs
    // and over the block in FP64
    float en_hi = 0.f, en_lo = 0.f, eg_hi = 0.f, eg_lo = 0.f;
    if (local < S.n_atoms) {
      const long long i = S.atom0 + local;
      const float q = atom_q(atoms[i]);
      const typename Types<real>::res f = far ? far[i] : typename Types<real>::res{};
      const typename Types<real>::res nr = nearres[i];
      const uint32_t o = perm[i];
      const float pre = S.prefactor_f;
      if (forces) {
        forces[3ll * o + 0] = out_cast<Out>(pre * fmaf(-q, f.y, nr.y));
        forces[3ll * o + 1] = out_cast<Out>(pre * fmaf(-q, f.z, nr.z));
        forces[3ll * o + 2] = out_cast<Out>(pre * fmaf(-q, f.w, nr.w));
      }
      if (pot) pot[o] = out_cast<Out>(pre * (fmaf(-q, S.self_coef_f, f.x + nr.x) + S.bg_shift_f));
      en_hi = 0.5f * q * nr.x;
      eg_hi = 0.5f * q * f.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      two_sum_add(en_hi, en_lo, __shfl_xor_sync(0xffffffffu, en_hi, o), __shfl_xor_sync(0xffffffffu, en_lo, o));
      two_sum_add(eg_hi, eg_lo, __shfl_xor_sync(0xffffffffu, eg_hi, o), __shfl_xor_sync(0xffffffffu, eg_lo, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
      red[wid] = (double)en_hi + (double)en_lo;
      red[16 + wid] = (double)eg_hi + (double)eg_lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < nw; ++w) {
        a += red[w];
        b += red[16 + w];
      }
      partials[blockIdx.x] = a;
      partials[n_chunks + blockIdx.x] = b;
    }
  } else {
  double en = 0.0, eg = 0.0;
  if (local < S.n_atoms) {
    const long long i = S.atom0 + local;
    const typename Types<real>::atom at = atoms[i];
    const double q = (double)atom_q(at);
    const typename Types<real>::res f = far ? far[i] : typename Types<real>::res{};
    const typename Types<real>::res nr = nearres[i];
    const uint32_t o = perm[i];
    const double u = (double)f.x + (double)nr.x - q * S.self_coef + S.bg_shift;
    const double pre = S.prefactor;
    if (forces) {
      forces[3ll * o + 0] = (Out)(pre * (-q * (double)f.y + (double)nr.y));
      forces[3ll * o + 1] = (Out)(pre * (-q * (double)f.z + (double)nr.z));
      forces[3ll * o + 2] = (Out)(pre * (-q * (double)f.w + (double)nr.w));
    }
    if (pot) pot[o] = (Out)(pre * u);
    en = 0.5 * q * (double)nr.x;
    eg = 0.5 * q * (double)f.x;
  }
  en = block_sum(en, red);
  eg = block_sum(eg, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = en;
    partials[n_chunks + blockIdx.x] = eg;
  }
  }
  if (ea.ticket) {
    if (threadIdx.x == 0) {
      __threadfence();                               // this CTA's partials before its ticket
      last_cta = atomicAdd(ea.ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (last_cta) {
      __threadfence();
      for (int sy = 0; sy < ea.nsys; ++sy) energy_of_system(sy, sys, ea, partials, n_chunks, red);
      if (threadIdx.x == 0) *ea.ticket = 0u;         // ready for the next launch
    }
  }
}

// Exclusions: inv[perm[s]] = s, the sorted position of every caller index.
static __global__ void __launch_bounds__(256) k_inverse_perm(const uint32_t* __restrict__ perm,
                                                             uint32_t* __restrict__ inv, long long n) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) inv[perm[s]] = (uint32_t)s;
}

// Exclusions (one system): every listed pair (caller indices) loses its
// direct interaction q_i q_j / (4 pi r), which the local and spectral parts
// hold in full; the correction is added to the local-part results (sorted
// order) before the finalize, so potentials, forces and the energy all see
// it. The pair vector is the image nearest in wrapped fractional
// coordinates, the minimum image for pairs closer than half the smallest
// cell height.
template <typename real>
__global__ void __launch_bounds__(256) k_exclusions(
    const SysDesc* __restrict__ sys, const int2* __restrict__ pairs, long long n_pairs,
    const uint32_t* __restrict__ inv, const typename Types<real>::atom* __restrict__ atoms,
    typename Types<real>::res* __restrict__ nearres) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_pairs) return;
  const SysDesc& S = sys[0];
  const int2 pr = pairs[k];
  const uint32_t a = inv[pr.x], b = inv[pr.y];
  const typename Types<real>::atom A = atoms[a], B = atoms[b];
  real dx, dy, dz;
  if constexpr (sizeof(real) == 4) {
    if (S.tri) {
      // wrapped fractional difference, then H (cell vectors = n_c tcell)
      const double f = 2.3283064365386962890625e-10 * S.n_c;
      const double sx = (double)(int)(A.x - B.x) * f, sy = (double)(int)(A.y - B.y) * f,
                   sz = (double)(int)(A.z - B.z) * f;
      const double* e = S.tcell;
      dx = (float)(sx * e[0] + sy * e[1] + sz * e[3]);
      dy = (float)(sy * e[2] + sz * e[4]);
      dz = (float)(sz * e[5]);
    } else {
      pair_geometry<real>(S, A, B, dx, dy, dz);
    }
  } else {
    pair_geometry<real>(S, A, B, dx, dy, dz);
  }
  const real r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > real(0))) return;                    // coincident sites: nothing was added either
  const real rinv = real(1) / sqrt_real(r2);
  const real k4 = real(1.0 / kFourPi);
  const real qa = (real)atom_q(A), qb = (real)atom_q(B);
  const real fs = qa * qb * rinv * rinv * rinv * k4;   // pair force on a is +fs d: removed
  if constexpr (sizeof(real) == 4) {
    atomicAdd(nearres + a, make_float4(-qb * rinv * k4, -fs * dx, -fs * dy, -fs * dz));
    atomicAdd(nearres + b, make_float4(-qa * rinv * k4, fs * dx, fs * dy, fs * dz));
  } else {
    atomicAdd(&nearres[a].x, -qb * rinv * k4);
    atomicAdd(&nearres[a].y, -fs * dx);
    atomicAdd(&nearres[a].z, -fs * dy);
    atomicAdd(&nearres[a].w, -fs * dz);
    atomicAdd(&nearres[b].x, -qa * rinv * k4);
    atomicAdd(&nearres[b].y, fs * dx);
    atomicAdd(&nearres[b].z, fs * dy);
    atomicAdd(&nearres[b].w, fs * dz);
  }
}

// Compensated (Neumaier) sum of a strided range, then a pairwise block tree.
__device__ inline void neumaier_add(double& s, double& c, double v) {
  double t = s + v;
  if (fabs(s) >= fabs(v)) c += (s - t) + v; else c += (v - t) + s;
  s = t;
}

// Per-system energy: E = prefactor (E_fourier + E_near + E_self + E_bg).
// One block of 1024 threads per system. out[3 s + 0] = E, [1] = E_fourier, [2] = E_gather.
// The energy of system s from the partials of the scale and finalize
// kernels (and its virial), by the calling CTA: a few plain FP64 additions
// per thread, then a pairwise tree over the CTA (the rounding error stays
// near log2(terms) ulp, and the FP64 work is small: FP64 is scarce on this
// GPU); the four parts are combined with compensation. The partials are
// read through L2 (the finalize kernel's own CTAs may have just written
// them).
static __device__ void energy_of_system(int s, const SysDesc* __restrict__ sys, const EnergyArgs& ea,
                                        const double* __restrict__ partials, int n_chunks, double* red) {
  double vs[3] = {0, 0, 0};
  for (int j = threadIdx.x; j < ea.n_fourier_blocks; j += blockDim.x)
    vs[0] += ea.fourier[(long long)s * ea.n_fourier_blocks + j];
  for (int j = ea.chunk_first[s] + threadIdx.x; j < ea.chunk_first[s + 1]; j += blockDim.x) {
    vs[1] += __ldcg(partials + j);
    vs[2] += __ldcg(partials + n_chunks + j);
  }
  double tot[3];
  for (int a = 0; a < 3; ++a) tot[a] = block_sum(vs[a], red);
  if (threadIdx.x == 0) {
    const double pre = sys[s].prefactor;
    // consts[2 s] = E_self, consts[2 s + 1] = E_bg (host FP64)
    double acc = 0.0, cc = 0.0;
    neumaier_add(acc, cc, tot[0]);
    neumaier_add(acc, cc, tot[1]);
    neumaier_add(acc, cc, ea.consts[2 * s]);
    neumaier_add(acc, cc, ea.consts[2 * s + 1]);
    const double e = pre * (acc + cc);
    ea.out[3 * s + 0] = e;
    ea.out[3 * s + 1] = pre * tot[0];
    ea.out[3 * s + 2] = pre * tot[2];
    if (ea.user_energy) ea.user_energy[s] = e;
  }
  if (ea.vout) {
    // virial: spectral partials, local sums, background energy on the diagonal
    for (int c = 0; c < 6; ++c) {
      double v = 0.0;
      for (int j = threadIdx.x; j < ea.n_fourier_blocks; j += blockDim.x)
        v += ea.vpart[((long long)s * ea.n_fourier_blocks + j) * 6 + c];
      v = block_sum(v, red);
      if (threadIdx.x == 0)
        ea.vout[6 * s + c] = sys[s].prefactor * (v + ea.vloc[6 * s + c] + (c < 3 ? ea.consts[2 * s + 1] : 0.0));
    }
  }
}

// One CTA per system.
static __global__ void __launch_bounds__(1024) k_energy(const SysDesc* __restrict__ sys, const EnergyArgs ea,
                                                        const double* __restrict__ partials, int n_chunks) {
  __shared__ double red[32];
  energy_of_system(blockIdx.x, sys, ea, partials, n_chunks, red);
}

}  // namespace espk
