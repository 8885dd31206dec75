// Device code of the ESP solve (sm_103a). Every kernel works on a pool of one
// or more independent systems described by SysDesc records, so the same code
// serves a single system and a batch of systems.
//
// Pipeline (paper, Methods; one pass per esp_compute):
//   ingest   wrap positions into the box, fixed-point (FP32 mode) or wrapped
//            FP64 coordinates, cell key and rank within the cell
//   scan     exclusive scan of the per-cell counts (cell list offsets)
//   scatter  counting-sort scatter: sorted atoms (coords + charge), permutation
//   spread   Eq. spread: b_l = sum_j q_j phi~(r_j - h l), one CTA per brick of
//            cells accumulating into a shared-memory tile with a P-1 halo,
//            flushed to the periodic grid with global atomics
//   R2C FFT  cuFFT (library)
//   scale    Eq. pk: ch_k = p_k bh_k, p_k = G[|k|^2] w[kx] w[ky] w[kz], fused
//            with the spectral energy 1/2 sum_k p_k |bh_k|^2
//   C2R FFT  cuFFT (library)
//   gather   Eq. interp: u~_i and grad u~_i (analytic derivatives of the
//            piecewise polynomials), same tile structure, read-only
//   near     Eq. localpart: cell-list pair sum within r_c, L(r) and -L'(r)
//            from polynomials in x = r / r_c
//   finalize self term, background, per-atom totals in the caller's order,
//            energy partials
//   reduce   compensated FP64 energy per system
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace espk {

constexpr int kMaxP = 16;
constexpr int kMinP = 4;
constexpr int kChunk = 256;   // atoms per chunk = threads of a per-atom block

// Polynomial degrees (coefficient counts) per precision.
template <typename real> struct Deg;
template <> struct Deg<float> { static constexpr int si = 10; static constexpr int nr = 12; };
template <> struct Deg<double> { static constexpr int si = 18; static constexpr int nr = 24; };

// Each cell-list cell is split into kSub slabs along z; atoms are sorted by
// (cell, slab), so the local part reads only the slabs a cutoff sphere meets.
constexpr int kSub = 4;

// Atoms per i-cluster of the FP32 local part (host-visible for buffer sizes).
constexpr int kClusterAtomsHost = 8;

// SI kernel: P pieces, piece a gives the weight of grid point l0 + a as a
// polynomial in y = 2 delta - 1, delta = t - l0 - (P/2 - 1) in (0, 1].
template <typename real> struct SICoef { real c[kMaxP][Deg<real>::si]; };
// Local part L(r) = (1 - g(r/r_c)) / (4 pi r) written as bare Coulomb minus a
// smooth correction. With x = r/r_c and s = x^2 (g is odd and chi even, so
// both corrections are even in x, i.e. polynomials in s):
//   4 pi L(r)          = 1/r - H(s)/r_c,          H(s) = g(x)/x,
//   -4 pi L'(r) / r    = 1/r^3 + K(s)/r_c^3,      K(s) = (x chi(x) - g(x))/x^3,
// both as polynomials in y = 2 s - 1.
template <typename real> struct NearCoef { real h[Deg<real>::nr]; real k[Deg<real>::nr]; };

// Per-system geometry and constants (same record on host and device).
struct SysDesc {
  int n_f;        // grid points per axis
  int n_c;        // cell-list cells per axis (cell edge >= r_c / 2)
  int bc;         // cells per brick edge (n_c % bc == 0)
  int nb;         // bricks per axis (n_c / bc)
  int T;          // shared tile edge in grid points
  int tpy, tpz;   // tile row and plane pitch in elements (tile_pitches)
  int n_atoms;
  int gsize;      // entries of the radial table G (3 (n_f/2)^2 + 1)
  int reach;      // neighbour cells per side in the local part (edge w >= r_c / reach)
  long long atom0;   // first atom of the system in the pooled atom arrays
  long long cell0;   // first entry of the system in the pooled count/start arrays
                     // (arrays indexed by cell key * kSub + slab)
  long long grid0;   // first element of the system's real grid
  long long spec0;   // first element of the system's half spectrum
  long long tab0;    // first element of the system's G table (w follows G)
  long long col0;    // first cell-list column (cx, cy) of the system in pooled column arrays
  double L, inv_L, h, inv_h;
  double r_c, rc2, inv_rc, inv_rc2, inv_rc3;
  double w;          // cell edge L / n_c
  double fix_scale;  // L / 2^32
  double to_fixed;   // 2^32 / L
  // 2^32 / L as fix_m 2^fix_e (fix_m: 64 bits, top bit set, rounded down):
  // the FP32 ingest's exact integer conversion to fixed point
  unsigned long long fix_m;
  int fix_e;
  double w32;        // w / 2^32
  double self_coef;  // chi(0) / (4 pi r_c)
  double bg_shift;   // -(Q/V) (r_c^2/2) int_0^1 x^2 chi
  double prefactor;
  // FP32 copies for the FP32 local part
  float wf, r_cf, rc2f, inv_rcf, inv_rc2x2f, inv_rc3f, inv_bcf;
  float w32f;                       // wf / 2^32 (exact)
  float self_coef_f, bg_shift_f, prefactor_f;
  double vol;                       // cell volume (L^3 for a cube)
  // Triclinic cell (tri = 1): H = [a b c] with a = (ax,0,0), b = (bx,by,0),
  // c = (cx,cy,cz); the grid, cells and fixed-point coordinates are laid over
  // fractional coordinates s = H^-1 r. Unused when tri = 0.
  int tri;
  double tfix[6];   // 2^32 H^-1: (xx, xy, xz, yy, yz, zz) entries of the upper triangle
  double tcell[6];  // cell vectors / n_c: a_x, b_x, b_y, c_x, c_y, c_z
  float tgrad[6];   // n_f H^-T (lower triangle): (xx, yx, yy, zx, zy, zz)
  float tcol[3];    // a_x, b_x, b_y over n_c: offsets of neighbouring columns
  float tbrick[3];  // bc c / n_c: offset of one brick up the column
};

// Padded pitches of a spread/gather tile of edge T (elements): rows of odd
// length, and a plane pitch equal to P rows modulo 32, so that the P x P rows
// of one stencil (lane r = P z + y) start on banks r * py mod 32, all
// distinct. Unpadded, a tile of edge 16 put every row of a stencil on two
// banks.
__host__ __device__ inline void tile_pitches(int T, int P, int& py, int& pz) {
  py = T | 1;
  pz = py * T;
  const int want = (P * py) & 31;
  while ((pz & 31) != want) ++pz;
}

// ------------------------------------------------------------ coordinates
// FP32 mode stores coordinates as 32-bit fixed-point fractions of L: the grid
// index of the stencil origin is then exact integer arithmetic and pair
// differences are exact integer differences (minimum image = int32 wrap).
// u = floor(x S) mod 2^32 for S = fix_m 2^fix_e, in integer arithmetic on the
// bits of the double x = m 2^E (m the 53-bit significand): x S = (m fix_m)
// 2^(E + fix_e), the 117-bit product formed exactly and shifted; a negative x
// rounds down (one less when a fraction remains). No FP64 instruction: FP64
// units are scarce on this GPU. x must be finite.
__device__ __forceinline__ uint32_t fixed_from_double(double x, unsigned long long fix_m, int fix_e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
  const int sh = (ex ? ex : 1) - 1075 + fix_e;         // x S = (hi:lo) 2^sh
  const unsigned long long lo = m * fix_m, hi = __umul64hi(m, fix_m);
  uint32_t ip;                                          // floor(|x| S) mod 2^32
  bool frac;                                            // |x| S is not an integer
  if (sh >= 0) {
    ip = sh >= 32 ? 0u : (uint32_t)(lo << sh);
    frac = false;
  } else {
    const int r = -sh;
    if (r >= 128) {
      ip = 0u;
      frac = (hi | lo) != 0ull;
    } else if (r >= 64) {
      ip = (uint32_t)(hi >> (r - 64));
      frac = lo != 0ull || (r > 64 && (hi << (128 - r)) != 0ull);
    } else {
      ip = (uint32_t)((lo >> r) | (hi << (64 - r)));
      frac = (lo << (64 - r)) != 0ull;
    }
  }
  return (bits >> 63) ? 0u - ip - (frac ? 1u : 0u) : ip;
}

__host__ __device__ inline void stencil_fixed(uint32_t u, int n_f, int P, int& l0, int64_t& r) {
  // t = u n_f / 2^32 (32.32 fixed point); l0 = ceil(t - P/2);
  // r = (t - l0 - P/2 + 1) * 2^32 in (0, 2^32]
  int64_t v = (int64_t)((uint64_t)u * (uint64_t)n_f) - ((int64_t)P << 31);
  int64_t l = (v + 0xFFFFFFFFLL) >> 32;   // arithmetic shift: ceil(v / 2^32)
  l0 = (int)l;
  r = v - (l << 32) + (1LL << 32);
}

__host__ __device__ inline uint32_t cell_min_fixed(int c, int n_c) {
  // smallest u with (u n_c) >> 32 == c
  return (uint32_t)((((uint64_t)c << 32) + (uint64_t)n_c - 1) / (uint64_t)n_c);
}

__host__ __device__ inline int tile_origin_fixed(int cb, int n_c, int n_f, int P) {
  int l0; int64_t r;
  stencil_fixed(cell_min_fixed(cb, n_c), n_f, P, l0, r);
  return l0;
}

__host__ __device__ inline int tile_last_fixed(int cb_end, int n_c, int n_f, int P) {
  // l0 of the largest u below cell cb_end
  uint64_t umax = (cb_end >= n_c) ? 0xFFFFFFFFull : (uint64_t)cell_min_fixed(cb_end, n_c) - 1;
  int l0; int64_t r;
  stencil_fixed((uint32_t)umax, n_f, P, l0, r);
  return l0;
}

// FP64 mode keeps wrapped FP64 coordinates; the grid coordinate is computed as
// t = (x / L) n_f (IEEE division, then product) so that the measure-zero tie
// t - P/2 in Z is decided by the same rounding as in the FP64 reference.
__host__ __device__ inline int stencil_origin_f64(double x, double L, int n_f, int P, double& delta) {
  double t = (x / L) * (double)n_f;
  double l0 = ceil(t - 0.5 * P);
  delta = t - l0 - 0.5 * P + 1.0;
  return (int)l0;
}

__host__ __device__ inline int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}
// The same for indices within a few periods of [0, n) (tile points around a
// brick): additions instead of an integer division.
__host__ __device__ inline int wrap_near(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// Arguments of the per-system energy combination (the four energy parts,
// optional virial): see launch_energy. ticket: a counter that is zero between
// launches; when set, the finalize kernel's last CTA does the combination.
struct EnergyArgs {
  int nsys = 0;
  const double* fourier = nullptr;
  int n_fourier_blocks = 0;
  const int* chunk_first = nullptr;
  const double* consts = nullptr;
  double* out = nullptr;
  double* user_energy = nullptr;
  const double* vpart = nullptr;
  const double* vloc = nullptr;
  double* vout = nullptr;
  unsigned* ticket = nullptr;
};

// Exact float -> double by bit manipulation (the double has the float's
// value: sign, exponent rebiased, significand widened; a subnormal float
// becomes a normal double), without an FP64 conversion instruction (FP64
// units are scarce on this GPU).
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  unsigned long long r;
  if (e == 0xffu) {
    r = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);            // inf, NaN
  } else if (e != 0u) {
    r = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    r = sign;                                                                 // +-0
  } else {
    const int lz = __clz((int)m) - 8;                   // top bit of m moves to bit 23
    const unsigned long long mm = (unsigned long long)((m << lz) & 0x7fffffu);
    r = sign | ((unsigned long long)(897 - lz) << 52) | (mm << 29);
  }
  return __longlong_as_double((long long)r);
}
// --------------------------------------------------------------- reductions
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
__device__ inline double block_sum(double v, double* smem32) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) smem32[wid] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

}  // namespace espk
