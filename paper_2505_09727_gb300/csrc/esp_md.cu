// MD loop around the solve: velocity Verlet for flexible SPC/E-shaped water
// with ESP electrostatics (the plan, with the intramolecular pairs excluded),
// harmonic O-H bonds and H-O-H angle, and O-O Lennard-Jones within a cutoff,
// shifted to zero there. Molecules are consecutive (O, H, H) triples of the
// plan's atoms; positions, velocities and forces stay on the device in FP64,
// caller order. One step: kick + drift, esp_step on the device positions
// (sort and compute replayed as one graph) and, beside it on a second
// stream, the bonded and Lennard-Jones forces into a second buffer, then the
// kick on their sum with the kinetic energy summed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/esp.h"
#include "esp_engine.h"
#include "esp_launch.h"

struct esp_md_s {
  esp_plan_t plan = nullptr;
  esp_md_params prm{};
  int device = 0;
  long long n_atoms = 0;
  int n_mol = 0;
  double L = 0.0;
  int nc = 0;                      // Lennard-Jones cells per axis (0: all pairs)
  bool fp32 = true;                // the plan's precision (the Lennard-Jones pairs follow it)
  bool have_forces = false;
  double* d_x = nullptr;
  double* d_v = nullptr;
  double* d_f = nullptr;           // forces of the solve (Coulomb)
  double* d_f2 = nullptr;          // bonded and Lennard-Jones forces
  cudaStream_t st3 = nullptr;      // the bonded and Lennard-Jones terms, beside the solve
  cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
  double* d_e = nullptr;           // energies [(capacity) x 4]
  double* d_ecur = nullptr;        // energies of the step in progress (Coulomb, bonded, LJ, kinetic)
  int* d_row = nullptr;            // next row of d_e the step writes
  long long e_cap = 0;
  cudaGraph_t graph = nullptr;     // one velocity-Verlet step, replayed n times
  cudaGraphExec_t gexec = nullptr;
  const double* graph_e = nullptr; // the d_e the graph was captured with
  long long graph_cap = 0;         // and its row capacity (a reallocation may return the same address)
  double e_now[4] = {0, 0, 0, 0};  // energies at the current positions
  uint32_t *d_cell = nullptr, *d_count = nullptr, *d_start = nullptr, *d_tiles = nullptr, *d_cursor = nullptr,
           *d_sorted = nullptr;
  double* d_opos = nullptr;        // packed O positions (4 values of the plan's precision per O)
  std::vector<void*> allocs;
};

namespace {

constexpr double kPiMd = 3.14159265358979323846;

esp_status md_fail(esp_status s, const std::string& msg) {
  espe::set_last_error(msg);
  return s;
}

#define MD_CU(call)                                                                               \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return md_fail(ESP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct MdConst {
  double dt, k_bond, r0, k_angle, theta0, sigma2, eps4, rc2, shift, inv_mO, inv_mH, L, inv_L;
  double mO, mH;                                              // masses (kinetic energy)
  float k_bond_f, r0_f, k_angle_f, theta0_f, L_f, inv_L_f;   // FP32 copies (FP32 bonded terms)
  int n_mol, nc;
};

__device__ __forceinline__ double wrap_d(double d, double L, double inv_L) { return d - L * rint(d * inv_L); }

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block added to *out (blockDim.x a multiple of 32).
__device__ void block_add(double v, double* out) {
  __shared__ double red[32];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum_d(v);
    if (lane == 0) atomicAdd(out, v);
  }
}

// The FP32 sum of v over the block added to *out with one FP64 atomic.
__device__ void block_add_f(float v, double* out) {
  __shared__ float redf[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) redf[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? redf[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(out, espk::f32_to_f64(v));
  }
}

__device__ __forceinline__ double inv_mass(const MdConst& C, long long i) { return i % 3 == 0 ? C.inv_mO : C.inv_mH; }

// v += dt F / 2m; r += dt v (F = f + f2)
__global__ void k_kick_drift(double* __restrict__ x, double* __restrict__ v, const double* __restrict__ f,
                             const double* __restrict__ f2, MdConst C, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double h = 0.5 * C.dt * inv_mass(C, i);
  for (int a = 0; a < 3; ++a) {
    const double vv = v[3 * i + a] + h * (f[3 * i + a] + f2[3 * i + a]);
    v[3 * i + a] = vv;
    x[3 * i + a] += C.dt * vv;
  }
}

// v += dt F / 2m (scale 1) or nothing (scale 0), F = f + f2; the kinetic
// energy added to *ek
__global__ void k_kick(double* __restrict__ v, const double* __restrict__ f, const double* __restrict__ f2,
                       MdConst C, long long n, double scale, double* __restrict__ ek) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n) {
    const bool is_o = i % 3 == 0;
    const double im = is_o ? C.inv_mO : C.inv_mH, mass = is_o ? C.mO : C.mH;
    const double h = 0.5 * C.dt * im * scale;
    for (int a = 0; a < 3; ++a) {
      const double vv = v[3 * i + a] + h * (f[3 * i + a] + f2[3 * i + a]);
      v[3 * i + a] = vv;
      e += 0.5 * mass * vv * vv;                       // (no FP64 division)
    }
  }
  block_add(e, ek);
}

// End of a step: the step's energies become row *row of e (when it exists),
// the accumulators are cleared and the row advances.
__global__ void k_commit(double* __restrict__ ecur, double* __restrict__ e, int* __restrict__ row, long long cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int r = *row;
    if (r < cap)
      for (int c = 0; c < 4; ++c) e[4ll * r + c] = ecur[c];
    for (int c = 0; c < 4; ++c) ecur[c] = 0.0;
    *row = r + 1;
  }
}

// Bonds and angle of one molecule per thread, stored into f (the first
// writer of the step's bonded and Lennard-Jones forces); energy to *eb.
// F32 (FP32 plans): the O-H differences in FP64, the rest in FP32 (FP64
// units are scarce on this GPU; the FP32 Coulomb forces set the precision of
// such a step).
template <bool F32>
__global__ void k_bonded(const double* __restrict__ x, double* __restrict__ f, MdConst C, double* __restrict__ eb) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (F32) {
    float e = 0.f;
    if (m < C.n_mol) {
      const double* o = x + 9ll * m;
      float d[2][3], r[2], fh[2][3];
      for (int k = 0; k < 2; ++k) {
        for (int a = 0; a < 3; ++a) {
          const float t = (float)(o[3 * (k + 1) + a] - o[a]);
          d[k][a] = t - C.L_f * rintf(t * C.inv_L_f);
        }
        r[k] = sqrtf(d[k][0] * d[k][0] + d[k][1] * d[k][1] + d[k][2] * d[k][2]);
        const float dr = r[k] - C.r0_f;
        e += 0.5f * C.k_bond_f * dr * dr;
        for (int a = 0; a < 3; ++a) fh[k][a] = -C.k_bond_f * dr / r[k] * d[k][a];
      }
      float c = (d[0][0] * d[1][0] + d[0][1] * d[1][1] + d[0][2] * d[1][2]) / (r[0] * r[1]);
      c = fminf(1.f, fmaxf(-1.f, c));
      const float th = acosf(c);
      const float sn = sqrtf(fmaxf(1.f - c * c, 1e-30f));
      const float de = C.k_angle_f * (th - C.theta0_f);
      e += 0.5f * C.k_angle_f * (th - C.theta0_f) * (th - C.theta0_f);
      for (int a = 0; a < 3; ++a) {
        const float dtu = -(d[1][a] / (r[0] * r[1]) - c / (r[0] * r[0]) * d[0][a]) / sn;
        const float dtv = -(d[0][a] / (r[0] * r[1]) - c / (r[1] * r[1]) * d[1][a]) / sn;
        fh[0][a] -= de * dtu;
        fh[1][a] -= de * dtv;
      }
      double* fo = f + 9ll * m;
      for (int a = 0; a < 3; ++a) {
        fo[3 + a] = espk::f32_to_f64(fh[0][a]);
        fo[6 + a] = espk::f32_to_f64(fh[1][a]);
        fo[a] = espk::f32_to_f64(-(fh[0][a] + fh[1][a]));
      }
    }
    block_add_f(e, eb);
  } else {
    double e = 0.0;
    if (m < C.n_mol) {
      const double* o = x + 9ll * m;
      double d[2][3], r[2];
      double fh[2][3];
      for (int k = 0; k < 2; ++k) {
        for (int a = 0; a < 3; ++a) d[k][a] = wrap_d(o[3 * (k + 1) + a] - o[a], C.L, C.inv_L);
        r[k] = sqrt(d[k][0] * d[k][0] + d[k][1] * d[k][1] + d[k][2] * d[k][2]);
        const double dr = r[k] - C.r0;
        e += 0.5 * C.k_bond * dr * dr;
        for (int a = 0; a < 3; ++a) fh[k][a] = -C.k_bond * dr / r[k] * d[k][a];
      }
      double c = (d[0][0] * d[1][0] + d[0][1] * d[1][1] + d[0][2] * d[1][2]) / (r[0] * r[1]);
      c = fmin(1.0, fmax(-1.0, c));
      const double th = acos(c);
      const double sn = sqrt(fmax(1.0 - c * c, 1e-300));
      const double de = C.k_angle * (th - C.theta0);
      e += 0.5 * C.k_angle * (th - C.theta0) * (th - C.theta0);
      // d theta / d u = -(v / (|u||v|) - cos u / |u|^2) / sin theta, likewise for v
      for (int a = 0; a < 3; ++a) {
        const double dtu = -(d[1][a] / (r[0] * r[1]) - c / (r[0] * r[0]) * d[0][a]) / sn;
        const double dtv = -(d[0][a] / (r[0] * r[1]) - c / (r[1] * r[1]) * d[1][a]) / sn;
        fh[0][a] -= de * dtu;
        fh[1][a] -= de * dtv;
      }
      double* fo = f + 9ll * m;
      for (int a = 0; a < 3; ++a) {
        fo[3 + a] = fh[0][a];
        fo[6 + a] = fh[1][a];
        fo[a] = -(fh[0][a] + fh[1][a]);
      }
    }
    block_add(e, eb);
  }
}

__device__ __forceinline__ int lj_cell_axis(double s, int nc) {
  s -= floor(s);
  const int c = (int)(s * nc);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Oxygen cells: cell of every molecule's O and the per-cell counts.
__global__ void k_lj_bin(const double* __restrict__ x, MdConst C, uint32_t* __restrict__ cell,
                         uint32_t* __restrict__ count) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= C.n_mol) return;
  const double* o = x + 9ll * m;
  const int cx = lj_cell_axis(o[0] * C.inv_L, C.nc), cy = lj_cell_axis(o[1] * C.inv_L, C.nc),
            cz = lj_cell_axis(o[2] * C.inv_L, C.nc);
  const uint32_t k = (uint32_t)((cx * C.nc + cy) * C.nc + cz);
  cell[m] = k;
  atomicAdd(count + k, 1u);
}

__global__ void k_lj_fill(const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
                          uint32_t* __restrict__ cursor, uint32_t* __restrict__ sorted, int n_mol) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_mol) return;
  const uint32_t k = cell[m];
  sorted[start[k] + atomicAdd(cursor + k, 1u)] = (uint32_t)m;
}

// O positions in cell order (cells) or molecule order (no cells), packed
// as (x, y, z, molecule) in the precision of the plan, for coalesced reads.
template <typename real> struct __align__(4 * sizeof(real)) OPos { real x, y, z, m; };

template <typename real>
__global__ void k_lj_pack(const double* __restrict__ x, const uint32_t* __restrict__ sorted, int use_cells,
                          int n_mol, MdConst C, OPos<real>* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_mol) return;
  const int m = use_cells ? (int)sorted[s] : s;
  const double* o = x + 9ll * m;
  // wrapped into [0, L): with cells, a neighbouring cell's image shift is
  // then +-L or 0 along each axis
  double w[3];
  for (int a = 0; a < 3; ++a) {
    w[a] = o[a] - C.L * floor(o[a] * C.inv_L);
    if (w[a] >= C.L) w[a] -= C.L;
  }
  out[s] = OPos<real>{(real)w[0], (real)w[1], (real)w[2], (real)m};
}

// One O-O pair seen from i, in the precision of the plan (FP32 plans: FP32
// coordinates and arithmetic, as the solve's own pair terms). d = x_i - x_j
// with the minimum image taken by `rint` (no cells) or by the neighbouring
// cell's shift sh (cells; wrapped positions).
// The Lennard-Jones constants in the plan's precision, converted once per
// thread (FP64 conversions are slow on this GPU).
template <typename real> struct LjC {
  real L, inv_L, rc2, sigma2, eps4, shift;
  __device__ explicit LjC(const MdConst& C)
      : L((real)C.L), inv_L((real)C.inv_L), rc2((real)C.rc2), sigma2((real)C.sigma2), eps4((real)C.eps4),
        shift((real)C.shift) {}
};

// One candidate pair; the O itself (self) and pairs outside (0, r_c)
// contribute nothing.
template <typename real, bool CELLS>
__device__ __forceinline__ void lj_pair(const real* xi, const OPos<real>& pj, const real* sh, const LjC<real>& C,
                                        bool self, real* fi, real& e) {
  const real xj[3] = {pj.x, pj.y, pj.z};
  real d[3];
  for (int a = 0; a < 3; ++a) {
    const real t = xi[a] - xj[a];
    if constexpr (CELLS) d[a] = t + sh[a];
    else d[a] = t - C.L * rint(t * C.inv_L);
  }
  const real r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (self || r2 >= C.rc2 || r2 <= real(0)) return;
  const real inv_r2 = real(1) / r2;
  const real s2 = C.sigma2 * inv_r2, s6 = s2 * s2 * s2;
  e += real(0.5) * (C.eps4 * (s6 * s6 - s6) - C.shift);   // every pair is met from both sides
  const real fm = real(6) * C.eps4 * (real(2) * s6 * s6 - s6) * inv_r2;
  fi[0] += fm * d[0];
  fi[1] += fm * d[1];
  fi[2] += fm * d[2];
}

// O-O Lennard-Jones, one warp per O (taken in cell order, so the warps of a
// block read the same neighbouring cells): the lanes stride over the
// candidates of the neighbouring cells (cell edge >= cutoff) that the cutoff
// sphere reaches, or of every O when there are fewer than 3 cells per axis;
// sums over the warp.
template <typename real>
__global__ void k_lj(const OPos<real>* __restrict__ op, const uint32_t* __restrict__ cell,
                     const uint32_t* __restrict__ start, MdConst C, double* __restrict__ f,
                     double* __restrict__ el) {
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const LjC<real> LC(C);
  real e = 0;
  if (w < C.n_mol) {
    const OPos<real> pi = op[w];
    const int m = (int)pi.m;
    const real xi[3] = {pi.x, pi.y, pi.z};
    real fi[3] = {0, 0, 0};
    if (C.nc >= 3) {
      const int nc = C.nc;
      const int k = (int)cell[m];
      const int cz = k % nc, cy = (k / nc) % nc, cx = k / (nc * nc);
      auto wrap = [&](int u) { return u < 0 ? u + nc : (u >= nc ? u - nc : u); };
      auto shift = [&](int u) { return u < 0 ? LC.L : (u >= nc ? -LC.L : real(0)); };
      // the z-neighbouring cells of a column (nx, ny) are consecutive in cell
      // order: one range, or two where the column wraps in z
      auto sweep = [&](uint32_t b, uint32_t e2, const real* sh) {
        for (uint32_t s = b + lane; s < e2; s += 32) lj_pair<real, true>(xi, op[s], sh, LC, s == (uint32_t)w, fi, e);
      };
      // the O's place in its cell; a column whose xy gap from the O is >= the
      // cutoff is skipped, and a column's z range keeps the cells the cutoff
      // sphere reaches over that gap (a small margin keeps the cull
      // conservative where the FP64 cell and the wrapped position disagree
      // by a rounding)
      const real cw = LC.L / (real)nc, margin = real(1e-4) * cw;
      const real fx = xi[0] - (real)cx * cw, fy = xi[1] - (real)cy * cw, fz = xi[2] - (real)cz * cw;
      auto gap = [&](int o, real f) {
        const real g = o == 0 ? real(0) : (o < 0 ? f : cw - f);
        return g > margin ? g - margin : real(0);
      };
      const real glo = gap(-1, fz), ghi = gap(1, fz);
      for (int ox = -1; ox <= 1; ++ox)
        for (int oy = -1; oy <= 1; ++oy) {
          const real gx = gap(ox, fx), gy = gap(oy, fy);
          const real h2 = LC.rc2 - gx * gx - gy * gy;
          if (h2 <= real(0)) continue;
          const int lo = glo * glo < h2 ? cz - 1 : cz;
          const int hi = ghi * ghi < h2 ? cz + 1 : cz;
          const int ux = cx + ox, uy = cy + oy;
          const int col = (wrap(ux) * nc + wrap(uy)) * nc;
          real sh[3] = {shift(ux), shift(uy), real(0)};
          if (lo < 0) {
            sweep(start[col], start[col + hi + 1], sh);            // cells 0 ... hi
            sh[2] = LC.L;
            sweep(start[col + nc - 1], start[col + nc], sh);       // cell nc - 1, one period down
          } else if (hi >= nc) {
            sweep(start[col + lo], start[col + nc], sh);           // cells lo ... nc - 1
            sh[2] = -LC.L;
            sweep(start[col], start[col + 1], sh);                 // cell 0, one period up
          } else {
            sweep(start[col + lo], start[col + hi + 1], sh);       // cells lo ... hi
          }
        }
    } else {
      for (int s = lane; s < C.n_mol; s += 32) lj_pair<real, false>(xi, op[s], nullptr, LC, s == w, fi, e);
    }
    for (int o = 16; o > 0; o >>= 1) {
      fi[0] += __shfl_xor_sync(0xffffffffu, fi[0], o);
      fi[1] += __shfl_xor_sync(0xffffffffu, fi[1], o);
      fi[2] += __shfl_xor_sync(0xffffffffu, fi[2], o);
    }
    if (lane == 0) {
      double* fo = f + 9ll * m;
      for (int c = 0; c < 3; ++c) {
        if constexpr (sizeof(real) == 4) fo[c] += espk::f32_to_f64(fi[c]);
        else fo[c] += (double)fi[c];
      }
    }
  }
  if constexpr (sizeof(real) == 4) block_add_f(e, el);
  else block_add(e, el);
}

MdConst make_const(const esp_md_s* md) {
  const esp_md_params& p = md->prm;
  MdConst C;
  C.dt = p.dt;
  C.k_bond = p.k_bond;
  C.r0 = p.r0;
  C.k_angle = p.k_angle;
  C.theta0 = p.theta0;
  C.sigma2 = p.lj_sigma * p.lj_sigma;
  C.eps4 = 4.0 * p.lj_epsilon;
  C.rc2 = p.lj_cutoff * p.lj_cutoff;
  const double sr6 = std::pow(p.lj_sigma / p.lj_cutoff, 6);
  C.shift = 4.0 * p.lj_epsilon * (sr6 * sr6 - sr6);
  C.inv_mO = 1.0 / p.mass_O;
  C.inv_mH = 1.0 / p.mass_H;
  C.mO = p.mass_O;
  C.mH = p.mass_H;
  C.L = md->L;
  C.inv_L = 1.0 / md->L;
  C.n_mol = md->n_mol;
  C.nc = md->nc;
  C.k_bond_f = (float)C.k_bond;
  C.r0_f = (float)C.r0;
  C.k_angle_f = (float)C.k_angle;
  C.theta0_f = (float)C.theta0;
  C.L_f = (float)C.L;
  C.inv_L_f = (float)C.inv_L;
  return C;
}

int blocks_of(long long n) { return (int)std::max<long long>(1, (n + 255) / 256); }

// Forces at the current positions: the solve's into d_f, the bonded and
// Lennard-Jones terms into d_f2 on a second stream while the solve runs;
// energies to e[0] (Coulomb, written), e[1] (bonded) and e[2]
// (Lennard-Jones), both added. st waits for both.
esp_status md_forces(esp_md_s* md, double* e, cudaStream_t st_main) {
  MD_CU(cudaEventRecord(md->ev_fork3, st_main));
  MD_CU(cudaStreamWaitEvent(md->st3, md->ev_fork3, 0));
  esp_status s = esp_step(md->plan, md->d_x, e, md->d_f, nullptr, ESP_DEVICE);
  if (s != ESP_OK) return s;
  cudaStream_t st = md->st3;
  const MdConst C = make_const(md);
  // the bonded kernel stores every atom's d_f2; Lennard-Jones adds to the O's
  if (md->fp32)
    k_bonded<true><<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_x, md->d_f2, C, e + 1);
  else
    k_bonded<false><<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_x, md->d_f2, C, e + 1);
  if (md->nc >= 3) {
    const long long ncell = (long long)md->nc * md->nc * md->nc;
    MD_CU(cudaMemsetAsync(md->d_count, 0, ncell * sizeof(uint32_t), st));
    MD_CU(cudaMemsetAsync(md->d_cursor, 0, ncell * sizeof(uint32_t), st));
    k_lj_bin<<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_x, C, md->d_cell, md->d_count);
    MD_CU(espk::launch_scan(md->d_count, md->d_start, md->d_tiles, ncell, st));
    k_lj_fill<<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_cell, md->d_start, md->d_cursor, md->d_sorted, md->n_mol);
  }
  const int use_cells = md->nc >= 3;
  const int wb = blocks_of(32ll * md->n_mol);                   // one warp per O
  if (md->fp32) {
    auto* op = reinterpret_cast<OPos<float>*>(md->d_opos);
    k_lj_pack<float><<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_x, md->d_sorted, use_cells, md->n_mol, C, op);
    k_lj<float><<<wb, 256, 0, st>>>(op, md->d_cell, md->d_start, C, md->d_f2, e + 2);
  } else {
    auto* op = reinterpret_cast<OPos<double>*>(md->d_opos);
    k_lj_pack<double><<<blocks_of(md->n_mol), 256, 0, st>>>(md->d_x, md->d_sorted, use_cells, md->n_mol, C, op);
    k_lj<double><<<wb, 256, 0, st>>>(op, md->d_cell, md->d_start, C, md->d_f2, e + 2);
  }
  MD_CU(cudaGetLastError());
  MD_CU(cudaEventRecord(md->ev_join3, st));
  MD_CU(cudaStreamWaitEvent(st_main, md->ev_join3, 0));
  return ESP_OK;
}

template <typename T>
esp_status md_alloc(esp_md_s* md, T** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(1, count) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return md_fail(ESP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  md->allocs.push_back(*p);
  return ESP_OK;
}

void md_release(esp_md_s* md) {
  for (void* a : md->allocs) cudaFree(a);
  md->allocs.clear();
}

void md_streams_release(esp_md_s* md) {
  if (md->st3) cudaStreamSynchronize(md->st3);
  if (md->ev_fork3) cudaEventDestroy(md->ev_fork3);
  if (md->ev_join3) cudaEventDestroy(md->ev_join3);
  if (md->st3) cudaStreamDestroy(md->st3);
  md->ev_fork3 = md->ev_join3 = nullptr;
  md->st3 = nullptr;
}

struct MdDevice {
  int prev = 0;
  explicit MdDevice(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~MdDevice() { cudaSetDevice(prev); }
};

// One velocity-Verlet step: kick + drift, forces, kick, commit of its energies.
esp_status md_step(esp_md_s* md, cudaStream_t st) {
  const MdConst C = make_const(md);
  const int nb = blocks_of(md->n_atoms);
  k_kick_drift<<<nb, 256, 0, st>>>(md->d_x, md->d_v, md->d_f, md->d_f2, C, md->n_atoms);
  esp_status s = md_forces(md, md->d_ecur, st);
  if (s != ESP_OK) return s;
  k_kick<<<nb, 256, 0, st>>>(md->d_v, md->d_f, md->d_f2, C, md->n_atoms, 1.0, md->d_ecur + 3);
  k_commit<<<1, 32, 0, st>>>(md->d_ecur, md->d_e, md->d_row, md->e_cap);
  MD_CU(cudaGetLastError());
  return ESP_OK;
}

void drop_graph(esp_md_s* md) {
  if (md->gexec) cudaGraphExecDestroy(md->gexec);
  if (md->graph) cudaGraphDestroy(md->graph);
  md->gexec = nullptr;
  md->graph = nullptr;
  md->graph_e = nullptr;
  md->graph_cap = 0;
}

// The step as a CUDA graph on the plan's stream (captured once per energy
// buffer; the solve inside is launched directly into the capture).
esp_status md_graph(esp_md_s* md, cudaStream_t st) {
  if (md->gexec && md->graph_e == md->d_e && md->graph_cap == md->e_cap) return ESP_OK;
  drop_graph(md);
  MD_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  esp_status s = md_step(md, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != ESP_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return md_fail(ESP_ERR_CUDA, std::string("MD step capture: ") + cudaGetErrorString(e));
  md->graph = g;
  MD_CU(cudaGraphInstantiate(&md->gexec, g, 0));
  md->graph_e = md->d_e;
  md->graph_cap = md->e_cap;
  return ESP_OK;
}

}  // namespace

extern "C" {

void esp_md_params_init(esp_md_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dt = 0.0005;
  p->k_bond = 345000.0;
  p->r0 = 0.1;
  p->k_angle = 383.0;
  p->theta0 = 109.47 * kPiMd / 180.0;
  p->lj_sigma = 0.316557;
  p->lj_epsilon = 0.650194;
  p->lj_cutoff = 1.0;
  p->mass_O = 15.9994;
  p->mass_H = 1.008;
}

esp_status esp_md_create(esp_plan_t plan, const esp_md_params* params, const double* xyz, const double* vel,
                         esp_md_t* out) {
  if (!plan || !params || !xyz || !vel || !out) return md_fail(ESP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  esp_plan_params info;
  esp_status s = esp_plan_info(plan, &info);
  if (s != ESP_OK) return s;
  if (info.triclinic) return md_fail(ESP_ERR_UNSUPPORTED, "the MD loop runs on cubic plans");
  if (info.N <= 0 || info.N % 3 != 0) return md_fail(ESP_ERR_INVALID_ARG, "the plan's atoms must be (O, H, H) triples");
  const esp_md_params& p = *params;
  if (!(p.dt > 0) || !(p.mass_O > 0) || !(p.mass_H > 0) || !(p.r0 > 0) || !(p.lj_sigma > 0) ||
      !(p.lj_cutoff > 0) || !(p.lj_cutoff < 0.5 * info.L) || !(p.k_bond >= 0) || !(p.k_angle >= 0) ||
      !(p.lj_epsilon >= 0))
    return md_fail(ESP_ERR_INVALID_ARG, "MD parameters: positive dt, masses, r0, sigma; 0 < cutoff < L/2");
  esp_md_s* md = new esp_md_s();
  md->plan = plan;
  md->prm = p;
  md->device = espe::plan_device(plan);
  md->n_atoms = info.N;
  md->n_mol = (int)(info.N / 3);
  md->L = info.L;
  md->nc = (int)std::floor(info.L / p.lj_cutoff);
  md->fp32 = info.precision == ESP_FP32;
  if (md->nc < 3) md->nc = 0;
  MdDevice g(md->device);
  const size_t n3 = (size_t)md->n_atoms * 3;
  esp_status st = ESP_OK;
  if ((st = md_alloc(md, &md->d_x, n3)) != ESP_OK || (st = md_alloc(md, &md->d_v, n3)) != ESP_OK ||
      (st = md_alloc(md, &md->d_f, n3)) != ESP_OK || (st = md_alloc(md, &md->d_f2, n3)) != ESP_OK ||
      (st = md_alloc(md, &md->d_ecur, 4)) != ESP_OK ||
      (st = md_alloc(md, &md->d_row, 1)) != ESP_OK ||
      (st = md_alloc(md, &md->d_cell, (size_t)md->n_mol)) != ESP_OK ||
      (st = md_alloc(md, &md->d_sorted, (size_t)md->n_mol)) != ESP_OK ||
      (st = md_alloc(md, &md->d_opos, (size_t)md->n_mol * 4)) != ESP_OK) {
    md_release(md);
    delete md;
    return st;
  }
  if (md->nc >= 3) {
    const long long ncell = (long long)md->nc * md->nc * md->nc;
    if ((st = md_alloc(md, &md->d_count, (size_t)ncell)) != ESP_OK ||
        (st = md_alloc(md, &md->d_cursor, (size_t)ncell)) != ESP_OK ||
        (st = md_alloc(md, &md->d_start, (size_t)ncell + 1)) != ESP_OK ||
        (st = md_alloc(md, &md->d_tiles, (size_t)espk::scan_tiles(ncell) + 1)) != ESP_OK) {
      md_release(md);
      delete md;
      return st;
    }
  }
  // the three intramolecular pairs of every molecule are excluded
  std::vector<int32_t> pairs((size_t)md->n_mol * 6);
  for (int m = 0; m < md->n_mol; ++m) {
    const int32_t o = 3 * m;
    const int32_t pr[6] = {o, o + 1, o, o + 2, o + 1, o + 2};
    std::copy(pr, pr + 6, pairs.begin() + 6ll * m);
  }
  if ((st = esp_set_exclusions(plan, pairs.data(), (int64_t)md->n_mol * 3)) != ESP_OK) {
    md_release(md);
    delete md;
    return st;
  }
  if (cudaMemcpy(md->d_x, xyz, n3 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(md->d_v, vel, n3 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    md_release(md);
    delete md;
    return md_fail(ESP_ERR_CUDA, "copy of the initial state failed");
  }
  if (cudaStreamCreateWithFlags(&md->st3, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&md->ev_fork3, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&md->ev_join3, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    md_streams_release(md);
    md_release(md);
    delete md;
    return md_fail(ESP_ERR_CUDA, "stream/event creation failed");
  }
  *out = md;
  return ESP_OK;
}

esp_status esp_md_run(esp_md_t md, int n_steps, double* energies) {
  if (!md || n_steps < 0) return md_fail(ESP_ERR_INVALID_ARG, "NULL md or n_steps < 0");
  MdDevice g(md->device);
  cudaStream_t st = espe::plan_stream(md->plan);
  const long long rows = (long long)n_steps + 1;
  if (rows > md->e_cap) {
    if (md->d_e) {
      md->allocs.erase(std::find(md->allocs.begin(), md->allocs.end(), (void*)md->d_e));
      cudaFree(md->d_e);
      md->d_e = nullptr;
    }
    esp_status s = md_alloc(md, &md->d_e, (size_t)rows * 4);
    if (s != ESP_OK) return s;
    md->e_cap = rows;
  }
  MD_CU(cudaMemsetAsync(md->d_e, 0, (size_t)rows * 4 * sizeof(double), st));
  MD_CU(cudaMemsetAsync(md->d_ecur, 0, 4 * sizeof(double), st));
  MD_CU(cudaMemsetAsync(md->d_row, 0, sizeof(int), st));
  const MdConst C = make_const(md);
  const int nb = blocks_of(md->n_atoms);
  // row 0: the current state (forces computed once, then carried over)
  if (!md->have_forces) {
    esp_status s = md_forces(md, md->d_ecur, st);
    if (s != ESP_OK) return s;
    md->have_forces = true;
  } else {
    MD_CU(cudaMemcpyAsync(md->d_ecur, md->e_now, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  k_kick<<<nb, 256, 0, st>>>(md->d_v, md->d_f, md->d_f2, C, md->n_atoms, 0.0, md->d_ecur + 3);
  k_commit<<<1, 32, 0, st>>>(md->d_ecur, md->d_e, md->d_row, md->e_cap);
  MD_CU(cudaGetLastError());
  if (n_steps > 0) {
    esp_status s = md_graph(md, st);
    if (s != ESP_OK) return s;
    for (int k = 1; k <= n_steps; ++k) MD_CU(cudaGraphLaunch(md->gexec, st));
  }
  std::vector<double> h((size_t)rows * 4);
  MD_CU(cudaMemcpyAsync(h.data(), md->d_e, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  MD_CU(cudaStreamSynchronize(st));
  std::copy(h.end() - 4, h.end() - 1, md->e_now);
  if (energies) std::copy(h.begin(), h.end(), energies);
  return ESP_OK;
}

esp_status esp_md_state(esp_md_t md, double* xyz, double* vel) {
  if (!md) return md_fail(ESP_ERR_INVALID_ARG, "NULL md");
  MdDevice g(md->device);
  cudaStream_t st = espe::plan_stream(md->plan);
  const size_t bytes = (size_t)md->n_atoms * 3 * sizeof(double);
  if (xyz) MD_CU(cudaMemcpyAsync(xyz, md->d_x, bytes, cudaMemcpyDeviceToHost, st));
  if (vel) MD_CU(cudaMemcpyAsync(vel, md->d_v, bytes, cudaMemcpyDeviceToHost, st));
  MD_CU(cudaStreamSynchronize(st));
  return ESP_OK;
}

esp_status esp_md_destroy(esp_md_t md) {
  if (!md) return ESP_OK;
  {
    MdDevice g(md->device);
    cudaStream_t st = espe::plan_stream(md->plan);
    if (st) cudaStreamSynchronize(st);
    drop_graph(md);
    md_streams_release(md);
    md_release(md);
    // the intramolecular exclusions belong to the MD state, not to the plan
    esp_set_exclusions(md->plan, nullptr, 0);
  }
  delete md;
  return ESP_OK;
}

}  // extern "C"
