// Local part (Eq. localpart) in FP32 with one warp per i-cluster.
//
// An i-cluster is up to kClusterAtoms consecutive atoms of one cell-list
// column (cx, cy), taken in z order across the column's bricks; a small
// kernel lists every cluster's atoms once per step. The warp of a cluster
//  1. loads the cluster's atoms into shared memory, in a frame whose origin is
//     the column's cell corner (x, y) and the bottom of the first atom's brick
//     (z), and forms their bounding box;
//  2. visits the (2R+1)^2 neighbouring image columns (one per lane); a column
//     whose xy gap to the box is >= r_c is skipped, otherwise the z window of
//     the cutoff around the box is cut at brick boundaries into contiguous
//     slab ranges, appended to a per-warp list of ranges (first atom, prefix
//     count, image offsets);
//  3. walks the listed candidates with all 32 lanes, 32 * kWalk per step,
//     lane k taking candidates k, k + 32, ... (coalesced loads; each lane
//     advances a range cursor shared through the warp), moves each into the
//     cluster frame and keeps those within r_c of the box in a per-warp
//     queue, and
//  4. whenever 32 are queued, lane k takes queued candidate k and evaluates it
//     against every atom of the cluster; pairs outside 0 < r < r_c are
//     evaluated at r = r_c with zero charge, so no lane branches. At the end
//     the per-lane sums are summed over the warp.
#pragma once
#include "esp_cluster_list.cuh"

namespace espk {

// Warps per block: 16 (one block per SM, 16 consecutive clusters sharing its
// L1) for long cluster lists, 8 (two blocks per SM) for short ones, whose
// blocks then leave room for concurrent work on the same SMs.
constexpr int kClusterWarpsLarge = 16;
constexpr int kClusterWarpsSmall = 8;
constexpr int kWalk = 4;                         // candidates per lane and step
constexpr int kClusterQueue = 32 + 32 * kWalk;   // queued candidates per warp
constexpr int kSegCap = 96;                      // listed ranges per warp

__device__ __forceinline__ float fmax3(float a, float b, float c) { return fmaxf(fmaxf(a, b), c); }

template <int NC>
__device__ __forceinline__ float horner_f(const float* c, float y) {
  float v = c[NC - 1];
#pragma unroll
  for (int k = NC - 2; k >= 0; --k) v = fmaf(v, y, c[k]);
  return v;
}

// 1/sqrt(r2) by the PTX approximate instruction (relative error below
// 2^-22), subnormal inputs flushed: no slow path for them.
__device__ __forceinline__ float rsqrt_approx(float r2) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
  return r;
}

// The two local-part polynomials interleaved, (H_k, K_k) for k = 0 ... : one
// packed multiply-add per Horner step advances both.
struct NearCoefHK {
  float2 hk[Deg<float>::nr];
};

__host__ inline NearCoefHK interleave(const NearCoef<float>& nc) {
  NearCoefHK o;
  for (int k = 0; k < Deg<float>::nr; ++k) o.hk[k] = make_float2(nc.h[k], nc.k[k]);
  return o;
}

// Per-warp shared state of the cluster kernel.
template <bool HALF>
struct ClusterSmem {
  float4 queue[kClusterQueue];          // queued candidates (cluster frame, charge)
  int qidx[HALF ? kClusterQueue : 1];   // their atom indices (HALF)
  float4 idata[kClusterAtoms];          // the cluster's atoms
  // the same atoms in pairs (2m, 2m + 1) for the packed pair arithmetic:
  // ipair[2m] = (x, x', y, y'), ipair[2m + 1] = (z, z', q, q')
  float4 ipair[kClusterAtoms];
  float4 seg_off[kSegCap];              // image offsets of each listed range
  uint32_t seg_pos[kSegCap];            // first atom of each listed range
  int seg_pre[kSegCap + 1];             // exclusive prefix counts (+ total)
};

// HALF = false: every pair is evaluated from both sides (each warp owns its
// atoms' sums; plain stores). HALF = true: every pair is evaluated once
// (Newton's third law): a cluster takes the image columns of one half plane,
// (oy > 0) or (oy = 0, ox > 0), plus the atoms that follow it in its own
// column (upwards, including the periodic images above), and its pairs among
// themselves; the reaction on each candidate is added to its result with one
// float4 atomic, and the cluster's own sums likewise (results zeroed before).
// VIR (HALF only): also the local virial 1/2 sum_ij F_ij d_ij^T, summed per
// warp over its clusters of one system and added to vloc[6 * system + c]
// (xx, yy, zz, xy, xz, yz) with FP64 atomics when the system changes and at
// the end.
// TRI: triclinic cell. Cells are cells of fractional coordinates, a column
// (ox, oy) away sits at ox a/n_c + oy b/n_c and a brick up the column at
// bc c/n_c (Cartesian offsets), and the records hold Cartesian positions
// relative to their brick corner. The z window is the cutoff around the box
// in Cartesian z (z depends on the fractional z alone); a column is culled
// when the xy extent it can reach over the cutoff's z window (its sheared
// cross-section) lies r_c or more from the cluster's box.
template <int NC, bool HALF, bool VIR, int WARPS, bool TRI = false>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) k_near_cluster(
    const SysDesc* __restrict__ sys, const int2* __restrict__ cmap, const int2* __restrict__ catoms,
    const uint32_t* __restrict__ n_clusters, const float4* __restrict__ rel,
    const uint32_t* __restrict__ start, float4* __restrict__ nearres, const NearCoefHK nc,
    int* __restrict__ err, double* __restrict__ vloc = nullptr) {
  static_assert(HALF || !VIR, "the virial is formed in the half form");
  static_assert(!(TRI && VIR), "no virial on a triclinic cell");
  constexpr int kClusterWarps = WARPS;
  __shared__ ClusterSmem<HALF> smem_all[kClusterWarps];
  __shared__ int next_cluster;                      // the block's next cluster (offset from g_begin)
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  ClusterSmem<HALF>& W = smem_all[wib];
  const unsigned lt_mask = (1u << lane) - 1u;
  const float k4 = (float)(1.0 / kFourPi);
  const float far_away = 1e18f;
  // each block takes a contiguous run of clusters (neighbours in z share most
  // candidates, so they meet in the block's L1)
  const long long total_clusters = *n_clusters;
  const long long per_block = (total_clusters + gridDim.x - 1) / gridDim.x;
  const long long g_begin = (long long)blockIdx.x * per_block;
  const long long g_end = min(total_clusters, g_begin + per_block);
  float2 vir[6];                                    // VIR: this lane's pair sums (two partial sums each)
#pragma unroll
  for (int c = 0; c < 6; ++c) vir[c] = make_float2(0.f, 0.f);
  int vsys = -1;                                    // VIR: their system
  auto flush_virial = [&]() {
    if constexpr (VIR) {
      if (vsys >= 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          float t = vir[c].x + vir[c].y;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
          if (lane == 0) atomicAdd(vloc + 6 * vsys + c, (double)t * (1.0 / kFourPi));
          vir[c] = make_float2(0.f, 0.f);
        }
      }
    }
  };

  // the warps take the block's clusters in order from a shared counter, so
  // a warp that meets cheap clusters takes more of them (no tail of one
  // warp working while the others wait for the block to end)
  if (threadIdx.x == 0) next_cluster = 0;
  __syncthreads();
  for (;;) {
    int take = 0;
    if (lane == 0) take = atomicAdd(&next_cluster, 1);
    take = __shfl_sync(full, take, 0);
    const long long g = g_begin + take;
    if (g >= g_end) break;
    const int2 cm = cmap[g];
    if constexpr (VIR) {
      if (cm.x != vsys) {
        flush_virial();
        vsys = cm.x;
      }
    }
    const SysDesc& S = sys[cm.x];
    const int n_c = S.n_c, bc = S.bc, nb = S.nb, R = S.reach;
    const float inv_bc = S.inv_bcf;
    const long long brick_plane = (long long)nb * nb * bc * bc * bc;   // key stride of one z brick
    const int cx = cm.y / n_c, cy = cm.y - (cm.y / n_c) * n_c;
    const uint32_t* st = start + S.cell0;
    const float w = S.wf;
    const float bcw = (float)bc * w;
    const long long a_lo = S.atom0, a_hi = S.atom0 + S.n_atoms;

    // ---- 1. the cluster's atoms
    int2 ca = make_int2(-1, 0);
    if (lane < kClusterAtoms) ca = catoms[g * kClusterAtoms + lane];
    const long long my_idx = ca.x;
    const int my_bz = ca.y;
    const bool mine = lane < kClusterAtoms && my_idx >= a_lo && my_idx < a_hi;
    if (lane < kClusterAtoms && my_idx >= 0 && !mine) atomicOr(err, 4);
    const int m = __popc(__ballot_sync(full, mine));
    if (m == 0) continue;
    const int bz_0 = __shfl_sync(full, my_bz, 0);
    float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) {
      ri = rel[my_idx];
      if constexpr (TRI) {
        const float dbz = (float)(my_bz - bz_0);
        ri.x = fmaf(dbz, S.tbrick[0], ri.x);
        ri.y = fmaf(dbz, S.tbrick[1], ri.y);
        ri.z = fmaf(dbz, S.tbrick[2], ri.z);
      } else {
        ri.z += (float)(my_bz - bz_0) * bcw;
      }
    }
    // bounding box. Cube: all coordinates are >= 0 in this frame, so the
    // float bit patterns order like the values. Triclinic: x and y may be
    // negative; the keys flip the sign bit (and the rest for negatives).
    float bx_lo, by_lo, bz_lo, bx_hi, by_hi, bz_hi;
    if constexpr (TRI) {
      auto key = [](float v) {
        const unsigned b = __float_as_uint(v);
        return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
      };
      auto unkey = [](unsigned k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); };
      bx_lo = unkey(__reduce_min_sync(full, mine ? key(ri.x) : 0xffffffffu));
      by_lo = unkey(__reduce_min_sync(full, mine ? key(ri.y) : 0xffffffffu));
      bz_lo = unkey(__reduce_min_sync(full, mine ? key(ri.z) : 0xffffffffu));
      bx_hi = unkey(__reduce_max_sync(full, mine ? key(ri.x) : 0u));
      by_hi = unkey(__reduce_max_sync(full, mine ? key(ri.y) : 0u));
      bz_hi = unkey(__reduce_max_sync(full, mine ? key(ri.z) : 0u));
    } else {
      const unsigned inf_bits = 0x7f800000u;
      bx_lo = __uint_as_float(__reduce_min_sync(full, mine ? __float_as_uint(ri.x) : inf_bits));
      by_lo = __uint_as_float(__reduce_min_sync(full, mine ? __float_as_uint(ri.y) : inf_bits));
      bz_lo = __uint_as_float(__reduce_min_sync(full, mine ? __float_as_uint(ri.z) : inf_bits));
      bx_hi = __uint_as_float(__reduce_max_sync(full, mine ? __float_as_uint(ri.x) : 0u));
      by_hi = __uint_as_float(__reduce_max_sync(full, mine ? __float_as_uint(ri.y) : 0u));
      bz_hi = __uint_as_float(__reduce_max_sync(full, mine ? __float_as_uint(ri.z) : 0u));
    }
    // missing atoms (m < 8) sit far away with zero charge: every pair with
    // them is masked off, so the eight pair evaluations need no branch
    if (lane < kClusterAtoms) {
      const float4 a = mine ? ri : make_float4(far_away, far_away, far_away, 0.f);
      W.idata[lane] = a;
      float* pa = reinterpret_cast<float*>(&W.ipair[2 * (lane >> 1)]);
      const int o = lane & 1;
      pa[o] = a.x;
      pa[2 + o] = a.y;
      pa[4 + o] = a.z;
      pa[6 + o] = a.w;
    }
    __syncwarp();

    // per-lane sums for the cluster atoms in pairs (2m, 2m + 1): potential
    // and force components, packed two-wide
    float2 pu[kClusterAtoms / 2], px[kClusterAtoms / 2], py[kClusterAtoms / 2], pz[kClusterAtoms / 2];
#pragma unroll
    for (int m = 0; m < kClusterAtoms / 2; ++m) pu[m] = px[m] = py[m] = pz[m] = make_float2(0.f, 0.f);

    const float rc2 = S.rc2f, inv_rc = S.inv_rcf;
    const float inv_rc2x2 = S.inv_rc2x2f, inv_rc3 = S.inv_rc3f;
    const float margin = 1e-4f * w;
    const float cull2 = rc2 + 2.f * margin * S.r_cf;
    // slabs per unit of z (cube: w per cell; triclinic: c_z / n_c per cell)
    const float slab_per_len = TRI ? (float)kSub / (S.tbrick[2] * inv_bc) : (float)kSub / w;
    int qn = 0;                                   // queued candidates
    int nseg = 0, total = 0;                      // listed ranges, their candidates

    // pair work on queued candidate `jd` (atom index jx or -1). The eight
    // cluster atoms are taken two at a time with the packed f32x2 multiply-
    // adds, so one instruction does the arithmetic of two pairs; every
    // packed operation rounds like its scalar form, in the same order.
    const float2 inv_rc2x2_2 = make_float2(inv_rc2x2, inv_rc2x2);
    const float2 neg_inv_rc_2 = make_float2(-inv_rc, -inv_rc);
    const float2 inv_rc3_2 = make_float2(inv_rc3, inv_rc3);
    const float2 minus_one_2 = make_float2(-1.f, -1.f);
    auto evaluate = [&](const float4 jd, int jx) {
      const float2 njx = make_float2(-jd.x, -jd.x), njy = make_float2(-jd.y, -jd.y),
                   njz = make_float2(-jd.z, -jd.z);
      float2 uj = make_float2(0.f, 0.f), fjx = uj, fjy = uj, fjz = uj;
#pragma unroll
      for (int m = 0; m < kClusterAtoms / 2; ++m) {
        const float4 A = W.ipair[2 * m], B = W.ipair[2 * m + 1];
        const float2 dx = __fadd2_rn(make_float2(A.x, A.y), njx);
        const float2 dy = __fadd2_rn(make_float2(A.z, A.w), njy);
        const float2 dz = __fadd2_rn(make_float2(B.x, B.y), njz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        // HALF never queues a cluster atom against itself, so 0 < r2 holds
        // for distinct positions; the full form meets the cluster's own atoms
        const bool in0 = HALF ? r2.x < rc2 : (r2.x < rc2 && r2.x > 0.f);
        const bool in1 = HALF ? r2.y < rc2 : (r2.y < rc2 && r2.y > 0.f);
        // masked pairs (outside r_c, or the far-away padding) are evaluated
        // at r = r_c with zero charge: every lane runs the same instructions
        const float2 r2m = make_float2(in0 ? r2.x : rc2, in1 ? r2.y : rc2);
        const float2 qj = make_float2(in0 ? jd.w : 0.f, in1 ? jd.w : 0.f);
        const float2 rinv = make_float2(rsqrt_approx(r2m.x), rsqrt_approx(r2m.y));
        const float2 y = __ffma2_rn(r2m, inv_rc2x2_2, minus_one_2);
        // Horner for (H, K) together, one chain per atom
        const float2 y0 = make_float2(y.x, y.x), y1 = make_float2(y.y, y.y);
        float2 hk0 = nc.hk[NC - 1], hk1 = nc.hk[NC - 1];
#pragma unroll
        for (int k = NC - 2; k >= 0; --k) {
          hk0 = __ffma2_rn(hk0, y0, nc.hk[k]);
          hk1 = __ffma2_rn(hk1, y1, nc.hk[k]);
        }
        const float2 h = make_float2(hk0.x, hk1.x), kk = make_float2(hk0.y, hk1.y);
        const float2 t1 = __ffma2_rn(h, neg_inv_rc_2, rinv);
        const float2 t2 = __ffma2_rn(kk, inv_rc3_2, __fmul2_rn(__fmul2_rn(rinv, rinv), rinv));
        pu[m] = __ffma2_rn(qj, t1, pu[m]);
        const float2 fs = __fmul2_rn(qj, t2);
        px[m] = __ffma2_rn(fs, dx, px[m]);
        py[m] = __ffma2_rn(fs, dy, py[m]);
        pz[m] = __ffma2_rn(fs, dz, pz[m]);
        if constexpr (HALF) {
          const float2 qi = make_float2(in0 ? B.z : 0.f, in1 ? B.w : 0.f);
          uj = __ffma2_rn(qi, t1, uj);
          const float2 fsj = __fmul2_rn(qi, t2);
          fjx = __ffma2_rn(fsj, dx, fjx);
          fjy = __ffma2_rn(fsj, dy, fjy);
          fjz = __ffma2_rn(fsj, dz, fjz);
          if constexpr (VIR) {
            // pair virial q_i q_j t2 d d^T (the 1/(4 pi) at the flush)
            const float2 v = __fmul2_rn(fsj, make_float2(jd.w, jd.w));
            const float2 vx = __fmul2_rn(v, dx), vy = __fmul2_rn(v, dy), vz = __fmul2_rn(v, dz);
            vir[0] = __ffma2_rn(vx, dx, vir[0]);
            vir[1] = __ffma2_rn(vy, dy, vir[1]);
            vir[2] = __ffma2_rn(vz, dz, vir[2]);
            vir[3] = __ffma2_rn(vx, dy, vir[3]);
            vir[4] = __ffma2_rn(vx, dz, vir[4]);
            vir[5] = __ffma2_rn(vy, dz, vir[5]);
          }
        }
      }
      if constexpr (HALF) {
        if (jx >= 0) {
          const float qk = -jd.w * k4;
          atomicAdd(nearres + jx, make_float4((uj.x + uj.y) * k4, qk * (fjx.x + fjx.y), qk * (fjy.x + fjy.y),
                                              qk * (fjz.x + fjz.y)));
        }
      }
    };

    // ---- 2. neighbouring image columns, in passes of 32 (one per lane). The
    // per-lane column state survives the walks, so listing resumes where it
    // stopped when the range list was full.
    const int side = 2 * R + 1;
    const int ncol = side * side;
    long long idx_last = 0;                        // HALF: last atom of the cluster
    int bz_last = 0;
    if constexpr (HALF) {
      idx_last = __shfl_sync(full, my_idx, m - 1);
      bz_last = __shfl_sync(full, my_bz, m - 1);
    }
    int c0 = 0;                                    // next column pass
    bool pass_open = false;
    int cur = 0, u_hi = -1;                        // this lane's unwrapped slab cursor, last slab
    int xx = 0, yy = 0;
    long long kxy = 0;                             // cell key of (xx, yy, 0)
    float offx = 0.f, offy = 0.f;
    long long own_pos = 0, own_end = 0;
    bool own_first = false;
    for (;;) {
      // list ranges until the list is nearly full or no column is left
      while (nseg <= kSegCap - 32) {
        if (!pass_open) {
          if (c0 >= ncol) break;
          const int ci = c0 + lane;
          c0 += 32;
          pass_open = true;
          const int ox = ci % side - R, oy = ci / side - R;
          const bool own = ox == 0 && oy == 0;
          bool use = ci < ncol;
          if constexpr (HALF) use = use && (oy > 0 || (oy == 0 && ox >= 0));
          float d2 = 0.f;
          if constexpr (!TRI) {
            const float gx = fmax3(0.f, (float)ox * w - bx_hi, bx_lo - (float)(ox + 1) * w);
            const float gy = fmax3(0.f, (float)oy * w - by_hi, by_lo - (float)(oy + 1) * w);
            d2 = gx * gx + gy * gy;
          } else {
            // triclinic: a point of the column at Cartesian height z (cluster
            // frame) has x = (f_x a_x + f_y b_x) / n_c + z c_x / c_z and
            // y = f_y b_y / n_c + z c_y / c_z with f_x in [ox, ox + 1),
            // f_y in [oy, oy + 1). Over the z window of the full cutoff that
            // bounds the column's xy extent, whose gap to the cluster's box
            // bounds every candidate's xy distance from below
            const float z1 = bz_lo - S.r_cf - margin, z2 = bz_hi + S.r_cf + margin;
            const float sx = S.tbrick[0] / S.tbrick[2], sy = S.tbrick[1] / S.tbrick[2];
            const float xb0 = (float)oy * S.tcol[1], xb1 = (float)(oy + 1) * S.tcol[1];
            const float x_lo = fmaf((float)ox, S.tcol[0], fminf(xb0, xb1)) + fminf(z1 * sx, z2 * sx);
            const float x_hi = fmaf((float)(ox + 1), S.tcol[0], fmaxf(xb0, xb1)) + fmaxf(z1 * sx, z2 * sx);
            const float y_lo = (float)oy * S.tcol[2] + fminf(z1 * sy, z2 * sy);
            const float y_hi = (float)(oy + 1) * S.tcol[2] + fmaxf(z1 * sy, z2 * sy);
            const float gx = fmax3(0.f, x_lo - bx_hi, bx_lo - x_hi);
            const float gy = fmax3(0.f, y_lo - by_hi, by_lo - y_hi);
            d2 = gx * gx + gy * gy;
          }
          const bool col_on = use && d2 < cull2;
          cur = 0;
          u_hi = -1;
          own_first = false;
          if (col_on) {
            const float hz = sqrtf(rc2 - fminf(d2, rc2)) + margin;
            const int base_slab = bz_0 * bc * kSub;
            cur = base_slab + (int)floorf((bz_lo - hz) * slab_per_len);
            u_hi = base_slab + (int)floorf((bz_hi + hz) * slab_per_len);
            xx = wrap_index(cx + ox, n_c);
            yy = wrap_index(cy + oy, n_c);
            kxy = cell_key(S, xx, yy, 0);
          }
          if constexpr (TRI) {
            offx = fmaf((float)ox, S.tcol[0], (float)oy * S.tcol[1]);
            offy = (float)oy * S.tcol[2];
          } else {
            offx = (float)ox * w;
            offy = (float)oy * w;
          }
          // HALF, own column: the first range runs from just after the
          // cluster's last atom to the window top inside that atom's brick;
          // the listing then continues with the next brick up
          if (HALF && own && col_on) {
            const int top_brick_end = (bz_last + 1) * bc * kSub - 1;
            const int send = min(u_hi, top_brick_end);
            const long long k1 = cell_key(S, xx, yy, send >> 2);   // inside brick bz_last: no wrap
            own_pos = idx_last + 1;
            own_end = st[k1 * kSub + (send & 3) + 1];
            if (own_end < own_pos) own_end = own_pos;
            cur = top_brick_end + 1;
            own_first = true;
          }
        }
        if (!__any_sync(full, cur <= u_hi || own_first)) {
          pass_open = false;
          continue;
        }
        // one round: each lane with slabs left lists its next brick range
        long long pos = 0, end = 0;
        float offz = 0.f;
        int dbrick = 0;                                             // TRI: bricks up from bz_0
        if (own_first) {
          pos = own_pos;
          end = own_end;
          offz = (float)(bz_last - bz_0) * bcw;
          dbrick = bz_last - bz_0;
          own_first = false;
        } else if (cur <= u_hi) {
          const int ucell = cur >> 2;                               // kSub = 4
          // floor(ucell / bc) through the FP32 reciprocal (exact for the
          // small |ucell| here: the +0.5 keeps the product off integers)
          const int ubrick = __float2int_rd(((float)ucell + 0.5f) * inv_bc);
          const int lz = ucell - ubrick * bc;
          int wb = ubrick;                                          // periodic brick index
          while (wb < 0) wb += nb;
          while (wb >= nb) wb -= nb;
          const int send = min(u_hi, (ubrick + 1) * bc * kSub - 1);
          const long long k0 = kxy + (long long)wb * brick_plane + lz;
          const long long k1 = k0 + ((send >> 2) - ucell);
          pos = st[k0 * kSub + (cur & 3)];
          end = st[k1 * kSub + (send & 3) + 1];
          offz = (float)(ubrick - bz_0) * bcw;
          dbrick = ubrick - bz_0;
          cur = send + 1;
        }
        if (pos < end && (pos < a_lo || end > a_hi)) {
          atomicOr(err, 4);
          pos = end = 0;
        }
        const int cnt = pos < end ? (int)(end - pos) : 0;
        const unsigned bal = __ballot_sync(full, cnt > 0);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(full, incl, o);
          if (lane >= o) incl += t;
        }
        __syncwarp();
        if (cnt > 0) {
          const int slot = nseg + __popc(bal & lt_mask);
          W.seg_pos[slot] = (uint32_t)pos;
          W.seg_pre[slot] = total + incl - cnt;
          if constexpr (TRI) {
            const float db = (float)dbrick;
            W.seg_off[slot] = make_float4(fmaf(db, S.tbrick[0], offx), fmaf(db, S.tbrick[1], offy),
                                          db * S.tbrick[2], 0.f);
          } else {
            W.seg_off[slot] = make_float4(offx, offy, offz, 0.f);
          }
        }
        nseg += __popc(bal);
        total += __shfl_sync(full, incl, 31);
        __syncwarp();
        if (lane == 0) W.seg_pre[nseg] = total;
      }
      const bool last_walk = !pass_open && c0 >= ncol;

      // ---- 3. walk the listed candidates; evaluate every 32 kept (on the
      // last walk the final partial batch too, padded with far-away
      // chargeless candidates)
      __syncwarp();
      int base = 0;
      int scur = 0;
      for (;;) {
        if (qn >= 32 || (last_walk && qn > 0 && base >= total)) {
          const bool has = lane < qn;
          const int slot = qn >= 32 ? qn - 32 + lane : lane;
          __syncwarp();
          const float4 jd = W.queue[slot];
          const int jx = HALF ? W.qidx[slot] : -1;
          // padding candidates sit at -far_away, the cluster's padding atoms at
          // +far_away: never within r_c of each other (no 0 * inf)
          evaluate(qn >= 32 || has ? jd : make_float4(-far_away, -far_away, -far_away, 0.f),
                   (HALF && (qn >= 32 || has)) ? jx : -1);
          __syncwarp();
          qn = qn >= 32 ? qn - 32 : 0;
          continue;
        }
        if (base >= total) break;
        float4 v[kWalk];
        int jv[kWalk];
#pragma unroll
        for (int u = 0; u < kWalk; ++u) {
          const int f = base + u * 32 + lane;
          jv[u] = -1;
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          int s = scur;
          if (f < total) {
            while (W.seg_pre[s + 1] <= f) ++s;
            const int j = (int)W.seg_pos[s] + (f - W.seg_pre[s]);
            const float4 o = W.seg_off[s];
            v[u] = rel[j];
            v[u].x += o.x;
            v[u].y += o.y;
            v[u].z += o.z;
            jv[u] = j;
          }
          scur = __shfl_sync(full, s, 31);
        }
        base += 32 * kWalk;
#pragma unroll
        for (int u = 0; u < kWalk; ++u) {
          const float ex = fmax3(0.f, bx_lo - v[u].x, v[u].x - bx_hi);
          const float ey = fmax3(0.f, by_lo - v[u].y, v[u].y - by_hi);
          const float ez = fmax3(0.f, bz_lo - v[u].z, v[u].z - bz_hi);
          const bool pass = jv[u] >= 0 && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < cull2;
          const unsigned bal = __ballot_sync(full, pass);
          if (pass) {
            const int slot = qn + __popc(bal & lt_mask);
            W.queue[slot] = v[u];
            if constexpr (HALF) W.qidx[slot] = jv[u];
          }
          qn += __popc(bal);
        }
      }
      nseg = 0;
      total = 0;
      __syncwarp();
      if (last_walk) break;
    }

    // ---- 4. warp sums, output. The 32 per-lane sums (4 quantities x 8
    // atoms) are reduced over the warp by halving exchanges: at offset o a
    // lane keeps one half of its values, sends the other to lane ^ o and adds
    // what it receives; afterwards lane k holds the warp sum of value k =
    // 8 * quantity + atom.
    __syncwarp();
    float v[4 * kClusterAtoms];
#pragma unroll
    for (int m = 0; m < kClusterAtoms / 2; ++m) {
      v[2 * m] = pu[m].x;
      v[2 * m + 1] = pu[m].y;
      v[kClusterAtoms + 2 * m] = px[m].x;
      v[kClusterAtoms + 2 * m + 1] = px[m].y;
      v[2 * kClusterAtoms + 2 * m] = py[m].x;
      v[2 * kClusterAtoms + 2 * m + 1] = py[m].y;
      v[3 * kClusterAtoms + 2 * m] = pz[m].x;
      v[3 * kClusterAtoms + 2 * m + 1] = pz[m].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < o; ++k) {
        const float send = up ? v[k] : v[k + o];
        const float keep = up ? v[k + o] : v[k];
        v[k] = keep + __shfl_xor_sync(full, send, o);
      }
    }
    if constexpr (HALF) {
      // pairs inside the cluster (same image), every ordered pair (a, b):
      // lane k takes atom a = k % 8 against b = k / 8 and k / 8 + 4
      const int a_at = lane & (kClusterAtoms - 1);
      const float4 ra = W.idata[a_at];
      float su = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        const int b_at = (lane >> 3) + 4 * hb;
        const float4 rb = W.idata[b_at];
        const float dx = ra.x - rb.x, dy = ra.y - rb.y, dz = ra.z - rb.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool in = a_at != b_at && r2 < rc2 && r2 > 0.f;
        const float r2m = in ? r2 : rc2;
        const float qe = in ? rb.w : 0.f;
        const float rinv = rsqrt_approx(r2m);
        const float y = fmaf(r2m, inv_rc2x2, -1.f);
        float2 hk = nc.hk[NC - 1];
#pragma unroll
        for (int k = NC - 2; k >= 0; --k) hk = __ffma2_rn(hk, make_float2(y, y), nc.hk[k]);
        const float h = hk.x, kk = hk.y;
        su = fmaf(qe, fmaf(-h, inv_rc, rinv), su);
        const float fs = qe * fmaf(kk, inv_rc3, rinv * rinv * rinv);
        sx = fmaf(fs, dx, sx);
        sy = fmaf(fs, dy, sy);
        sz = fmaf(fs, dz, sz);
        if constexpr (VIR) {
          // ordered pairs: each unordered pair twice, half weight
          const float v = 0.5f * ra.w * fs;
          const float vx = v * dx, vy = v * dy, vz = v * dz;
          vir[0].x = fmaf(vx, dx, vir[0].x);
          vir[1].x = fmaf(vy, dy, vir[1].x);
          vir[2].x = fmaf(vz, dz, vir[2].x);
          vir[3].x = fmaf(vx, dy, vir[3].x);
          vir[4].x = fmaf(vx, dz, vir[4].x);
          vir[5].x = fmaf(vy, dz, vir[5].x);
        }
      }
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        su += __shfl_xor_sync(full, su, o);
        sx += __shfl_xor_sync(full, sx, o);
        sy += __shfl_xor_sync(full, sy, o);
        sz += __shfl_xor_sync(full, sz, o);
      }
      v[0] += lane < kClusterAtoms ? su : (lane < 2 * kClusterAtoms ? sx : (lane < 3 * kClusterAtoms ? sy : sz));
    }
    // lane t < 8 gathers atom t's four sums from lanes t, t + 8, t + 16, t + 24
    const float ou = v[0];
    const float ofx = __shfl_sync(full, v[0], (lane + kClusterAtoms) & 31);
    const float ofy = __shfl_sync(full, v[0], (lane + 2 * kClusterAtoms) & 31);
    const float ofz = __shfl_sync(full, v[0], (lane + 3 * kClusterAtoms) & 31);
    if (mine) {
      const float4 out = make_float4(ou * k4, ri.w * ofx * k4, ri.w * ofy * k4, ri.w * ofz * k4);
      if constexpr (HALF) atomicAdd(nearres + my_idx, out);
      else nearres[my_idx] = out;
    }
    __syncwarp();
  }
  flush_virial();
}

}  // namespace espk
