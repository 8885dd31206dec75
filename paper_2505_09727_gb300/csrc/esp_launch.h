// Host-callable launchers for the ESP kernels, one set per precision.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "esp_device.cuh"

namespace espk {

template <typename real>
struct Launch {
  static cudaError_t ingest(const SysDesc* sys, const int2* chunks, int n_chunks, const void* xyz,
                            bool xyz_is_double, void* coord, uint32_t* key, uint32_t* rank,
                            uint32_t* count, int* err, cudaStream_t st);
  static cudaError_t scatter(const SysDesc* sys, const int2* chunks, int n_chunks, const void* coord,
                             const uint32_t* key, const uint32_t* rank, const uint32_t* start,
                             const real* q, void* atoms, void* rel, uint32_t* perm, cudaStream_t st);
  static cudaError_t spread(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem,
                            const void* atoms, const uint32_t* start, real* grids,
                            const SICoef<real>& si, int* err, cudaStream_t st);
  // spec_ik (nullable): the ik method's three gradient spectra, component
  // a at spec_ik + a * spec_total (the pool's half-spectrum length)
  // vpart (nullable): spectral virial partials [nsys][nblk][6]
  static cudaError_t scale(const SysDesc* sys, int nsys, int nblk, void* spec, const real* tabs,
                           double* partials, void* spec_ik, long long spec_total, double* vpart,
                           cudaStream_t st);
  // grids_ik (nullable): the ik method's gradient grids, component a at
  // grids_ik + a * grid_total; then the forces come from them, not from
  // derivatives of the SI kernel
  static cudaError_t gather(int P, const SysDesc* sys, const int2* work, int n_work, size_t smem,
                            const void* atoms, const uint32_t* start, const real* grids,
                            const real* grids_ik, long long grid_total, void* far,
                            const SICoef<real>& si, int* err, cudaStream_t st);
  static cudaError_t near(const SysDesc* sys, const int2* chunks, int n_chunks, const void* atoms,
                          const void* rel, const uint32_t* start, void* nearres,
                          const NearCoef<real>& nc, int terms, bool queued, cudaStream_t st,
                          double* vloc = nullptr);
  // Local part with one warp per i-cluster (FP32 only): per-column cluster
  // counts into ccount[n_cols], their scan into cstart[n_cols + 1] (ctiles:
  // scan_tiles(n_cols) entries), the cluster list into cmap[cmap_cap] and
  // catoms[cmap_cap * 8], then the pair kernel; half = each pair once
  // (Newton's third law, atomics into nearres[n_atoms], cleared first).
  // stage 0: everything; 2: the cluster lists only; 1: the pair kernel only.
  static cudaError_t near_clusters(const SysDesc* sys, int nsys, long long n_cols, const uint32_t* start,
                                   const void* rel, void* nearres, const NearCoef<real>& nc, int terms,
                                   uint32_t* ccount, uint32_t* cstart, uint32_t* ctiles, int2* cmap,
                                   int2* catoms, long long cmap_cap, bool half, long long n_atoms, int stage,
                                   int* err, cudaStream_t st, double* vloc = nullptr, bool tri = false);
  // ea.ticket set: the last CTA also combines the energies (no launch_energy)
  static cudaError_t finalize(const SysDesc* sys, const int2* chunks, int n_chunks, const void* atoms,
                              const uint32_t* perm, const void* far, const void* nearres,
                              void* forces, void* pot, bool out_double, double* partials,
                              cudaStream_t st, const EnergyArgs& ea = EnergyArgs{});
  static cudaError_t convert_charges(const void* src, bool src_double, real* dst, long long n,
                                     cudaStream_t st);
  // Exclusions of one system: inv[perm[s]] = s, then every pair (caller
  // indices) removes its direct interaction from nearres (sorted order).
  static cudaError_t exclusions(const SysDesc* sys, const int2* pairs, long long n_pairs, const uint32_t* perm,
                                uint32_t* inv, long long n_atoms, const void* atoms, void* nearres,
                                cudaStream_t st);
  static bool supports_P(int P);
  static size_t atom_bytes();
  static size_t res_bytes();
};

// Exclusive scan of n counts into start[0..n] (start[n] = total); tile_sum
// needs scan_tiles(n) entries.
long long scan_tiles(long long n);
cudaError_t launch_scan(const uint32_t* count, uint32_t* start, uint32_t* tile_sum, long long n,
                        cudaStream_t st);
// vpart/vloc/vout (nullable): virial partials of the scale kernel, local
// virial sums, and the per-system totals [nsys][6] (xx, yy, zz, xy, xz, yz).
cudaError_t launch_energy(const SysDesc* sys, int nsys, const double* fourier, int n_fourier_blocks,
                          const double* partials, int n_chunks, const int* chunk_first,
                          const double* consts, double* out, double* user_energy, cudaStream_t st,
                          const double* vpart = nullptr, const double* vloc = nullptr,
                          double* vout = nullptr);

}  // namespace espk
