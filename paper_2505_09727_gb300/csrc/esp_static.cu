// Local part of the solve without any device allocation.
//
// esp_local_part_static evaluates, for positions and charges already in
// device memory, everything esp_compute returns except the spectral part:
// the cell-list pair sum of the local part, the self term and the
// neutralising background. Its working memory (cell counts and offsets, the
// sorted atom copy, per-atom results, energy partials) is carved out of one
// file-scope device array instead of cudaMalloc, for callers that cannot
// allocate device memory: code that runs while a framework's caching
// allocator owns the device heap, inside a region where an allocation would
// synchronise the device, or in a process whose device-memory budget is
// fixed up front.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/esp.h"
#include "esp_launch.h"
#include "esp_plan.h"

namespace {

// 6 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kStaticBytes = 6u << 20;
static __device__ __align__(256) unsigned char g_local_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

esp_status sfail(esp_status s, const std::string& m) {
  espe::set_last_error(m);
  return s;
}

// Device address of the static array on the current device (set up once per
// device, with that device current).
esp_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return sfail(ESP_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_local_scratch);
    if (e != cudaSuccess)
      return sfail(ESP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return ESP_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += align256(count * sizeof(T) + 1);
    return p;
  }
};

template <typename real>
esp_status run_local(const espe::HostPlan& hp, unsigned char* scratch, const double* xyz,
                     const double* q, double Q, double Q2, double* energy, double* forces,
                     double* potential, cudaStream_t st) {
  using L = espk::Launch<real>;
  const long long N = hp.info.N;
  const int n_chunks = (int)((N + espk::kChunk - 1) / espk::kChunk);
  // layout (sizes checked by the caller against kStaticBytes)
  Carve c{scratch};
  auto* d_desc = c.take<espk::SysDesc>(1);
  auto* d_chunks = c.take<int2>(std::max(1, n_chunks));
  auto* d_chunk_first = c.take<int>(2);
  auto* d_coord = c.take<unsigned char>(N * L::atom_bytes());
  auto* d_key = c.take<uint32_t>(N);
  auto* d_rank = c.take<uint32_t>(N);
  auto* d_count = c.take<uint32_t>(hp.n_keys);
  auto* d_start = c.take<uint32_t>(hp.n_keys + 1);
  auto* d_tiles = c.take<uint32_t>(espk::scan_tiles(hp.n_keys));
  auto* d_rel = c.take<unsigned char>(N * L::res_bytes());
  auto* d_atoms = c.take<unsigned char>(N * L::atom_bytes());
  auto* d_perm = c.take<uint32_t>(N);
  auto* d_q = c.take<real>(N);
  auto* d_far = c.take<unsigned char>(N * L::res_bytes());
  auto* d_near = c.take<unsigned char>(N * L::res_bytes());
  auto* d_partials = c.take<double>(2 * std::max(1, n_chunks));
  auto* d_fourier = c.take<double>(1);
  auto* d_consts = c.take<double>(2);
  auto* d_eout = c.take<double>(3);
  auto* d_err = c.take<int>(1);

  espk::SysDesc d = hp.desc;
  double consts[2], bg_shift;
  espe::charge_constants(hp, Q, Q2, &consts[0], &consts[1], &bg_shift);
  d.bg_shift = bg_shift;
  d.bg_shift_f = (float)bg_shift;
  std::vector<int2> chunks(n_chunks);
  for (int k = 0; k < n_chunks; ++k) chunks[k] = make_int2(0, k * espk::kChunk);
  int chunk_first[2] = {0, n_chunks};

#define SCU(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return sfail(ESP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // the array keeps the previous call's contents: everything read before it
  // is written is (re)initialised here
  SCU(cudaMemcpyAsync(d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, st));
  if (n_chunks)
    SCU(cudaMemcpyAsync(d_chunks, chunks.data(), n_chunks * sizeof(int2), cudaMemcpyHostToDevice, st));
  SCU(cudaMemcpyAsync(d_chunk_first, chunk_first, sizeof(chunk_first), cudaMemcpyHostToDevice, st));
  SCU(cudaMemcpyAsync(d_consts, consts, sizeof(consts), cudaMemcpyHostToDevice, st));
  SCU(cudaMemsetAsync(d_count, 0, hp.n_keys * sizeof(uint32_t), st));
  SCU(cudaMemsetAsync(d_far, 0, N * L::res_bytes(), st));
  SCU(cudaMemsetAsync(d_fourier, 0, sizeof(double), st));
  SCU(cudaMemsetAsync(d_err, 0, sizeof(int), st));

  const espk::NearCoef<real>& nc = *reinterpret_cast<const espk::NearCoef<real>*>(
      sizeof(real) == 4 ? (const void*)&hp.nc32 : (const void*)&hp.nc64);
  SCU(L::convert_charges(q, true, d_q, N, st));
  SCU(L::ingest(d_desc, d_chunks, n_chunks, xyz, true, d_coord, d_key, d_rank, d_count, d_err, st));
  SCU(espk::launch_scan(d_count, d_start, d_tiles, hp.n_keys, st));
  SCU(L::scatter(d_desc, d_chunks, n_chunks, d_coord, d_key, d_rank, d_start, d_q, d_atoms, d_rel, d_perm,
                 st));
  SCU(L::near(d_desc, d_chunks, n_chunks, d_atoms, d_rel, d_start, d_near, nc, hp.near_nc, hp.near_queued, st));
  SCU(L::finalize(d_desc, d_chunks, n_chunks, d_atoms, d_perm, d_far, d_near, forces, potential, true,
                  d_partials, st));
  SCU(espk::launch_energy(d_desc, 1, d_fourier, 1, d_partials, n_chunks, d_chunk_first, d_consts,
                          d_eout, energy, st));
  // the kernels' error flag: a non-finite position (zeroed by the ingest) or
  // a failed bounds check leaves the outputs wrong, so the call waits for its
  // kernels and reports it
  int flag = 0;
  SCU(cudaMemcpyAsync(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SCU(cudaStreamSynchronize(st));
#undef SCU
  if (flag & 1) return sfail(ESP_ERR_NONFINITE, "a position is NaN or infinite");
  if (flag) return sfail(ESP_ERR_INTERNAL, "a kernel bounds check failed (flag " + std::to_string(flag) + ")");
  return ESP_OK;
}

// Whether p is memory the GPU `dev` can address as a device pointer (device
// memory of that GPU, or managed memory); host and unregistered pointers are
// refused before any launch.
bool device_pointer(const void* p, int dev) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Bytes of the static array one call needs.
size_t needed_bytes(const espe::HostPlan& hp, int precision) {
  const long long N = hp.info.N;
  const size_t ab = precision == ESP_FP32 ? 16 : 32;
  const size_t rb = precision == ESP_FP32 ? 4 : 8;
  const long long n_chunks = (N + espk::kChunk - 1) / espk::kChunk;
  size_t b = 0;
  b += align256(sizeof(espk::SysDesc) + 1) + align256(std::max<long long>(1, n_chunks) * 8 + 1) +
       align256(9);
  b += align256(N * ab + 1) * 2 + align256(N * 4 + 1) * 3;
  b += align256(hp.n_keys * 4 + 1) + align256((hp.n_keys + 1) * 4 + 1) +
       align256(espk::scan_tiles(hp.n_keys) * 4 + 1) + align256(N * ab + 1);
  b += align256(N * rb + 1) + align256(N * ab + 1) * 2;
  b += align256(2 * std::max<long long>(1, n_chunks) * 8 + 1) + 4 * 256;
  return b;
}

}  // namespace

extern "C" esp_status esp_local_part_static(const esp_box* box, int64_t N, double tolerance,
                                            const esp_plan_opts* opts, const double* xyz,
                                            const double* q, double* energy, double* forces,
                                            double* potential) {
  if (!box || (N > 0 && (!xyz || !q))) return sfail(ESP_ERR_INVALID_ARG, "NULL argument");
  esp_plan_opts o;
  if (opts) o = *opts;
  else esp_plan_opts_init(&o);
  const double L = box->L[0];
  if (!(std::fabs(box->L[1] - L) <= 1e-12 * std::fabs(L) && std::fabs(box->L[2] - L) <= 1e-12 * std::fabs(L)))
    return sfail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  // the grid is not used here: keep the planner's spectral work minimal;
  // this entry runs the one-thread-per-atom local part, so plan for it
  if (o.n_f == 0) o.n_f = 4;
  if (o.near_variant == 0 || o.near_variant >= 3) o.near_variant = 1;
  espe::HostPlan hp;
  std::string msg;
  esp_status s = espe::make_host_plan(L, N, tolerance, o, hp, msg);
  if (s != ESP_OK) return sfail(s, msg);
  const size_t need = needed_bytes(hp, o.precision);
  if (need > kStaticBytes)
    return sfail(ESP_ERR_UNSUPPORTED,
                 "system needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                     std::to_string(kStaticBytes) + " (about 65k FP32 or 32k FP64 atoms)");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(o.device) != cudaSuccess) {
    cudaGetLastError();
    return sfail(ESP_ERR_INVALID_ARG, "cannot select the requested device");
  }
  unsigned char* scratch = nullptr;
  s = scratch_address(o.device, &scratch);
  if (s == ESP_OK && !(device_pointer(xyz, o.device) && device_pointer(q, o.device) &&
                       device_pointer(energy, o.device) && device_pointer(forces, o.device) &&
                       device_pointer(potential, o.device)))
    s = sfail(ESP_ERR_INVALID_ARG, "xyz, q and every non-NULL output must be device (or managed) memory of "
                                   "opts->device");
  cudaStream_t st = (cudaStream_t)o.stream;
  if (s == ESP_OK && N == 0) {
    if (energy && cudaMemsetAsync(energy, 0, sizeof(double), st) != cudaSuccess)
      s = sfail(ESP_ERR_CUDA, "memset of the energy failed");
  } else if (s == ESP_OK) {
    // charge sums for the neutrality check, self energy and background
    std::vector<double> hq(N);
    cudaError_t e = cudaMemcpyAsync(hq.data(), q, N * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      s = sfail(ESP_ERR_CUDA, std::string("reading charges: ") + cudaGetErrorString(e));
    } else {
      double Q = 0, Q2 = 0, Qa = 0;
      bool finite = true;
      for (double v : hq) { finite &= std::isfinite(v); Q += v; Q2 += v * v; Qa += std::fabs(v); }
      const bool neutral = std::fabs(Q) <= 1e-10 * std::max(1.0, Qa);
      if (!finite) s = sfail(ESP_ERR_NONFINITE, "a charge is NaN or infinite");
      else if (!neutral && !o.allow_background)
        s = sfail(ESP_ERR_NOT_NEUTRAL, "sum of charges is nonzero and allow_background is 0");
      else {
        if (neutral) Q = 0.0;
        s = o.precision == ESP_FP32
                ? run_local<float>(hp, scratch, xyz, q, Q, Q2, energy, forces, potential, st)
                : run_local<double>(hp, scratch, xyz, q, Q, Q2, energy, forces, potential, st);
      }
    }
  }
  cudaSetDevice(prev);
  return s;
}
