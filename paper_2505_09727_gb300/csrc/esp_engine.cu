// Single-system execution engine and the C-ABI of include/esp.h.
//
// A plan owns every device buffer of one system, two cuFFT plans and a
// second stream on which the local part (Eq. localpart) runs concurrently with
// the spectral part (Eqs. spread ... interp).
#include <cuda_runtime.h>
#include <cufft.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/esp.h"
#include "esp_launch.h"
#include "esp_plan.h"

namespace {

thread_local std::string g_error;

esp_status fail(esp_status s, const std::string& m) {
  g_error = m;
  return s;
}

#define ESP_CU(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? ESP_ERR_OOM : ESP_ERR_CUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

#define ESP_FFT(call)                                                                     \
  do {                                                                                    \
    cufftResult r_ = (call);                                                              \
    if (r_ != CUFFT_SUCCESS)                                                              \
      return fail(ESP_ERR_CUFFT, std::string(#call) + ": cufft error " + std::to_string((int)r_)); \
  } while (0)

#define ESP_TRY(expr)                   \
  do {                                  \
    esp_status s_ = (expr);             \
    if (s_ != ESP_OK) return s_;        \
  } while (0)

constexpr int kPhases = 9;

#define ESP_XSTR(x) #x
#define ESP_STR(x) ESP_XSTR(x)

}  // namespace

namespace espe {
void set_last_error(const std::string& msg) { g_error = msg; }
}  // namespace espe

struct esp_plan_s {
  espe::HostPlan hp;
  int prec = ESP_FP32;
  int device = 0;
  double timeout_ms = 60000.0;
  bool allow_bg = false;
  long long N = 0;
  int n_chunks = 0;
  int n_fourier_blocks = 0;
  size_t smem = 0;
  double Q = 0, Q2 = 0;
  bool have_q = false, have_pos = false;
  bool timing = false;
  int timing_mode = 0;          // 1: events, 2: events with serialised phases
  bool own_stream = false;
  size_t bytes = 0;
  std::vector<void*> allocs;

  // device buffers
  espk::SysDesc* d_desc = nullptr;
  int2* d_chunks = nullptr;
  int* d_chunk_first = nullptr;
  int2* d_work = nullptr;
  void* d_pos = nullptr;       // staging for host positions (FP64, N x 3)
  void* d_coord = nullptr;
  uint32_t* d_key = nullptr;
  uint32_t* d_rank = nullptr;
  uint32_t* d_count = nullptr;
  uint32_t* d_start = nullptr;
  uint32_t* d_tiles = nullptr;   // scan tile totals
  void* d_atoms = nullptr;
  void* d_rel = nullptr;         // cell-relative coordinates + charge (local part)
  uint32_t* d_perm = nullptr;
  void* d_q = nullptr;
  void* d_qstage = nullptr;    // staging for host charges (FP64)
  void* d_grid = nullptr;
  void* d_spec = nullptr;
  void* d_tabs = nullptr;
  void* d_far = nullptr;
  void* d_near = nullptr;
  double* d_fourier = nullptr;
  double* d_partials = nullptr;
  double* d_consts = nullptr;
  double* d_eout = nullptr;
  void* d_outF = nullptr;      // staging for host outputs (FP64)
  void* d_outU = nullptr;
  int* d_err = nullptr;

  cufftHandle fwd = 0, inv = 0;
  bool fwd_ok = false, inv_ok = false;
  cudaStream_t st = nullptr, st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t tev[13] = {};
  float phase_ms[kPhases] = {};
  bool timed_valid = false;     // events of the last compute were recorded
  double e_fourier = 0, e_gather = 0;
};

namespace {

esp_status dev_alloc(esp_plan_s* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ESP_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  p->bytes += bytes;
  return ESP_OK;
}

template <typename T>
esp_status dev_alloc_t(esp_plan_s* p, T** ptr, size_t count) {
  return dev_alloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

void release(esp_plan_s* p) {
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->st) cudaStreamSynchronize(p->st);
  if (p->st2) cudaStreamSynchronize(p->st2);
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  if (p->fwd_ok) cufftDestroy(p->fwd);
  if (p->inv_ok) cufftDestroy(p->inv);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  for (auto& e : p->tev) if (e) cudaEventDestroy(e);
  if (p->st2) cudaStreamDestroy(p->st2);
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  cudaSetDevice(cur);
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

// Bounded wait: poll the stream until done or the plan deadline passes.
esp_status wait_stream(esp_plan_s* p, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return ESP_OK;
    if (e != cudaErrorNotReady) return fail(ESP_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms > p->timeout_ms) return fail(ESP_ERR_TIMEOUT, "device work exceeded the plan deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

esp_status check_err_flag(esp_plan_s* p) {
  int flag = 0;
  ESP_CU(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  ESP_TRY(wait_stream(p, p->st));
  if (flag) {
    ESP_CU(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->st));
    if (flag & 1) return fail(ESP_ERR_NONFINITE, "a position is NaN or infinite");
    return fail(ESP_ERR_INTERNAL, "a kernel bounds check failed (flag " + std::to_string(flag) + ")");
  }
  return ESP_OK;
}

void rec(esp_plan_s* p, int i, cudaStream_t s) {
  if (p->timing) cudaEventRecord(p->tev[i], s);
}

template <typename real>
esp_status build_buffers(esp_plan_s* p) {
  using L = espk::Launch<real>;
  const espe::HostPlan& hp = p->hp;
  const long long N = p->N;
  const size_t rb = sizeof(real);
  p->n_chunks = (int)((N + espk::kChunk - 1) / espk::kChunk);
  std::vector<int2> chunks(p->n_chunks);
  for (int c = 0; c < p->n_chunks; ++c) chunks[c] = make_int2(0, c * espk::kChunk);
  std::vector<int2> work(hp.n_bricks);
  for (int b = 0; b < hp.n_bricks; ++b) work[b] = make_int2(0, b);
  int chunk_first[2] = {0, p->n_chunks};
  // scale grid: enough blocks to fill the GPU, capped by the spectrum size
  long long spec_threads = hp.spec_elems;
  p->n_fourier_blocks = (int)std::min<long long>(152 * 4, std::max<long long>(1, (spec_threads + 255) / 256));

  ESP_TRY(dev_alloc_t(p, &p->d_desc, 1));
  ESP_TRY(dev_alloc_t(p, &p->d_chunks, std::max(1, p->n_chunks)));
  ESP_TRY(dev_alloc_t(p, &p->d_chunk_first, 2));
  ESP_TRY(dev_alloc_t(p, &p->d_work, std::max(1, hp.n_bricks)));
  ESP_TRY(dev_alloc(p, &p->d_pos, (size_t)N * 3 * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_coord, (size_t)N * L::atom_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_key, N));
  ESP_TRY(dev_alloc_t(p, &p->d_rank, N));
  ESP_TRY(dev_alloc_t(p, &p->d_count, hp.n_keys));
  ESP_TRY(dev_alloc_t(p, &p->d_start, hp.n_keys + 1));
  ESP_TRY(dev_alloc_t(p, &p->d_tiles, espk::scan_tiles(hp.n_keys)));
  ESP_TRY(dev_alloc(p, &p->d_rel, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc(p, &p->d_atoms, (size_t)N * L::atom_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_perm, N));
  ESP_TRY(dev_alloc(p, &p->d_q, (size_t)N * rb));
  ESP_TRY(dev_alloc(p, &p->d_qstage, (size_t)N * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_grid, (size_t)hp.grid_elems * rb));
  ESP_TRY(dev_alloc(p, &p->d_spec, (size_t)hp.spec_elems * 2 * rb));
  ESP_TRY(dev_alloc(p, &p->d_tabs, (hp.G.size() + hp.W.size()) * rb));
  ESP_TRY(dev_alloc(p, &p->d_far, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc(p, &p->d_near, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_fourier, p->n_fourier_blocks));
  ESP_TRY(dev_alloc_t(p, &p->d_partials, 2 * std::max(1, p->n_chunks)));
  ESP_TRY(dev_alloc_t(p, &p->d_consts, 2));
  ESP_TRY(dev_alloc_t(p, &p->d_eout, 3));
  ESP_TRY(dev_alloc(p, &p->d_outF, (size_t)N * 3 * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_outU, (size_t)N * sizeof(double)));
  ESP_TRY(dev_alloc_t(p, &p->d_err, 1));

  std::vector<real> tabs(hp.G.size() + hp.W.size());
  for (size_t i = 0; i < hp.G.size(); ++i) tabs[i] = (real)hp.G[i];
  for (size_t i = 0; i < hp.W.size(); ++i) tabs[hp.G.size() + i] = (real)hp.W[i];
  espk::SysDesc d = hp.desc;
  ESP_CU(cudaMemcpyAsync(p->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, p->st));
  if (p->n_chunks)
    ESP_CU(cudaMemcpyAsync(p->d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_chunk_first, chunk_first, sizeof(chunk_first), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_tabs, tabs.data(), tabs.size() * rb, cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->st));
  ESP_CU(cudaMemsetAsync(p->d_consts, 0, 2 * sizeof(double), p->st));
  p->smem = (size_t)hp.desc.T * hp.desc.T * hp.desc.T * rb;

  const int n = hp.desc.n_f;
  const bool f32 = sizeof(real) == 4;
  ESP_FFT(cufftPlan3d(&p->fwd, n, n, n, f32 ? CUFFT_R2C : CUFFT_D2Z));
  p->fwd_ok = true;
  ESP_FFT(cufftPlan3d(&p->inv, n, n, n, f32 ? CUFFT_C2R : CUFFT_Z2D));
  p->inv_ok = true;
  ESP_FFT(cufftSetStream(p->fwd, p->st));
  ESP_FFT(cufftSetStream(p->inv, p->st));
  size_t ws = 0;
  if (cufftGetSize(p->fwd, &ws) == CUFFT_SUCCESS) p->bytes += ws;
  if (cufftGetSize(p->inv, &ws) == CUFFT_SUCCESS) p->bytes += ws;
  ESP_CU(cudaStreamSynchronize(p->st));
  return ESP_OK;
}

template <typename real>
esp_status do_set_charges(esp_plan_s* p, const void* q, bool is_double, int where) {
  using L = espk::Launch<real>;
  const long long N = p->N;
  // FP64 host copy for the charge sums (and the staging source)
  std::vector<double> hq(N);
  if (where == ESP_HOST) {
    if (is_double) std::memcpy(hq.data(), q, N * sizeof(double));
    else for (long long i = 0; i < N; ++i) hq[i] = ((const float*)q)[i];
  } else {
    if (is_double) {
      ESP_CU(cudaMemcpyAsync(hq.data(), q, N * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    } else {
      std::vector<float> tmp(N);
      ESP_CU(cudaMemcpyAsync(tmp.data(), q, N * sizeof(float), cudaMemcpyDeviceToHost, p->st));
      ESP_TRY(wait_stream(p, p->st));
      for (long long i = 0; i < N; ++i) hq[i] = tmp[i];
    }
    ESP_TRY(wait_stream(p, p->st));
  }
  double Q = 0, Q2 = 0, Qa = 0;
  for (long long i = 0; i < N; ++i) {
    if (!std::isfinite(hq[i])) return fail(ESP_ERR_NONFINITE, "a charge is NaN or infinite");
    Q += hq[i];
    Q2 += hq[i] * hq[i];
    Qa += std::fabs(hq[i]);
  }
  if (std::fabs(Q) > 1e-10 * std::max(1.0, Qa) && !p->allow_bg)
    return fail(ESP_ERR_NOT_NEUTRAL, "sum of charges is " + std::to_string(Q) +
                                         "; set allow_background for a neutralising background");
  if (std::fabs(Q) <= 1e-10 * std::max(1.0, Qa)) Q = 0.0;
  ESP_CU(cudaMemcpyAsync(p->d_qstage, hq.data(), N * sizeof(double), cudaMemcpyHostToDevice, p->st));
  ESP_CU((cudaError_t)L::convert_charges(p->d_qstage, true, (real*)p->d_q, N, p->st));
  double consts[2], bg_shift;
  espe::charge_constants(p->hp, Q, Q2, &consts[0], &consts[1], &bg_shift);
  p->hp.desc.bg_shift = bg_shift;
  espk::SysDesc d = p->hp.desc;
  ESP_CU(cudaMemcpyAsync(p->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_consts, consts, sizeof(consts), cudaMemcpyHostToDevice, p->st));
  ESP_TRY(wait_stream(p, p->st));
  p->Q = Q;
  p->Q2 = Q2;
  p->have_q = true;
  return ESP_OK;
}

template <typename real>
esp_status do_set_positions(esp_plan_s* p, const void* xyz, bool is_double, int where) {
  using L = espk::Launch<real>;
  const long long N = p->N;
  const void* src = xyz;
  bool src_double = is_double;
  rec(p, 0, p->st);
  if (where == ESP_HOST && N > 0) {
    ESP_CU(cudaMemcpyAsync(p->d_pos, xyz, N * 3 * (is_double ? sizeof(double) : sizeof(float)),
                           cudaMemcpyHostToDevice, p->st));
    src = p->d_pos;
  }
  ESP_CU(cudaMemsetAsync(p->d_count, 0, p->hp.n_keys * sizeof(uint32_t), p->st));
  ESP_CU(L::ingest(p->d_desc, p->d_chunks, p->n_chunks, src, src_double, p->d_coord, p->d_key,
                   p->d_rank, p->d_count, p->d_err, p->st));
  ESP_CU(espk::launch_scan(p->d_count, p->d_start, p->d_tiles, p->hp.n_keys, p->st));
  rec(p, 1, p->st);
  p->have_pos = true;
  if (where == ESP_HOST) return wait_stream(p, p->st);
  return ESP_OK;
}

template <typename real>
esp_status do_compute(esp_plan_s* p, double* energy, void* forces, void* potential, bool out_double,
                      int where) {
  using L = espk::Launch<real>;
  if (!p->have_q) return fail(ESP_ERR_NOT_READY, "charges not set");
  if (!p->have_pos) return fail(ESP_ERR_NOT_READY, "positions not set");
  const espe::HostPlan& hp = p->hp;
  const long long N = p->N;
  const int P = hp.info.P;
  cudaStream_t st = p->st, st2 = p->st2;

  void* outF = forces;
  void* outU = potential;
  double* outE = energy;
  if (where == ESP_HOST) {
    outF = forces ? p->d_outF : nullptr;
    outU = potential ? p->d_outU : nullptr;
    outE = nullptr;
  }

  rec(p, 2, st);
  // A1b: scatter into cell order
  ESP_CU(L::scatter(p->d_desc, p->d_chunks, p->n_chunks, p->d_coord, p->d_key, p->d_rank, p->d_start,
                    (const real*)p->d_q, p->d_atoms, p->d_rel, p->d_perm, st));
  rec(p, 12, st);
  // fork: local part on the second stream (on the main stream when timing
  // mode 2 serialises the phases so each kernel is timed alone)
  const bool serial = p->timing_mode == 2;
  if (serial) st2 = st;
  else {
    ESP_CU(cudaEventRecord(p->ev_fork, st));
    ESP_CU(cudaStreamWaitEvent(st2, p->ev_fork, 0));
  }
  rec(p, 9, st2);
  const espk::NearCoef<real>& nc = *reinterpret_cast<const espk::NearCoef<real>*>(
      sizeof(real) == 4 ? (const void*)&hp.nc32 : (const void*)&hp.nc64);
  const espk::SICoef<real>& si = *reinterpret_cast<const espk::SICoef<real>*>(
      sizeof(real) == 4 ? (const void*)&hp.si32 : (const void*)&hp.si64);
  ESP_CU(L::near(p->d_desc, p->d_chunks, p->n_chunks, p->d_atoms, p->d_rel, p->d_start, p->d_near, nc,
                 hp.near_nc, hp.near_queued, st2));
  rec(p, 10, st2);
  if (!serial) ESP_CU(cudaEventRecord(p->ev_join, st2));

  // spectral part
  rec(p, 3, st);
  ESP_CU(cudaMemsetAsync(p->d_grid, 0, hp.grid_elems * sizeof(real), st));
  ESP_CU(L::spread(P, p->d_desc, p->d_work, hp.n_bricks, p->smem, p->d_atoms, p->d_start,
                   (real*)p->d_grid, si, p->d_err, st));
  rec(p, 4, st);
  if (sizeof(real) == 4)
    ESP_FFT(cufftExecR2C(p->fwd, (cufftReal*)p->d_grid, (cufftComplex*)p->d_spec));
  else
    ESP_FFT(cufftExecD2Z(p->fwd, (cufftDoubleReal*)p->d_grid, (cufftDoubleComplex*)p->d_spec));
  rec(p, 5, st);
  ESP_CU(L::scale(p->d_desc, 1, p->n_fourier_blocks, p->d_spec, (const real*)p->d_tabs, p->d_fourier, st));
  rec(p, 6, st);
  if (sizeof(real) == 4)
    ESP_FFT(cufftExecC2R(p->inv, (cufftComplex*)p->d_spec, (cufftReal*)p->d_grid));
  else
    ESP_FFT(cufftExecZ2D(p->inv, (cufftDoubleComplex*)p->d_spec, (cufftDoubleReal*)p->d_grid));
  rec(p, 7, st);
  ESP_CU(L::gather(P, p->d_desc, p->d_work, hp.n_bricks, p->smem, p->d_atoms, p->d_start,
                   (const real*)p->d_grid, p->d_far, si, p->d_err, st));
  rec(p, 8, st);
  // join and finish
  if (!serial) ESP_CU(cudaStreamWaitEvent(st, p->ev_join, 0));
  ESP_CU(L::finalize(p->d_desc, p->d_chunks, p->n_chunks, p->d_atoms, p->d_perm, p->d_far, p->d_near,
                     outF, outU, out_double, p->d_partials, st));
  ESP_CU(espk::launch_energy(p->d_desc, 1, p->d_fourier, p->n_fourier_blocks, p->d_partials,
                             p->n_chunks, p->d_chunk_first, p->d_consts, p->d_eout, outE, st));
  rec(p, 11, st);

  if (where == ESP_HOST) {
    const size_t ob = out_double ? sizeof(double) : sizeof(float);
    if (forces) ESP_CU(cudaMemcpyAsync(forces, p->d_outF, N * 3 * ob, cudaMemcpyDeviceToHost, st));
    if (potential) ESP_CU(cudaMemcpyAsync(potential, p->d_outU, N * ob, cudaMemcpyDeviceToHost, st));
    double e3[3];
    ESP_CU(cudaMemcpyAsync(e3, p->d_eout, sizeof(e3), cudaMemcpyDeviceToHost, st));
    ESP_TRY(wait_stream(p, st));
    if (energy) *energy = e3[0];
    p->e_fourier = e3[1];
    p->e_gather = e3[2];
    ESP_TRY(check_err_flag(p));
  }
  p->timed_valid = p->timing;
  return ESP_OK;
}

}  // namespace

// ====================================================================== C-ABI
extern "C" {

void esp_plan_opts_init(esp_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kernel = ESP_KERNEL_PSWF;
  o->precision = ESP_FP32;
  o->prefactor = 1.0;
  o->allow_background = 1;
  o->timeout_ms = 60000.0;
}

esp_status esp_plan(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                    esp_plan_t* out) {
  if (!box || !out) return fail(ESP_ERR_INVALID_ARG, "box and out must not be NULL");
  *out = nullptr;
  esp_plan_opts o;
  if (opts) o = *opts;
  else esp_plan_opts_init(&o);
  const double L = box->L[0];
  if (!(std::fabs(box->L[1] - L) <= 1e-12 * std::fabs(L) && std::fabs(box->L[2] - L) <= 1e-12 * std::fabs(L)))
    return fail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  esp_plan_s* p = new esp_plan_s();
  std::string msg;
  esp_status s = espe::make_host_plan(L, N, tolerance, o, p->hp, msg);
  if (s != ESP_OK) {
    delete p;
    return fail(s, msg);
  }
  p->prec = o.precision;
  p->device = o.device;
  p->timeout_ms = o.timeout_ms > 0 ? o.timeout_ms : 60000.0;
  p->allow_bg = o.allow_background != 0;
  p->N = N;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    delete p;
    return fail(ESP_ERR_CUDA, "no CUDA device available");
  }
  if (o.device < 0 || o.device >= ndev) {
    delete p;
    return fail(ESP_ERR_INVALID_ARG, "device ordinal out of range");
  }
  DeviceGuard g(p->device);
  auto bail = [&](esp_status st) {
    std::string m = g_error;
    release(p);
    delete p;
    return fail(st, m);
  };
  if (o.stream) {
    p->st = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(ESP_ERR_CUDA, "stream creation failed"));
    p->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(ESP_ERR_CUDA, "stream/event creation failed"));
  for (auto& e : p->tev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(ESP_ERR_CUDA, "event creation failed"));
  s = p->prec == ESP_FP32 ? build_buffers<float>(p) : build_buffers<double>(p);
  if (s != ESP_OK) return bail(s);
  p->hp.info.device_bytes = p->bytes;
  *out = p;
  return ESP_OK;
}

esp_status esp_plan_query(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                          esp_plan_params* out) {
  if (!box || !out) return fail(ESP_ERR_INVALID_ARG, "box and out must not be NULL");
  esp_plan_opts o;
  if (opts) o = *opts;
  else esp_plan_opts_init(&o);
  const double L = box->L[0];
  if (!(std::fabs(box->L[1] - L) <= 1e-12 * std::fabs(L) && std::fabs(box->L[2] - L) <= 1e-12 * std::fabs(L)))
    return fail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  espe::HostPlan hp;
  std::string msg;
  esp_status s = espe::make_host_plan(L, N, tolerance, o, hp, msg);
  if (s != ESP_OK) return fail(s, msg);
  const size_t rb = o.precision == ESP_FP32 ? 4 : 8;
  const size_t ab = o.precision == ESP_FP32 ? 16 : 32;
  size_t bytes = (size_t)N * (24 + 2 * ab + 4 * 3 + rb + 8 + 2 * ab + 32) +
                 (size_t)hp.n_keys * 8 + (size_t)hp.grid_elems * rb + (size_t)hp.spec_elems * 2 * rb +
                 (hp.G.size() + hp.W.size()) * rb;
  hp.info.device_bytes = bytes;
  *out = hp.info;
  return ESP_OK;
}

esp_status esp_plan_info(esp_plan_t p, esp_plan_params* out) {
  if (!p || !out) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  *out = p->hp.info;
  return ESP_OK;
}

static esp_status set_charges_any(esp_plan_t p, const void* q, bool dbl, int where) {
  if (!p || (!q && p->N > 0)) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (where != ESP_HOST && where != ESP_DEVICE) return fail(ESP_ERR_INVALID_ARG, "bad 'where'");
  DeviceGuard g(p->device);
  return p->prec == ESP_FP32 ? do_set_charges<float>(p, q, dbl, where)
                             : do_set_charges<double>(p, q, dbl, where);
}

esp_status esp_set_charges(esp_plan_t p, const double* q, int where) { return set_charges_any(p, q, true, where); }
esp_status esp_set_charges_f32(esp_plan_t p, const float* q, int where) { return set_charges_any(p, q, false, where); }

static esp_status set_positions_any(esp_plan_t p, const void* x, bool dbl, int where) {
  if (!p || (!x && p->N > 0)) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (where != ESP_HOST && where != ESP_DEVICE) return fail(ESP_ERR_INVALID_ARG, "bad 'where'");
  DeviceGuard g(p->device);
  esp_status s = p->prec == ESP_FP32 ? do_set_positions<float>(p, x, dbl, where)
                                     : do_set_positions<double>(p, x, dbl, where);
  if (s == ESP_OK && where == ESP_HOST) s = check_err_flag(p);
  return s;
}

esp_status esp_set_positions(esp_plan_t p, const double* xyz, int where) { return set_positions_any(p, xyz, true, where); }
esp_status esp_set_positions_f32(esp_plan_t p, const float* xyz, int where) { return set_positions_any(p, xyz, false, where); }

static esp_status compute_any(esp_plan_t p, double* e, void* f, void* u, bool dbl, int where) {
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL plan");
  if (where != ESP_HOST && where != ESP_DEVICE) return fail(ESP_ERR_INVALID_ARG, "bad 'where'");
  DeviceGuard g(p->device);
  if (p->N == 0) {
    if (e) {
      if (where == ESP_HOST) *e = 0.0;
      else if (cudaMemsetAsync(e, 0, sizeof(double), p->st) != cudaSuccess) return fail(ESP_ERR_CUDA, "memset");
    }
    return ESP_OK;
  }
  return p->prec == ESP_FP32 ? do_compute<float>(p, e, f, u, dbl, where)
                             : do_compute<double>(p, e, f, u, dbl, where);
}

esp_status esp_compute(esp_plan_t p, double* energy, double* forces, double* potential, int where) {
  return compute_any(p, energy, forces, potential, true, where);
}
esp_status esp_compute_f32(esp_plan_t p, double* energy, float* forces, float* potential, int where) {
  return compute_any(p, energy, forces, potential, false, where);
}

esp_status esp_synchronize(esp_plan_t p) {
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL plan");
  DeviceGuard g(p->device);
  ESP_TRY(wait_stream(p, p->st));
  ESP_TRY(wait_stream(p, p->st2));
  return check_err_flag(p);
}

esp_status esp_set_timing(esp_plan_t p, int enable) {
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL plan");
  p->timing = enable != 0;
  p->timing_mode = enable;
  return ESP_OK;
}

esp_status esp_phase_times(esp_plan_t p, float* ms, int n) {
  if (!p || !ms) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (!p->timing || !p->timed_valid) return fail(ESP_ERR_NOT_READY, "timing is off or no timed compute yet");
  DeviceGuard g(p->device);
  ESP_TRY(wait_stream(p, p->st));
  auto el = [&](int a, int b) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p->tev[a], p->tev[b]);
    return t;
  };
  p->phase_ms[0] = el(0, 1) + el(2, 12);  // ingest + scan, scatter
  p->phase_ms[1] = el(3, 4);              // spread (with grid clear)
  p->phase_ms[2] = el(4, 5);              // R2C FFT
  p->phase_ms[3] = el(5, 6);              // scale + energy
  p->phase_ms[4] = el(6, 7);              // C2R FFT
  p->phase_ms[5] = el(7, 8);              // gather
  p->phase_ms[6] = el(9, 10);             // near (second stream)
  p->phase_ms[7] = el(8, 11);             // join, finalize, energy
  p->phase_ms[8] = el(2, 11);             // whole compute
  for (int i = 0; i < n && i < kPhases; ++i) ms[i] = p->phase_ms[i];
  return ESP_OK;
}

esp_status esp_last_spectral_energy(esp_plan_t p, double* e_fourier, double* e_gather) {
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL plan");
  if (e_fourier) *e_fourier = p->e_fourier;
  if (e_gather) *e_gather = p->e_gather;
  return ESP_OK;
}

esp_status esp_destroy(esp_plan_t p) {
  if (!p) return ESP_OK;
  release(p);
  delete p;
  return ESP_OK;
}

const char* esp_last_error(void) { return g_error.c_str(); }

const char* esp_version(void) { return "esp_gb300 0.1 (sm_103a; CUDA " ESP_STR(CUDART_VERSION) ")"; }

}  // extern "C"
