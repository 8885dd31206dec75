// Execution engine and the C-ABI of include/esp.h.
//
// Everything runs on a pool of independent systems: the device arrays hold
// the systems back to back (atoms, cell lists, grids, spectra, influence
// tables), the kernels read per-system descriptors and work lists, and the
// FFTs run as one batched cuFFT plan per grid size. A plan (esp_plan) is a
// pool of one system; a batch (esp_batch_create) is a pool of many whose
// whole step is replayed from a CUDA graph. The local part (Eq. localpart)
// runs on a second stream concurrently with the spectral part
// (Eqs. spread ... interp).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "../../include/esp.h"
#include "esp_engine.h"
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
constexpr int kFourierBlocks = 152 * 4;   // scale-kernel blocks per system, at most

#define ESP_XSTR(x) #x
#define ESP_STR(x) ESP_XSTR(x)

// One batched FFT plan per grid size; the grids (and spectra) of its systems
// are consecutive in the pool.
struct Bucket {
  int n_f = 0;
  int count = 0;
  long long grid0 = 0, spec0 = 0;
  cufftHandle fwd = 0, inv = 0;
  bool fwd_ok = false, inv_ok = false;
};

}  // namespace

namespace espe {
void set_last_error(const std::string& msg) { g_error = msg; }
}  // namespace espe

struct esp_plan_s {
  std::vector<espe::HostPlan> hps;     // per system, offsets zero
  std::vector<espk::SysDesc> descs;    // per system, with pool offsets
  int nsys = 0;
  int prec = ESP_FP32;
  int P = 0;
  int device = 0;
  double timeout_ms = 60000.0;
  bool allow_bg = false;
  long long N = 0;                     // atoms of all systems
  long long n_keys = 0, grid_total = 0, spec_total = 0, tab_total = 0;
  long long n_cols = 0, cmap_cap = 0;  // cell-list columns, cluster-list capacity
  int n_chunks = 0, n_work = 0, F = 1;
  size_t smem = 0;                     // spread/gather tile bytes (largest system)
  std::vector<Bucket> buckets;
  std::vector<double> Q, Q2;
  bool have_q = false, have_pos = false;
  bool timing = false;
  int timing_mode = 0;                 // 1: events, 2: events with serialised phases
  bool own_stream = false;
  size_t bytes = 0;
  std::vector<void*> allocs;

  // device buffers
  espk::SysDesc* d_desc = nullptr;
  int2* d_chunks = nullptr;
  int* d_chunk_first = nullptr;
  int2* d_work = nullptr;
  void* d_pos = nullptr;       // staging for positions (FP64, N x 3)
  void* d_coord = nullptr;
  uint32_t* d_key = nullptr;
  uint32_t* d_rank = nullptr;
  uint32_t* d_count = nullptr;
  uint32_t* d_start = nullptr;
  uint32_t* d_tiles = nullptr;   // scan tile totals
  void* d_atoms = nullptr;
  void* d_rel = nullptr;         // pair records of the local part
  uint32_t* d_perm = nullptr;
  void* d_q = nullptr;
  void* d_qstage = nullptr;      // staging for charges (FP64)
  void* d_grid = nullptr;
  void* d_spec = nullptr;
  void* d_grid_ik = nullptr;     // ik method: three gradient grids, component-major
  void* d_spec_ik = nullptr;     // ... and their three half spectra
  bool ik = false;
  void* d_tabs = nullptr;
  void* d_far = nullptr;
  void* d_near = nullptr;
  double* d_fourier = nullptr;
  double* d_partials = nullptr;
  unsigned* d_ticket = nullptr;        // finalize's CTA ticket (zero between launches)
  double* d_consts = nullptr;
  double* d_eout = nullptr;      // per system: E, E_fourier, E_gather
  double* d_vpart = nullptr;     // virial: spectral partials [nsys][F][6]
  double* d_vloc = nullptr;      // virial: local part [nsys][6] (atomics)
  double* d_vout = nullptr;      // virial: totals [nsys][6]
  bool virial = false;
  bool computed = false;         // a compute has been enqueued
  int* h_flag = nullptr;         // pinned host copy of the device error flag
  double* d_energy = nullptr;    // per system: E (batch output)
  void* d_outF = nullptr;        // staging for outputs (FP64)
  void* d_outU = nullptr;
  int* d_err = nullptr;
  uint32_t* d_ccount = nullptr;  // clusters per column (local part, FP32)
  uint32_t* d_cstart = nullptr;
  uint32_t* d_ctiles = nullptr;
  int2* d_cmap = nullptr;
  int2* d_catoms = nullptr;

  cudaStream_t st = nullptr, st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_scat = nullptr;
  cudaEvent_t tev[14] = {};
  float phase_ms[kPhases] = {};
  bool timed_valid = false;      // events of the last compute were recorded
  std::vector<double> e_fourier, e_gather;

  // batches: one step captured as a CUDA graph after a first direct run
  int direct_runs = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;

  // single plans: the compute captured as a CUDA graph for its output
  // pointers (re-captured when they change; given up after kMaxRecaptures)
  int c_direct_runs = 0, c_captures = 0;
  cudaGraph_t cgraph = nullptr;
  cudaGraphExec_t cgexec = nullptr;
  const void* ckey[4] = {};
  // esp_step: sort + compute captured together, keyed like the compute graph
  // plus the position source
  int s_direct_runs = 0, s_captures = 0;
  cudaGraph_t sgraph = nullptr;
  cudaGraphExec_t sgexec = nullptr;
  const void* skey[5] = {};
  // exclusions (single plans): pairs of caller indices, and the inverse of
  // the sort permutation they are mapped through
  int2* d_excl = nullptr;
  long long n_excl = 0, excl_cap = 0;
  uint32_t* d_inv = nullptr;
};

struct esp_batch_s {
  esp_plan_s pool;
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
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cgexec) cudaGraphExecDestroy(p->cgexec);
  if (p->cgraph) cudaGraphDestroy(p->cgraph);
  if (p->sgexec) cudaGraphExecDestroy(p->sgexec);
  if (p->sgraph) cudaGraphDestroy(p->sgraph);
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  for (Bucket& b : p->buckets) {
    if (b.fwd_ok) cufftDestroy(b.fwd);
    if (b.inv_ok) cufftDestroy(b.inv);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_scat) cudaEventDestroy(p->ev_scat);
  for (auto& e : p->tev) if (e) cudaEventDestroy(e);
  if (p->st2) cudaStreamDestroy(p->st2);
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  p->h_flag = nullptr;
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
// Bounded wait: polls without sleeping for the first 2 ms (a step's host
// round trip is then a few microseconds), then every 20 us until the
// plan's deadline.
esp_status wait_stream(esp_plan_s* p, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return ESP_OK;
    if (e != cudaErrorNotReady) return fail(ESP_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms > p->timeout_ms) return fail(ESP_ERR_TIMEOUT, "device work exceeded the plan deadline");
    if (ms < 2.0) std::this_thread::yield();
    else std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// The device error flag: its read is enqueued with a call's other copies
// (one wait for all), then interpreted.
esp_status enqueue_flag_read(esp_plan_s* p) {
  ESP_CU(cudaMemcpyAsync(p->h_flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  return ESP_OK;
}

esp_status flag_result(esp_plan_s* p) {
  const int flag = *p->h_flag;
  if (flag) {
    *p->h_flag = 0;
    ESP_CU(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->st));
    if (flag & 1) return fail(ESP_ERR_NONFINITE, "a position is NaN or infinite");
    return fail(ESP_ERR_INTERNAL, "a kernel bounds check failed (flag " + std::to_string(flag) + ")");
  }
  return ESP_OK;
}

esp_status check_err_flag(esp_plan_s* p) {
  ESP_TRY(enqueue_flag_read(p));
  ESP_TRY(wait_stream(p, p->st));
  return flag_result(p);
}

void rec(esp_plan_s* p, int i, cudaStream_t s) {
  if (p->timing) cudaEventRecord(p->tev[i], s);
}

// Pool layout: per-system offsets, chunk and brick work lists, FFT buckets.
void layout(esp_plan_s* p, std::vector<int2>& chunks, std::vector<int>& chunk_first,
            std::vector<int2>& work) {
  const int n = p->nsys;
  p->descs.resize(n);
  std::map<int, std::vector<int>> by_nf;
  for (int s = 0; s < n; ++s) by_nf[p->hps[s].desc.n_f].push_back(s);
  long long grid0 = 0, spec0 = 0;
  p->buckets.clear();
  for (auto& kv : by_nf) {
    Bucket b;
    b.n_f = kv.first;
    b.count = (int)kv.second.size();
    b.grid0 = grid0;
    b.spec0 = spec0;
    for (int s : kv.second) {
      p->descs[s] = p->hps[s].desc;
      p->descs[s].grid0 = grid0;
      p->descs[s].spec0 = spec0;
      grid0 += p->hps[s].grid_elems;
      spec0 += p->hps[s].spec_elems;
    }
    p->buckets.push_back(b);
  }
  p->grid_total = grid0;
  p->spec_total = spec0;
  long long atom0 = 0, cell0 = 0, tab0 = 0, col0 = 0, max_spec = 0;
  chunks.clear();
  work.clear();
  chunk_first.assign(n + 1, 0);
  p->smem = 0;
  const size_t rb = p->prec == ESP_FP32 ? 4 : 8;
  for (int s = 0; s < n; ++s) {
    espk::SysDesc& d = p->descs[s];
    const espe::HostPlan& hp = p->hps[s];
    d.atom0 = atom0;
    d.cell0 = cell0;
    d.tab0 = tab0;
    d.col0 = col0;
    chunk_first[s] = (int)chunks.size();
    for (int c = 0; c * espk::kChunk < d.n_atoms; ++c) chunks.push_back(make_int2(s, c * espk::kChunk));
    for (int b = 0; b < hp.n_bricks; ++b) work.push_back(make_int2(s, b));
    atom0 += d.n_atoms;
    cell0 += hp.n_keys;
    tab0 += (long long)(hp.G.size() + hp.W.size() + hp.H.size());
    col0 += (long long)d.n_c * d.n_c;
    p->smem = std::max(p->smem, (size_t)d.tpz * d.T * rb);
    max_spec = std::max(max_spec, hp.spec_elems);
  }
  chunk_first[n] = (int)chunks.size();
  p->N = atom0;
  p->n_keys = cell0;
  p->tab_total = tab0;
  p->n_cols = col0;
  p->cmap_cap = atom0 / espk::kClusterAtomsHost + col0 + 1;
  p->n_chunks = (int)chunks.size();
  p->n_work = (int)work.size();
  // scale grid: enough blocks to fill the GPU, capped by the spectrum size
  p->F = (int)std::min<long long>(kFourierBlocks, std::max<long long>(1, (max_spec + 255) / 256));
}

template <typename real>
esp_status build_buffers(esp_plan_s* p) {
  using L = espk::Launch<real>;
  std::vector<int2> chunks, work;
  std::vector<int> chunk_first;
  layout(p, chunks, chunk_first, work);
  const long long N = p->N;
  const int n = p->nsys;
  const size_t rb = sizeof(real);

  ESP_TRY(dev_alloc_t(p, &p->d_desc, n));
  ESP_TRY(dev_alloc_t(p, &p->d_chunks, std::max(1, p->n_chunks)));
  ESP_TRY(dev_alloc_t(p, &p->d_chunk_first, n + 1));
  ESP_TRY(dev_alloc_t(p, &p->d_work, std::max(1, p->n_work)));
  ESP_TRY(dev_alloc(p, &p->d_pos, (size_t)N * 3 * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_coord, (size_t)N * L::atom_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_key, N));
  ESP_TRY(dev_alloc_t(p, &p->d_rank, N));
  ESP_TRY(dev_alloc_t(p, &p->d_count, p->n_keys));
  ESP_TRY(dev_alloc_t(p, &p->d_start, p->n_keys + 1));
  ESP_TRY(dev_alloc_t(p, &p->d_tiles, espk::scan_tiles(p->n_keys)));
  ESP_TRY(dev_alloc(p, &p->d_rel, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc(p, &p->d_atoms, (size_t)N * L::atom_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_perm, N));
  ESP_TRY(dev_alloc(p, &p->d_q, (size_t)N * rb));
  ESP_TRY(dev_alloc(p, &p->d_qstage, (size_t)N * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_grid, (size_t)p->grid_total * rb));
  ESP_TRY(dev_alloc(p, &p->d_spec, (size_t)p->spec_total * 2 * rb));
  p->ik = p->hps[0].info.diff == ESP_DIFF_IK;
  if (p->ik) {
    ESP_TRY(dev_alloc(p, &p->d_grid_ik, (size_t)p->grid_total * 3 * rb));
    ESP_TRY(dev_alloc(p, &p->d_spec_ik, (size_t)p->spec_total * 3 * 2 * rb));
  }
  ESP_TRY(dev_alloc(p, &p->d_tabs, (size_t)p->tab_total * rb));
  ESP_TRY(dev_alloc(p, &p->d_far, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc(p, &p->d_near, (size_t)N * L::res_bytes()));
  ESP_TRY(dev_alloc_t(p, &p->d_fourier, (size_t)p->F * n));
  ESP_TRY(dev_alloc_t(p, &p->d_partials, 2 * std::max(1, p->n_chunks)));
  ESP_TRY(dev_alloc_t(p, &p->d_ticket, 1));
  ESP_TRY(dev_alloc_t(p, &p->d_consts, 2 * n));
  ESP_TRY(dev_alloc_t(p, &p->d_eout, 3 * n));
  p->virial = p->hps[0].info.virial != 0;
  if (p->virial) {
    ESP_TRY(dev_alloc_t(p, &p->d_vpart, (size_t)n * p->F * 6));
    ESP_TRY(dev_alloc_t(p, &p->d_vloc, (size_t)n * 6));
    ESP_TRY(dev_alloc_t(p, &p->d_vout, (size_t)n * 6));
  }
  ESP_TRY(dev_alloc_t(p, &p->d_energy, n));
  ESP_TRY(dev_alloc(p, &p->d_outF, (size_t)N * 3 * sizeof(double)));
  ESP_TRY(dev_alloc(p, &p->d_outU, (size_t)N * sizeof(double)));
  ESP_TRY(dev_alloc_t(p, &p->d_err, 1));
  if (p->hps[0].near_clusters) {
    ESP_TRY(dev_alloc_t(p, &p->d_ccount, std::max<long long>(1, p->n_cols)));
    ESP_TRY(dev_alloc_t(p, &p->d_cstart, p->n_cols + 1));
    ESP_TRY(dev_alloc_t(p, &p->d_ctiles, espk::scan_tiles(p->n_cols)));
    ESP_TRY(dev_alloc_t(p, &p->d_cmap, p->cmap_cap));
    ESP_TRY(dev_alloc_t(p, &p->d_catoms, p->cmap_cap * espk::kClusterAtomsHost));
  }

  std::vector<real> tabs(std::max<long long>(1, p->tab_total));
  for (int s = 0; s < n; ++s) {
    const espe::HostPlan& hp = p->hps[s];
    const long long t0 = p->descs[s].tab0;
    for (size_t i = 0; i < hp.G.size(); ++i) tabs[t0 + i] = (real)hp.G[i];
    for (size_t i = 0; i < hp.W.size(); ++i) tabs[t0 + hp.G.size() + i] = (real)hp.W[i];
    for (size_t i = 0; i < hp.H.size(); ++i) tabs[t0 + hp.G.size() + hp.W.size() + i] = (real)hp.H[i];
  }
  ESP_CU(cudaMemcpyAsync(p->d_desc, p->descs.data(), n * sizeof(espk::SysDesc), cudaMemcpyHostToDevice, p->st));
  if (p->n_chunks)
    ESP_CU(cudaMemcpyAsync(p->d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_chunk_first, chunk_first.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, p->st));
  if (p->n_work)
    ESP_CU(cudaMemcpyAsync(p->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_tabs, tabs.data(), p->tab_total * rb, cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->st));
  ESP_CU(cudaMemsetAsync(p->d_ticket, 0, sizeof(unsigned), p->st));
  ESP_CU(cudaMemsetAsync(p->d_consts, 0, 2 * n * sizeof(double), p->st));

  const bool f32 = sizeof(real) == 4;
  for (Bucket& b : p->buckets) {
    int dims[3] = {b.n_f, b.n_f, b.n_f};
    const int real_elems = b.n_f * b.n_f * b.n_f;
    const int cplx_elems = b.n_f * b.n_f * (b.n_f / 2 + 1);
    ESP_FFT(cufftPlanMany(&b.fwd, 3, dims, nullptr, 1, real_elems, nullptr, 1, cplx_elems,
                          f32 ? CUFFT_R2C : CUFFT_D2Z, b.count));
    b.fwd_ok = true;
    ESP_FFT(cufftPlanMany(&b.inv, 3, dims, nullptr, 1, cplx_elems, nullptr, 1, real_elems,
                          f32 ? CUFFT_C2R : CUFFT_Z2D, b.count));
    b.inv_ok = true;
    ESP_FFT(cufftSetStream(b.fwd, p->st));
    ESP_FFT(cufftSetStream(b.inv, p->st));
    size_t ws = 0;
    if (cufftGetSize(b.fwd, &ws) == CUFFT_SUCCESS) p->bytes += ws;
    if (cufftGetSize(b.inv, &ws) == CUFFT_SUCCESS) p->bytes += ws;
  }
  p->Q.assign(n, 0.0);
  p->Q2.assign(n, 0.0);
  p->e_fourier.assign(n, 0.0);
  p->e_gather.assign(n, 0.0);
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
  std::vector<double> Qs(p->nsys), Q2s(p->nsys), consts(2 * p->nsys);
  for (int s = 0; s < p->nsys; ++s) {
    const espk::SysDesc& d = p->descs[s];
    double Q = 0, Q2 = 0, Qa = 0;
    for (long long i = d.atom0; i < d.atom0 + d.n_atoms; ++i) {
      if (!std::isfinite(hq[i])) return fail(ESP_ERR_NONFINITE, "a charge is NaN or infinite");
      Q += hq[i];
      Q2 += hq[i] * hq[i];
      Qa += std::fabs(hq[i]);
    }
    const bool neutral = std::fabs(Q) <= 1e-10 * std::max(1.0, Qa);
    if (!neutral && !p->allow_bg) {
      const std::string who = p->nsys > 1 ? "of system " + std::to_string(s) + " " : "";
      return fail(ESP_ERR_NOT_NEUTRAL, "sum of charges " + who + "is " + std::to_string(Q) +
                                           "; set allow_background for a neutralising background");
    }
    Qs[s] = neutral ? 0.0 : Q;
    Q2s[s] = Q2;
  }
  for (int s = 0; s < p->nsys; ++s) {
    double bg_shift;
    espe::charge_constants(p->hps[s], Qs[s], Q2s[s], &consts[2 * s], &consts[2 * s + 1], &bg_shift);
    p->descs[s].bg_shift = bg_shift;
    p->descs[s].bg_shift_f = (float)bg_shift;
  }
  ESP_CU(cudaMemcpyAsync(p->d_qstage, hq.data(), N * sizeof(double), cudaMemcpyHostToDevice, p->st));
  ESP_CU((cudaError_t)L::convert_charges(p->d_qstage, true, (real*)p->d_q, N, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_desc, p->descs.data(), p->nsys * sizeof(espk::SysDesc),
                         cudaMemcpyHostToDevice, p->st));
  ESP_CU(cudaMemcpyAsync(p->d_consts, consts.data(), consts.size() * sizeof(double), cudaMemcpyHostToDevice,
                         p->st));
  ESP_TRY(wait_stream(p, p->st));
  p->Q = Qs;
  p->Q2 = Q2s;
  p->have_q = true;
  return ESP_OK;
}

// Steps A0-A1: ingest (wrap, convert, finite check, cell keys) and the
// counting-sort scan of positions at `src` (device memory).
template <typename real>
esp_status launch_sort(esp_plan_s* p, const void* src, bool src_double) {
  using L = espk::Launch<real>;
  ESP_CU(cudaMemsetAsync(p->d_count, 0, p->n_keys * sizeof(uint32_t), p->st));
  ESP_CU(L::ingest(p->d_desc, p->d_chunks, p->n_chunks, src, src_double, p->d_coord, p->d_key,
                   p->d_rank, p->d_count, p->d_err, p->st));
  ESP_CU(espk::launch_scan(p->d_count, p->d_start, p->d_tiles, p->n_keys, p->st));
  return ESP_OK;
}

template <typename real>
esp_status do_set_positions(esp_plan_s* p, const void* xyz, bool is_double, int where) {
  const long long N = p->N;
  const void* src = xyz;
  rec(p, 0, p->st);
  if (where == ESP_HOST && N > 0) {
    ESP_CU(cudaMemcpyAsync(p->d_pos, xyz, N * 3 * (is_double ? sizeof(double) : sizeof(float)),
                           cudaMemcpyHostToDevice, p->st));
    src = p->d_pos;
  }
  ESP_TRY(launch_sort<real>(p, src, is_double));
  rec(p, 1, p->st);
  p->have_pos = true;
  if (where == ESP_HOST) {
    // the caller may reuse xyz on return; the ingest's finiteness check is
    // read in the same wait
    ESP_TRY(enqueue_flag_read(p));
    ESP_TRY(wait_stream(p, p->st));
    return flag_result(p);
  }
  return ESP_OK;
}

// Every kernel and FFT of one compute on the pool, enqueued without any
// host synchronisation (and therefore capturable in a CUDA graph).
template <typename real>
esp_status launch_compute(esp_plan_s* p, void* outF, void* outU, bool out_double, double* outE) {
  using L = espk::Launch<real>;
  const espe::HostPlan& hp = p->hps[0];   // P and the polynomial tables are common to the pool
  cudaStream_t st = p->st, st2 = p->st2;

  rec(p, 2, st);
  // fork: local part on the second stream (on the main stream when timing
  // mode 2 serialises the phases so each kernel is timed alone). Its cluster
  // lists need only the cell offsets of the sort, so they are built while the
  // main stream scatters the atoms; the pair kernel waits for the scatter.
  const bool serial = p->timing_mode == 2;
  if (serial) st2 = st;
  else {
    ESP_CU(cudaEventRecord(p->ev_fork, st));
    ESP_CU(cudaStreamWaitEvent(st2, p->ev_fork, 0));
  }
  const espk::NearCoef<real>& nc = *reinterpret_cast<const espk::NearCoef<real>*>(
      sizeof(real) == 4 ? (const void*)&hp.nc32 : (const void*)&hp.nc64);
  const espk::SICoef<real>& si = *reinterpret_cast<const espk::SICoef<real>*>(
      sizeof(real) == 4 ? (const void*)&hp.si32 : (const void*)&hp.si64);
  if (hp.near_clusters) {
    // cluster lists (timed with the bin sort)
    rec(p, 13, st2);
    ESP_CU(L::near_clusters(p->d_desc, p->nsys, p->n_cols, p->d_start, p->d_rel, p->d_near, nc, hp.near_nc,
                            p->d_ccount, p->d_cstart, p->d_ctiles, p->d_cmap, p->d_catoms, p->cmap_cap,
                            hp.near_half, p->N, 2, p->d_err, st2));
  }
  // A1b: scatter into cell order
  ESP_CU(L::scatter(p->d_desc, p->d_chunks, p->n_chunks, p->d_coord, p->d_key, p->d_rank, p->d_start,
                    (const real*)p->d_q, p->d_atoms, p->d_rel, p->d_perm, st));
  rec(p, 12, st);
  if (!serial) {
    ESP_CU(cudaEventRecord(p->ev_scat, st));
    ESP_CU(cudaStreamWaitEvent(st2, p->ev_scat, 0));
  }
  if (p->virial) ESP_CU(cudaMemsetAsync(p->d_vloc, 0, (size_t)p->nsys * 6 * sizeof(double), st2));
  if (hp.near_clusters) {
    // the pair kernel alone between the local-part events
    rec(p, 9, st2);
    ESP_CU(L::near_clusters(p->d_desc, p->nsys, p->n_cols, p->d_start, p->d_rel, p->d_near, nc, hp.near_nc,
                            p->d_ccount, p->d_cstart, p->d_ctiles, p->d_cmap, p->d_catoms, p->cmap_cap,
                            hp.near_half, p->N, 1, p->d_err, st2, p->d_vloc, hp.desc.tri != 0));
  } else {
    rec(p, 9, st2);
    ESP_CU(L::near(p->d_desc, p->d_chunks, p->n_chunks, p->d_atoms, p->d_rel, p->d_start, p->d_near, nc,
                   hp.near_nc, hp.near_queued, st2, p->d_vloc));
  }
  if (p->n_excl > 0)
    ESP_CU(L::exclusions(p->d_desc, p->d_excl, p->n_excl, p->d_perm, p->d_inv, p->N, p->d_atoms, p->d_near, st2));
  rec(p, 10, st2);
  if (!serial) ESP_CU(cudaEventRecord(p->ev_join, st2));

  // spectral part
  rec(p, 3, st);
  ESP_CU(cudaMemsetAsync(p->d_grid, 0, p->grid_total * sizeof(real), st));
  ESP_CU(L::spread(p->P, p->d_desc, p->d_work, p->n_work, p->smem, p->d_atoms, p->d_start,
                   (real*)p->d_grid, si, p->d_err, st));
  rec(p, 4, st);
  for (Bucket& b : p->buckets) {
    if (sizeof(real) == 4)
      ESP_FFT(cufftExecR2C(b.fwd, (cufftReal*)p->d_grid + b.grid0, (cufftComplex*)p->d_spec + b.spec0));
    else
      ESP_FFT(cufftExecD2Z(b.fwd, (cufftDoubleReal*)p->d_grid + b.grid0,
                           (cufftDoubleComplex*)p->d_spec + b.spec0));
  }
  rec(p, 5, st);
  ESP_CU(L::scale(p->d_desc, p->nsys, p->F, p->d_spec, (const real*)p->d_tabs, p->d_fourier, p->d_spec_ik,
                  p->spec_total, p->d_vpart, st));
  rec(p, 6, st);
  // energy only (no forces, no potentials): E needs the spectral sum of the
  // scale kernel and the local part, not the inverse FFT and the gather
  const bool atom_outputs = outF != nullptr || outU != nullptr;
  for (Bucket& b : p->buckets) {
    if (!atom_outputs) break;
    if (sizeof(real) == 4)
      ESP_FFT(cufftExecC2R(b.inv, (cufftComplex*)p->d_spec + b.spec0, (cufftReal*)p->d_grid + b.grid0));
    else
      ESP_FFT(cufftExecZ2D(b.inv, (cufftDoubleComplex*)p->d_spec + b.spec0,
                           (cufftDoubleReal*)p->d_grid + b.grid0));
  }
  if (p->ik && atom_outputs) {
    // ik method: the three gradient spectra back to the grid
    for (int a = 0; a < 3; ++a) {
      for (Bucket& b : p->buckets) {
        const long long so = a * p->spec_total + b.spec0, go = a * p->grid_total + b.grid0;
        if (sizeof(real) == 4)
          ESP_FFT(cufftExecC2R(b.inv, (cufftComplex*)p->d_spec_ik + so, (cufftReal*)p->d_grid_ik + go));
        else
          ESP_FFT(cufftExecZ2D(b.inv, (cufftDoubleComplex*)p->d_spec_ik + so, (cufftDoubleReal*)p->d_grid_ik + go));
      }
    }
  }
  rec(p, 7, st);
  if (atom_outputs)
    ESP_CU(L::gather(p->P, p->d_desc, p->d_work, p->n_work, p->smem, p->d_atoms, p->d_start,
                     (const real*)p->d_grid, (const real*)p->d_grid_ik, p->grid_total, p->d_far, si, p->d_err, st));
  rec(p, 8, st);
  // join and finish
  if (!serial) ESP_CU(cudaStreamWaitEvent(st, p->ev_join, 0));
  // per-atom totals; for one or two systems the finalize kernel's last CTA
  // combines the energies (one launch less), for more a CTA per system does
  espk::EnergyArgs ea;
  ea.nsys = p->nsys;
  ea.fourier = p->d_fourier;
  ea.n_fourier_blocks = p->F;
  ea.chunk_first = p->d_chunk_first;
  ea.consts = p->d_consts;
  ea.out = p->d_eout;
  ea.user_energy = outE;
  ea.vpart = p->d_vpart;
  ea.vloc = p->d_vloc;
  ea.vout = p->d_vout;
  const bool fused_energy = p->nsys <= 2;
  ea.ticket = fused_energy ? p->d_ticket : nullptr;
  ESP_CU(L::finalize(p->d_desc, p->d_chunks, p->n_chunks, p->d_atoms, p->d_perm,
                     atom_outputs ? p->d_far : nullptr, p->d_near,
                     outF, outU, out_double, p->d_partials, st, ea));
  if (!fused_energy)
    ESP_CU(espk::launch_energy(p->d_desc, p->nsys, p->d_fourier, p->F, p->d_partials, p->n_chunks,
                               p->d_chunk_first, p->d_consts, p->d_eout, outE, st, p->d_vpart, p->d_vloc,
                               p->d_vout));
  p->computed = true;
  rec(p, 11, st);
  return ESP_OK;
}

// Host tail of a compute with host outputs: copies, bounded wait, energies,
// device error flag.
// The device address of a page-locked host buffer mapped into the device's
// address space (nullptr for any other pointer).
void* mapped_host(const void* h) {
  if (!h) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

esp_status finish_host(esp_plan_s* p, double* energy, void* forces, void* potential, bool out_double) {
  const long long N = p->N;
  const size_t ob = out_double ? sizeof(double) : sizeof(float);
  if (forces) ESP_CU(cudaMemcpyAsync(forces, p->d_outF, N * 3 * ob, cudaMemcpyDeviceToHost, p->st));
  if (potential) ESP_CU(cudaMemcpyAsync(potential, p->d_outU, N * ob, cudaMemcpyDeviceToHost, p->st));
  std::vector<double> e3(3 * p->nsys);
  ESP_CU(cudaMemcpyAsync(e3.data(), p->d_eout, e3.size() * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  ESP_TRY(enqueue_flag_read(p));
  ESP_TRY(wait_stream(p, p->st));
  for (int s = 0; s < p->nsys; ++s) {
    if (energy) energy[s] = e3[3 * s];
    p->e_fourier[s] = e3[3 * s + 1];
    p->e_gather[s] = e3[3 * s + 2];
  }
  return flag_result(p);
}

constexpr int kMaxRecaptures = 4;

// One compute on the plan's streams: directly while timing (the phase events
// are recorded then), for the first run, inside a caller's own capture, or
// once the output pointers have changed too often; otherwise as a replay of
// the captured graph for these output pointers (no launch gaps between the
// dependent kernels).
template <typename real>
esp_status compute_enqueue(esp_plan_s* p, void* outF, void* outU, bool out_double, double* outE) {
  const void* key[4] = {outF, outU, out_double ? (const void*)1 : nullptr, outE};
  const bool same = std::equal(key, key + 4, p->ckey);
  if (p->cgexec && same && !p->timing) {
    ESP_CU(cudaGraphLaunch(p->cgexec, p->st));
    return ESP_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ESP_CU(cudaStreamIsCapturing(p->st, &cs));
  if (p->timing || p->c_direct_runs == 0 || cs != cudaStreamCaptureStatusNone || p->c_captures >= kMaxRecaptures) {
    ++p->c_direct_runs;
    return launch_compute<real>(p, outF, outU, out_double, outE);
  }
  cudaGraph_t graph = nullptr;
  ESP_CU(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
  const esp_status s = launch_compute<real>(p, outF, outU, out_double, outE);
  const cudaError_t e = cudaStreamEndCapture(p->st, &graph);
  if (s != ESP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(ESP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (p->cgexec) cudaGraphExecDestroy(p->cgexec);
  if (p->cgraph) cudaGraphDestroy(p->cgraph);
  if (p->sgexec) cudaGraphExecDestroy(p->sgexec);
  if (p->sgraph) cudaGraphDestroy(p->sgraph);
  p->cgexec = nullptr;
  p->cgraph = graph;
  ++p->c_captures;
  ESP_CU(cudaGraphInstantiate(&p->cgexec, graph, 0));
  std::copy(key, key + 4, p->ckey);
  ESP_CU(cudaGraphLaunch(p->cgexec, p->st));
  return ESP_OK;
}

template <typename real>
esp_status do_compute(esp_plan_s* p, double* energy, void* forces, void* potential, bool out_double,
                      int where) {
  if (!p->have_q) return fail(ESP_ERR_NOT_READY, "charges not set");
  if (!p->have_pos) return fail(ESP_ERR_NOT_READY, "positions not set");
  void* outF = forces;
  void* outU = potential;
  double* outE = energy;
  if (where == ESP_HOST) {
    outF = forces ? p->d_outF : nullptr;
    outU = potential ? p->d_outU : nullptr;
    outE = nullptr;
  }
  ESP_TRY(compute_enqueue<real>(p, outF, outU, out_double, outE));
  if (where == ESP_HOST) ESP_TRY(finish_host(p, energy, forces, potential, out_double));
  p->timed_valid = p->timing;
  return ESP_OK;
}

// esp_step: positions at `src` (device) sorted and computed; after a first
// direct run, sort and compute replay as one captured graph for the same
// source and output pointers.
template <typename real>
esp_status step_enqueue(esp_plan_s* p, const void* src, void* outF, void* outU, bool out_double, double* outE) {
  const void* key[5] = {outF, outU, out_double ? (const void*)1 : nullptr, outE, src};
  // inside a caller's stream capture (e.g. a step graph of the MD loop) the
  // kernels are launched directly into it
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ESP_CU(cudaStreamIsCapturing(p->st, &cs));
  if (cs == cudaStreamCaptureStatusNone && p->sgexec && std::equal(key, key + 5, p->skey)) {
    ESP_CU(cudaGraphLaunch(p->sgexec, p->st));
    return ESP_OK;
  }
  if (p->s_direct_runs == 0 || cs != cudaStreamCaptureStatusNone || p->s_captures >= kMaxRecaptures) {
    ++p->s_direct_runs;
    ESP_TRY(launch_sort<real>(p, src, true));
    return launch_compute<real>(p, outF, outU, out_double, outE);
  }
  cudaGraph_t graph = nullptr;
  ESP_CU(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
  esp_status st = launch_sort<real>(p, src, true);
  if (st == ESP_OK) st = launch_compute<real>(p, outF, outU, out_double, outE);
  const cudaError_t e = cudaStreamEndCapture(p->st, &graph);
  if (st != ESP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(ESP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (p->sgexec) cudaGraphExecDestroy(p->sgexec);
  if (p->sgraph) cudaGraphDestroy(p->sgraph);
  p->sgexec = nullptr;
  p->sgraph = graph;
  ++p->s_captures;
  ESP_CU(cudaGraphInstantiate(&p->sgexec, graph, 0));
  std::copy(key, key + 5, p->skey);
  ESP_CU(cudaGraphLaunch(p->sgexec, p->st));
  return ESP_OK;
}

template <typename real>
esp_status do_step(esp_plan_s* p, const double* xyz, double* energy, void* forces, void* potential, bool out_double,
                   int where) {
  if (!p->have_q) return fail(ESP_ERR_NOT_READY, "charges not set");
  if (p->timing) {
    // timing mode: the two calls, with their phase events
    ESP_TRY(do_set_positions<real>(p, xyz, true, where));
    return do_compute<real>(p, energy, forces, potential, out_double, where);
  }
  const void* src = xyz;
  void* outF = forces;
  void* outU = potential;
  double* outE = energy;
  if (where == ESP_HOST) {
    // positions in a page-locked host buffer mapped into the device's
    // address space are read in place by the ingest (coalesced, over the
    // CPU-GPU link): no staging copy. Results go back by copies: the
    // finalize writes them in caller order, scattered, which the link
    // serves worse than one bulk copy
    const void* xyz_dev = mapped_host(xyz);
    if (xyz_dev) {
      src = xyz_dev;
    } else {
      ESP_CU(cudaMemcpyAsync(p->d_pos, xyz, p->N * 3 * sizeof(double), cudaMemcpyHostToDevice, p->st));
      src = p->d_pos;
    }
    outF = forces ? p->d_outF : nullptr;
    outU = potential ? p->d_outU : nullptr;
    outE = nullptr;
  }
  ESP_TRY(step_enqueue<real>(p, src, outF, outU, out_double, outE));
  p->have_pos = true;
  p->timed_valid = false;
  if (where == ESP_HOST) ESP_TRY(finish_host(p, energy, forces, potential, out_double));
  return ESP_OK;
}


esp_status create_streams(esp_plan_s* p, const esp_plan_opts& o) {
  if (o.stream) {
    p->st = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ESP_ERR_CUDA, "stream creation failed");
    p->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_scat, cudaEventDisableTiming) != cudaSuccess)
    return fail(ESP_ERR_CUDA, "stream/event creation failed");
  for (auto& e : p->tev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(ESP_ERR_CUDA, "event creation failed");
  if (cudaMallocHost(reinterpret_cast<void**>(&p->h_flag), sizeof(int)) != cudaSuccess)
    return fail(ESP_ERR_CUDA, "pinned host allocation failed");
  *p->h_flag = 0;
  return ESP_OK;
}

// Device state of a pool whose host plans p->hps are made.
esp_status finish_pool(esp_plan_s* p, const esp_plan_opts& o) {
  p->prec = o.precision;
  p->device = o.device;
  p->timeout_ms = o.timeout_ms > 0 ? o.timeout_ms : 60000.0;
  p->allow_bg = o.allow_background != 0;
  p->nsys = (int)p->hps.size();
  p->P = p->hps[0].info.P;
  for (const espe::HostPlan& hp : p->hps)
    if (hp.info.P != p->P || hp.near_nc != p->hps[0].near_nc)
      return fail(ESP_ERR_INTERNAL, "systems of one pool differ in stencil width or local-part terms");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(ESP_ERR_CUDA, "no CUDA device available");
  }
  if (o.device < 0 || o.device >= ndev) return fail(ESP_ERR_INVALID_ARG, "device ordinal out of range");
  DeviceGuard g(p->device);
  ESP_TRY(create_streams(p, o));
  ESP_TRY(p->prec == ESP_FP32 ? build_buffers<float>(p) : build_buffers<double>(p));
  for (espe::HostPlan& hp : p->hps) hp.info.device_bytes = p->bytes;
  return ESP_OK;
}

esp_plan_opts resolve_opts(const esp_plan_opts* opts) {
  esp_plan_opts o;
  if (opts) o = *opts;
  else esp_plan_opts_init(&o);
  return o;
}

bool cubic(const esp_box& b) {
  const double L = b.L[0];
  return std::fabs(b.L[1] - L) <= 1e-12 * std::fabs(L) && std::fabs(b.L[2] - L) <= 1e-12 * std::fabs(L);
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

// A single-system plan from the box (cubic: cell == nullptr) or the cell.
static esp_status plan_single(const esp_box* box, const esp_cell* cell, int64_t N, double tolerance,
                              const esp_plan_opts* opts, esp_plan_t* out) {
  if ((!box && !cell) || !out) return fail(ESP_ERR_INVALID_ARG, "box/cell and out must not be NULL");
  *out = nullptr;
  const esp_plan_opts o = resolve_opts(opts);
  if (box && !cubic(*box)) return fail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  esp_plan_s* p = new esp_plan_s();
  p->hps.resize(1);
  std::string msg;
  esp_status s = box ? espe::make_host_plan(box->L[0], N, tolerance, o, p->hps[0], msg)
                     : espe::make_host_plan_cell(&cell->a[0], N, tolerance, o, p->hps[0], msg);
  if (s != ESP_OK) {
    delete p;
    return fail(s, msg);
  }
  s = finish_pool(p, o);
  if (s != ESP_OK) {
    const std::string m = g_error;
    release(p);
    delete p;
    return fail(s, m);
  }
  *out = p;
  return ESP_OK;
}

static esp_status query_single(const esp_box* box, const esp_cell* cell, int64_t N, double tolerance,
                               const esp_plan_opts* opts, esp_plan_params* out) {
  if ((!box && !cell) || !out) return fail(ESP_ERR_INVALID_ARG, "box/cell and out must not be NULL");
  const esp_plan_opts o = resolve_opts(opts);
  if (box && !cubic(*box)) return fail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  espe::HostPlan hp;
  std::string msg;
  esp_status s = box ? espe::make_host_plan(box->L[0], N, tolerance, o, hp, msg)
                     : espe::make_host_plan_cell(&cell->a[0], N, tolerance, o, hp, msg);
  if (s != ESP_OK) return fail(s, msg);
  const size_t rb = o.precision == ESP_FP32 ? 4 : 8;
  const size_t ab = o.precision == ESP_FP32 ? 16 : 32;
  size_t bytes = (size_t)N * (24 + 2 * ab + 4 * 3 + rb + 8 + 2 * ab + 32) +
                 (size_t)hp.n_keys * 8 + (size_t)hp.grid_elems * rb + (size_t)hp.spec_elems * 2 * rb +
                 (hp.G.size() + hp.W.size() + hp.H.size()) * rb;
  if (o.diff == ESP_DIFF_IK) bytes += 3 * ((size_t)hp.grid_elems * rb + (size_t)hp.spec_elems * 2 * rb);
  if (hp.near_clusters) {
    // cluster counts, offsets and lists of the local part
    const size_t n_cols = (size_t)hp.desc.n_c * hp.desc.n_c;
    const size_t cap = (size_t)N / espk::kClusterAtomsHost + n_cols + 1;
    bytes += n_cols * 8 + cap * (8 + 8 * espk::kClusterAtomsHost);
  }
  hp.info.device_bytes = bytes;
  *out = hp.info;
  return ESP_OK;
}

esp_status esp_plan(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                    esp_plan_t* out) {
  if (!box) return fail(ESP_ERR_INVALID_ARG, "box must not be NULL");
  return plan_single(box, nullptr, N, tolerance, opts, out);
}

esp_status esp_plan_cell(const esp_cell* cell, int64_t N, double tolerance, const esp_plan_opts* opts,
                         esp_plan_t* out) {
  if (!cell) return fail(ESP_ERR_INVALID_ARG, "cell must not be NULL");
  return plan_single(nullptr, cell, N, tolerance, opts, out);
}

esp_status esp_plan_query(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                          esp_plan_params* out) {
  if (!box) return fail(ESP_ERR_INVALID_ARG, "box must not be NULL");
  return query_single(box, nullptr, N, tolerance, opts, out);
}

esp_status esp_plan_query_cell(const esp_cell* cell, int64_t N, double tolerance, const esp_plan_opts* opts,
                               esp_plan_params* out) {
  if (!cell) return fail(ESP_ERR_INVALID_ARG, "cell must not be NULL");
  return query_single(nullptr, cell, N, tolerance, opts, out);
}

esp_status esp_influence_query(const esp_box* box, const esp_cell* cell, int64_t N, double tolerance,
                               const esp_plan_opts* opts, double* out, int64_t* len) {
  if (!len || (!box) == (!cell)) return fail(ESP_ERR_INVALID_ARG, "pass exactly one of box and cell, and len");
  const esp_plan_opts o = resolve_opts(opts);
  if (box && !cubic(*box)) return fail(ESP_ERR_INVALID_ARG, "only cubic boxes are supported (L[0] = L[1] = L[2])");
  espe::HostPlan hp;
  std::string msg;
  esp_status s = box ? espe::make_host_plan(box->L[0], N, tolerance, o, hp, msg)
                     : espe::make_host_plan_cell(&cell->a[0], N, tolerance, o, hp, msg);
  if (s != ESP_OK) return fail(s, msg);
  const int n = hp.desc.n_f, nh = n / 2 + 1, half = n / 2;
  const int64_t total = (int64_t)n * n * nh;
  const int64_t cap = *len;
  *len = total;
  if (!out) return ESP_OK;
  if (cap < total) return fail(ESP_ERR_INVALID_ARG, "out holds fewer than n_f^2 (n_f/2 + 1) entries");
  const bool tri = hp.desc.tri != 0;
  int64_t idx = 0;
  for (int kzi = 0; kzi < n; ++kzi)
    for (int kyi = 0; kyi < n; ++kyi)
      for (int kx = 0; kx < nh; ++kx, ++idx) {
        // the scale kernel's product, in FP64
        const int ky = kyi < half ? kyi : kyi - n, kz = kzi < half ? kzi : kzi - n;
        const double g = tri ? hp.G[idx] : hp.G[kx * kx + ky * ky + kz * kz];
        out[idx] = g * hp.W[kx] * hp.W[std::abs(ky)] * hp.W[std::abs(kz)];
      }
  return ESP_OK;
}

esp_status esp_plan_info(esp_plan_t p, esp_plan_params* out) {
  if (!p || !out) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  *out = p->hps[0].info;
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

esp_status esp_step(esp_plan_t p, const double* xyz, double* energy, double* forces, double* potential, int where) {
  if (!p || (!xyz && p->N > 0)) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (where != ESP_HOST && where != ESP_DEVICE) return fail(ESP_ERR_INVALID_ARG, "bad 'where'");
  DeviceGuard g(p->device);
  if (p->N == 0) return compute_any(p, energy, forces, potential, true, where);
  return p->prec == ESP_FP32 ? do_step<float>(p, xyz, energy, forces, potential, true, where)
                             : do_step<double>(p, xyz, energy, forces, potential, true, where);
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
  if (enable < 0 || enable > 2) return fail(ESP_ERR_INVALID_ARG, "timing mode must be 0, 1 or 2");
  p->timing = enable != 0;
  p->timing_mode = enable;
  return ESP_OK;
}

esp_status esp_phase_times(esp_plan_t p, float* ms, int n) {
  if (!p || !ms) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (!p->timing || !p->timed_valid) return fail(ESP_ERR_NOT_READY, "timing is off or no timed compute yet");
  DeviceGuard g(p->device);
  ESP_TRY(wait_stream(p, p->st));
  // a pair of events that was not recorded (e.g. positions set before timing
  // was enabled) reads as 0; its error is cleared so that later launches do
  // not see it
  auto el = [&](int a, int b) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->tev[a], p->tev[b]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    return t;
  };
  // ingest + scan, then scatter and (concurrently) the cluster lists
  p->phase_ms[0] = el(0, 1) + (p->hps[0].near_clusters ? el(2, 9) : el(2, 12));
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

esp_status esp_set_exclusions(esp_plan_t p, const int32_t* pairs, int64_t n_pairs) {
  if (!p || n_pairs < 0 || (n_pairs > 0 && !pairs)) return fail(ESP_ERR_INVALID_ARG, "NULL plan or pairs, or n_pairs < 0");
  if (p->nsys != 1) return fail(ESP_ERR_UNSUPPORTED, "exclusions belong to single-system plans");
  if (p->virial && n_pairs > 0) return fail(ESP_ERR_UNSUPPORTED, "exclusions are not combined with the virial");
  std::vector<std::pair<int32_t, int32_t>> sorted_pairs((size_t)n_pairs);
  for (int64_t k = 0; k < n_pairs; ++k) {
    const int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    if (i < 0 || j < 0 || i >= p->N || j >= p->N || i == j)
      return fail(ESP_ERR_INVALID_ARG, "exclusion pair " + std::to_string(k) + " = (" + std::to_string(i) + ", " +
                                           std::to_string(j) + ") is not two distinct atoms of the plan");
    sorted_pairs[k] = std::make_pair((int32_t)std::min(i, j), (int32_t)std::max(i, j));
  }
  // a pair listed twice, in either order, would be subtracted twice
  std::sort(sorted_pairs.begin(), sorted_pairs.end());
  for (size_t k = 1; k < sorted_pairs.size(); ++k)
    if (sorted_pairs[k] == sorted_pairs[k - 1])
      return fail(ESP_ERR_INVALID_ARG, "exclusion pair (" + std::to_string(sorted_pairs[k].first) + ", " +
                                           std::to_string(sorted_pairs[k].second) + ") is listed more than once");
  DeviceGuard g(p->device);
  ESP_TRY(wait_stream(p, p->st));                // nothing in flight reads the old list
  if (n_pairs > p->excl_cap) {
    if (p->d_excl) {
      p->allocs.erase(std::find(p->allocs.begin(), p->allocs.end(), (void*)p->d_excl));
      p->bytes -= (size_t)p->excl_cap * sizeof(int2);
      cudaFree(p->d_excl);
      p->d_excl = nullptr;
      p->excl_cap = 0;
    }
    ESP_TRY(dev_alloc_t(p, &p->d_excl, (size_t)n_pairs));
    p->excl_cap = n_pairs;
  }
  if (n_pairs > 0 && !p->d_inv) ESP_TRY(dev_alloc_t(p, &p->d_inv, (size_t)std::max<long long>(1, p->N)));
  if (n_pairs > 0)
    ESP_CU(cudaMemcpy(p->d_excl, pairs, (size_t)n_pairs * sizeof(int2), cudaMemcpyHostToDevice));
  p->n_excl = n_pairs;
  // the captured graphs hold the old launch sequence
  if (p->cgexec) cudaGraphExecDestroy(p->cgexec);
  if (p->cgraph) cudaGraphDestroy(p->cgraph);
  if (p->sgexec) cudaGraphExecDestroy(p->sgexec);
  if (p->sgraph) cudaGraphDestroy(p->sgraph);
  p->cgexec = nullptr;
  p->cgraph = nullptr;
  p->sgexec = nullptr;
  p->sgraph = nullptr;
  std::fill(p->ckey, p->ckey + 4, nullptr);
  std::fill(p->skey, p->skey + 5, nullptr);
  return ESP_OK;
}

esp_status esp_last_virial(esp_plan_t p, double* virial) {
  if (!p || !virial) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (!p->virial) return fail(ESP_ERR_NOT_READY, "the plan was made without opts.virial");
  if (!p->computed) return fail(ESP_ERR_NOT_READY, "no compute yet");
  DeviceGuard g(p->device);
  ESP_CU(cudaMemcpyAsync(virial, p->d_vout, 6 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  return wait_stream(p, p->st);
}

esp_status esp_last_spectral_energy(esp_plan_t p, double* e_fourier, double* e_gather) {
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL plan");
  if (e_fourier) *e_fourier = p->e_fourier[0];
  if (e_gather) *e_gather = p->e_gather[0];
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

// ============================================================ server hooks
namespace {

template <typename real>
esp_status enqueue_step(esp_plan_s* p, const double* xyz, double* forces, double* potential, double* energy,
                        int* err_host, cudaEvent_t done) {
  const long long N = p->N;
  ESP_CU(cudaMemcpyAsync(p->d_pos, xyz, N * 3 * sizeof(double), cudaMemcpyHostToDevice, p->st));
  ESP_TRY(launch_sort<real>(p, p->d_pos, true));
  p->have_pos = true;
  ESP_TRY(compute_enqueue<real>(p, p->d_outF, p->d_outU, true, nullptr));
  ESP_CU(cudaMemcpyAsync(forces, p->d_outF, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  ESP_CU(cudaMemcpyAsync(potential, p->d_outU, N * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  ESP_CU(cudaMemcpyAsync(energy, p->d_eout, sizeof(double), cudaMemcpyDeviceToHost, p->st));
  ESP_CU(cudaMemcpyAsync(err_host, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  ESP_CU(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->st));
  ESP_CU(cudaEventRecord(done, p->st));
  return ESP_OK;
}

}  // namespace

namespace espe {

esp_status plan_enqueue_step(esp_plan_t p, const double* xyz, double* forces, double* potential,
                             double* energy, int* err_host, cudaEvent_t done) {
  if (!p || !xyz || !forces || !potential || !energy || !err_host) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_q) return fail(ESP_ERR_NOT_READY, "charges not set");
  if (p->N == 0) return fail(ESP_ERR_INVALID_ARG, "empty system");
  DeviceGuard g(p->device);
  return p->prec == ESP_FP32 ? enqueue_step<float>(p, xyz, forces, potential, energy, err_host, done)
                             : enqueue_step<double>(p, xyz, forces, potential, energy, err_host, done);
}

size_t plan_device_bytes(esp_plan_t p) { return p ? p->bytes : 0; }

int plan_device(esp_plan_t p) { return p ? p->device : 0; }

cudaStream_t plan_stream(esp_plan_t p) { return p ? p->st : nullptr; }

}  // namespace espe

// ==================================================================== batches
namespace {

// Grid sizes of a batch: even 2^a 3^b 5^c 7^d sizes at least 12% apart, so
// systems of similar size share one batched FFT plan.
int bucket_size(int n_f) {
  static const std::vector<int> ladder = [] {
    std::vector<int> v;
    int last = 0;
    for (int n = 4; n <= 1024; n += 2) {
      if (!espm::is_smooth(n)) continue;
      if (last == 0 || n >= 1.12 * last) {
        v.push_back(n);
        last = n;
      }
    }
    return v;
  }();
  for (int n : ladder)
    if (n >= n_f) return n;
  return n_f;
}

// Host plans of a batch: every system plans alone, the most frequent
// SI-kernel shape c1/c becomes common (the spread and gather kernels take one
// coefficient set), each system re-plans with it, and its grid is raised to
// the next ladder size. A larger grid at fixed c1 only lowers the aliasing
// estimate, so each system still meets the tolerance.
esp_status batch_plans(const esp_box* boxes, const int64_t* N, int nsys, double tol, const esp_plan_opts& o,
                       std::vector<espe::HostPlan>& hps) {
  hps.assign(nsys, espe::HostPlan());
  std::string msg;
  std::map<long long, int> votes;
  double c = 0.0;
  for (int s = 0; s < nsys; ++s) {
    if (!cubic(boxes[s]))
      return fail(ESP_ERR_INVALID_ARG, "system " + std::to_string(s) + ": only cubic boxes are supported");
    esp_status st = espe::make_host_plan(boxes[s].L[0], N[s], tol, o, hps[s], msg);
    if (st != ESP_OK) return fail(st, "system " + std::to_string(s) + ": " + msg);
    c = hps[s].info.c;
    votes[std::llround(hps[s].info.c1 / c * 1000.0)] += 1;
  }
  long long ratio = votes.begin()->first;
  int most = -1;
  for (auto& kv : votes)
    if (kv.second > most) { ratio = kv.first; most = kv.second; }
  for (int s = 0; s < nsys; ++s) {
    esp_plan_opts oo = o;
    oo.c = c;
    oo.c1 = c * (double)ratio / 1000.0;
    espe::HostPlan tmp;
    esp_status st = espe::make_host_plan(boxes[s].L[0], N[s], tol, oo, tmp, msg);
    if (st == ESP_OK && o.n_f <= 0) {
      oo.n_f = bucket_size(tmp.info.n_f);
      st = espe::make_host_plan(boxes[s].L[0], N[s], tol, oo, hps[s], msg);
    } else if (st == ESP_OK) {
      hps[s] = tmp;
    }
    if (st != ESP_OK) return fail(st, "system " + std::to_string(s) + ": " + msg);
  }
  // One spread launch serves every system with the batch's largest tile, so
  // a system whose brick shape gives an outlying tile (a single brick across
  // a small box, say) shrinks every CTA's warp count: such systems are
  // re-planned with the largest smaller brick whose tile is within two
  // points of the batch's median tile.
  if (o.brick_cells <= 0 && nsys > 2) {
    std::vector<int> tiles(nsys);
    for (int s = 0; s < nsys; ++s) tiles[s] = hps[s].desc.T;
    std::nth_element(tiles.begin(), tiles.begin() + nsys / 2, tiles.end());
    const int t_cap = tiles[nsys / 2] + 2;
    for (int s = 0; s < nsys; ++s) {
      if (hps[s].desc.T <= t_cap) continue;
      for (int b = hps[s].desc.bc - 1; b >= 1; --b) {
        esp_plan_opts oo = o;
        oo.c = hps[s].info.c;
        oo.c1 = hps[s].info.c1;
        oo.n_f = hps[s].info.n_f;
        oo.brick_cells = b;
        espe::HostPlan tmp;
        if (espe::make_host_plan(boxes[s].L[0], N[s], tol, oo, tmp, msg) != ESP_OK) continue;
        if (tmp.desc.T <= t_cap) {
          hps[s] = tmp;
          break;
        }
      }
    }
  }
  return ESP_OK;
}

template <typename real>
esp_status batch_step(esp_plan_s* p) {
  rec(p, 0, p->st);
  ESP_TRY(launch_sort<real>(p, p->d_pos, true));
  rec(p, 1, p->st);
  return launch_compute<real>(p, p->d_outF, p->d_outU, true, p->d_energy);
}

esp_status run_batch_step(esp_plan_s* p) {
  return p->prec == ESP_FP32 ? batch_step<float>(p) : batch_step<double>(p);
}

// Capture one step into p->gexec (after a first direct run has set every
// kernel attribute and loaded every module).
esp_status capture_batch_step(esp_plan_s* p) {
  cudaGraph_t graph = nullptr;
  ESP_CU(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
  esp_status s = run_batch_step(p);
  cudaError_t e = cudaStreamEndCapture(p->st, &graph);
  if (s != ESP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(ESP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  p->graph = graph;
  ESP_CU(cudaGraphInstantiate(&p->gexec, graph, 0));
  return ESP_OK;
}

esp_plan_s* pool_of(esp_batch_t b) { return b ? &b->pool : nullptr; }

}  // namespace

extern "C" {

esp_status esp_batch_create(const esp_box* boxes, const int64_t* N, int n_systems, double tolerance,
                            const esp_plan_opts* opts, esp_batch_t* out) {
  if (!boxes || !N || !out) return fail(ESP_ERR_INVALID_ARG, "boxes, N and out must not be NULL");
  *out = nullptr;
  if (n_systems <= 0) return fail(ESP_ERR_INVALID_ARG, "n_systems must be positive");
  const esp_plan_opts o = resolve_opts(opts);
  if (!(o.r_c > 0)) return fail(ESP_ERR_INVALID_ARG, "a batch needs an explicit cutoff r_c");
  for (int s = 0; s < n_systems; ++s)
    if (N[s] <= 0) return fail(ESP_ERR_INVALID_ARG, "system " + std::to_string(s) + " has no atoms");
  esp_batch_s* b = new esp_batch_s();
  esp_plan_s* p = &b->pool;
  esp_status s = batch_plans(boxes, N, n_systems, tolerance, o, p->hps);
  if (s != ESP_OK) {
    delete b;
    return s;
  }
  s = finish_pool(p, o);
  if (s != ESP_OK) {
    const std::string m = g_error;
    release(p);
    delete b;
    return fail(s, m);
  }
  *out = b;
  return ESP_OK;
}

esp_status esp_batch_query(const esp_box* boxes, const int64_t* N, int n_systems, double tolerance,
                           const esp_plan_opts* opts, esp_plan_params* out) {
  if (!boxes || !N || !out) return fail(ESP_ERR_INVALID_ARG, "boxes, N and out must not be NULL");
  if (n_systems <= 0) return fail(ESP_ERR_INVALID_ARG, "n_systems must be positive");
  const esp_plan_opts o = resolve_opts(opts);
  if (!(o.r_c > 0)) return fail(ESP_ERR_INVALID_ARG, "a batch needs an explicit cutoff r_c");
  std::vector<espe::HostPlan> hps;
  ESP_TRY(batch_plans(boxes, N, n_systems, tolerance, o, hps));
  for (int s = 0; s < n_systems; ++s) out[s] = hps[s].info;
  return ESP_OK;
}

esp_status esp_batch_info(esp_batch_t b, int sys, esp_plan_params* out) {
  esp_plan_s* p = pool_of(b);
  if (!p || !out) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (sys < 0 || sys >= p->nsys) return fail(ESP_ERR_INVALID_ARG, "system index out of range");
  *out = p->hps[sys].info;
  return ESP_OK;
}

esp_status esp_batch_set_charges(esp_batch_t b, const double* q, int where) {
  esp_plan_s* p = pool_of(b);
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL batch");
  return set_charges_any(p, q, true, where);
}

esp_status esp_batch_compute(esp_batch_t b, const double* xyz, double* energies, double* forces,
                             double* potential, int where) {
  esp_plan_s* p = pool_of(b);
  if (!p || !xyz) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (where != ESP_HOST && where != ESP_DEVICE) return fail(ESP_ERR_INVALID_ARG, "bad 'where'");
  if (!p->have_q) return fail(ESP_ERR_NOT_READY, "charges not set");
  DeviceGuard g(p->device);
  const long long N = p->N;
  ESP_CU(cudaMemcpyAsync(p->d_pos, xyz, N * 3 * sizeof(double),
                         where == ESP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, p->st));
  p->have_pos = true;
  if (p->timing) {
    ESP_TRY(run_batch_step(p));
  } else if (p->gexec) {
    ESP_CU(cudaGraphLaunch(p->gexec, p->st));
  } else if (p->direct_runs == 0) {
    ESP_TRY(run_batch_step(p));
    p->direct_runs = 1;
  } else {
    ESP_TRY(capture_batch_step(p));
    ESP_CU(cudaGraphLaunch(p->gexec, p->st));
  }
  p->timed_valid = p->timing;
  const cudaMemcpyKind kind = where == ESP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (forces) ESP_CU(cudaMemcpyAsync(forces, p->d_outF, N * 3 * sizeof(double), kind, p->st));
  if (potential) ESP_CU(cudaMemcpyAsync(potential, p->d_outU, N * sizeof(double), kind, p->st));
  if (energies) ESP_CU(cudaMemcpyAsync(energies, p->d_energy, p->nsys * sizeof(double), kind, p->st));
  if (where == ESP_HOST) {
    ESP_TRY(enqueue_flag_read(p));
    ESP_TRY(wait_stream(p, p->st));
    return flag_result(p);
  }
  return ESP_OK;
}

esp_status esp_batch_synchronize(esp_batch_t b) {
  esp_plan_s* p = pool_of(b);
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL batch");
  return esp_synchronize(p);
}

esp_status esp_batch_set_timing(esp_batch_t b, int enable) {
  esp_plan_s* p = pool_of(b);
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL batch");
  return esp_set_timing(p, enable);
}

esp_status esp_batch_phase_times(esp_batch_t b, float* ms, int n) {
  esp_plan_s* p = pool_of(b);
  if (!p) return fail(ESP_ERR_INVALID_ARG, "NULL batch");
  return esp_phase_times(p, ms, n);
}

esp_status esp_batch_last_virial(esp_batch_t b, double* virial) {
  esp_plan_s* p = pool_of(b);
  if (!p || !virial) return fail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (!p->virial) return fail(ESP_ERR_NOT_READY, "the batch was made without opts.virial");
  if (!p->computed) return fail(ESP_ERR_NOT_READY, "no compute yet");
  DeviceGuard g(p->device);
  ESP_CU(cudaMemcpyAsync(virial, p->d_vout, (size_t)p->nsys * 6 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  return wait_stream(p, p->st);
}

esp_status esp_batch_destroy(esp_batch_t b) {
  if (!b) return ESP_OK;
  release(&b->pool);
  delete b;
  return ESP_OK;
}

}  // extern "C"
