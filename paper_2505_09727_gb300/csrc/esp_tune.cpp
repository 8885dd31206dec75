// Autotuner (include/esp.h, esp_autotune): times candidate cell-list, brick
// and local-part shapes of one system on its own positions and keeps the
// fastest. Host code over the public C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/esp.h"
#include "esp_engine.h"

namespace {

struct TuneKey {
  long long N;
  double L, tol, r_c;
  int precision, kernel, device;
  bool operator<(const TuneKey& o) const {
    return std::tie(N, L, tol, r_c, precision, kernel, device) <
           std::tie(o.N, o.L, o.tol, o.r_c, o.precision, o.kernel, o.device);
  }
};

struct TuneResult {
  int cell_reach, near_variant, brick_cells;
  double ms;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune_cache;

esp_status tfail(esp_status s, const std::string& m) {
  espe::set_last_error(m);
  return s;
}

// Median whole-compute time of `reps` computes with options o (ms), or a
// negative value when the candidate cannot be planned or run.
double time_candidate(const esp_box* box, int64_t N, double tol, const esp_plan_opts& o, const double* xyz,
                      const double* q, int where, int reps, esp_plan_params* info, std::string* why) {
  esp_plan_t p = nullptr;
  if (esp_plan(box, N, tol, &o, &p) != ESP_OK) {
    *why = esp_last_error();
    return -1.0;
  }
  double best = -1.0;
  esp_status st = esp_plan_info(p, info);
  if (st == ESP_OK) st = esp_set_charges(p, q, where);
  if (st == ESP_OK) st = esp_set_positions(p, xyz, where);
  if (st == ESP_OK) st = esp_compute(p, nullptr, nullptr, nullptr, ESP_HOST);
  if (st == ESP_OK) st = esp_set_timing(p, 1);
  std::vector<double> t;
  for (int r = 0; st == ESP_OK && r < reps; ++r) {
    float ms[9];
    st = esp_compute(p, nullptr, nullptr, nullptr, ESP_HOST);
    if (st == ESP_OK) st = esp_phase_times(p, ms, 9);
    if (st == ESP_OK) t.push_back(ms[8]);
  }
  if (st == ESP_OK && (int)t.size() == reps) {
    std::sort(t.begin(), t.end());
    best = t[t.size() / 2];
  } else {
    *why = esp_last_error();
  }
  esp_destroy(p);
  return best;
}

}  // namespace

extern "C" esp_status esp_autotune(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                                   const double* xyz, const double* q, int where, int reps, esp_plan_opts* out,
                                   double* best_ms) {
  if (!box || !xyz || !q || !out) return tfail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (N <= 0) return tfail(ESP_ERR_INVALID_ARG, "autotuning needs atoms");
  if (where != ESP_HOST && where != ESP_DEVICE) return tfail(ESP_ERR_INVALID_ARG, "bad 'where'");
  esp_plan_opts base;
  if (opts) base = *opts;
  else esp_plan_opts_init(&base);
  if (reps <= 0) reps = 5;
  // the planner's own choice first: it fixes r_c and the default shapes
  esp_plan_params info0;
  esp_status st = esp_plan_query(box, N, tolerance, &base, &info0);
  if (st != ESP_OK) return st;
  base.r_c = info0.r_c;
  const TuneKey key{N, box->L[0], tolerance, base.r_c, base.precision, base.kernel, base.device};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out = base;
      out->cell_reach = it->second.cell_reach;
      out->near_variant = it->second.near_variant;
      out->brick_cells = it->second.brick_cells;
      if (best_ms) *best_ms = it->second.ms;
      return ESP_OK;
    }
  }
  // candidates: cell reach x local-part kernel x brick edge around the
  // planner's choice (options the caller fixed are kept)
  std::vector<int> reaches = base.cell_reach > 0 ? std::vector<int>{base.cell_reach} : std::vector<int>{2, 3};
  std::vector<int> variants;
  if (base.near_variant > 0) variants = {base.near_variant};
  else if (base.precision == ESP_FP32) variants = {3, 4};
  else variants = {1};
  TuneResult best{0, 0, 0, -1.0};
  std::string why;
  for (int reach : reaches) {
    for (int var : variants) {
      esp_plan_opts o = base;
      o.cell_reach = reach;
      o.near_variant = var;
      esp_plan_params info;
      std::vector<int> bricks;
      if (base.brick_cells > 0) {
        bricks = {base.brick_cells};
      } else {
        esp_plan_opts probe = o;
        if (esp_plan_query(box, N, tolerance, &probe, &info) != ESP_OK) continue;
        bricks = {info.brick_cells};
        for (int b : {info.brick_cells - 1, info.brick_cells + 1})
          if (b >= 1 && b <= 8) bricks.push_back(b);
      }
      for (int b : bricks) {
        o.brick_cells = b;
        const double ms = time_candidate(box, N, tolerance, o, xyz, q, where, reps, &info, &why);
        if (ms > 0 && (best.ms < 0 || ms < best.ms)) best = TuneResult{reach, var, b, ms};
      }
    }
  }
  if (best.ms < 0)
    return tfail(ESP_ERR_INTERNAL, "no candidate configuration could be planned and run (" + why + ")");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  *out = base;
  out->cell_reach = best.cell_reach;
  out->near_variant = best.near_variant;
  out->brick_cells = best.brick_cells;
  if (best_ms) *best_ms = best.ms;
  return ESP_OK;
}
