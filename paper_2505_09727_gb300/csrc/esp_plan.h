// Host planning of one system: parameter choice (paper's rules), polynomial
// tables and influence tables. Shared by the single-system and batch paths.
#pragma once
#include <string>
#include <vector>

#include "../../include/esp.h"
#include "esp_device.cuh"
#include "esp_math.h"

namespace espe {

struct HostPlan {
  esp_plan_params info{};
  double tol = 0;
  double self_unit = 0;        // chi(0) / (4 pi r_c)
  double m2 = 0;               // int_0^1 x^2 chi
  espk::SysDesc desc{};        // atom0/cell0/grid0/spec0/tab0 are zero here
  espk::SICoef<float> si32{};
  espk::SICoef<double> si64{};
  espk::NearCoef<float> nc32{};
  espk::NearCoef<double> nc64{};
  std::vector<double> G, W;    // influence tables: G[|k|^2], W[|k_a|]
  std::vector<double> H;       // virial table: d G / d ln|k| at |k|^2
  long long n_keys = 0;        // n_c^3 * kSub: length of the cell-list count array
  long long grid_elems = 0;    // n_f^3
  long long spec_elems = 0;    // n_f^2 (n_f/2 + 1)
  int n_bricks = 0;            // nb^3
  int near_nc = 0;             // polynomial terms used by the local part
  bool near_queued = false;    // local-part variant (queued pairs)
  bool near_clusters = false;  // local-part variant (one warp per i-cluster, FP32)
  bool near_half = false;      // ... with each pair evaluated once
};

// Fill `hp` for a cubic box of edge L with N atoms. Returns ESP_OK or an
// error with a message in `msg`.
esp_status make_host_plan(double L, long long N, double tol, const esp_plan_opts& opts, HostPlan& hp,
                          std::string& msg);

// The same for a triclinic cell: rows a, b, c of cell[9] with a = (ax,0,0),
// b = (bx,by,0), c = (cx,cy,cz). FP32 only, AD forces, no virial.
esp_status make_host_plan_cell(const double cell[9], long long N, double tol, const esp_plan_opts& opts,
                               HostPlan& hp, std::string& msg);

// Message reported by esp_last_error() for the calling thread.
void set_last_error(const std::string& msg);

// Constants that depend on the charges (self energy, background).
void charge_constants(const HostPlan& hp, double Q, double Q2, double* e_self, double* e_bg,
                      double* bg_shift);

}  // namespace espe
