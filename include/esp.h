/*
 * esp.h -- C-ABI of the GB300 ESP electrostatics library (libesp_gb300.so).
 *
 * ESP ("Ewald summation with prolates") computes, for N point charges q_i at
 * r_i in a cubic periodic box of edge L, the quantities of the paper's
 * problem statement (Methods, Eq. task):
 *     u_i = sum'_{j,n} q_j / (4 pi |r_i - r_j - n L|)   (k = 0 mode dropped),
 *     E   = 1/2 sum_i q_i u_i,          F_i = -grad_{r_i} E,
 * through the split 1/(4 pi r) = S(r) + L(r) of Eq. kernelsplitting with the
 * prolate spheroidal wave function (PSWF) of Eq. pswf as splitting kernel:
 *   - the local part (Eq. localpart) is a cell-list pair sum within r_c;
 *   - the spectral part is the five-step method of Eqs. spread ... interp:
 *     spread on an n_f^3 grid with a P-point-per-axis PSWF stencil, R2C FFT,
 *     scaling by the influence function p_k of Eq. pk, C2R FFT, interpolation
 *     of potentials and (analytic-derivative) forces;
 *   - the self term q_i chi(0)/(4 pi r_c) is removed and, for non-neutral
 *     systems, a neutralising background is added.
 * Parameter choice follows Eq. pswfparameters, Table 2 and the aliasing
 * estimate Eq. errorformula. A Gaussian split (Eq. cem) runs on the same
 * machinery for comparison.
 *
 * Units: the kernel is 1/(4 pi r) (the paper's nondimensionalised form);
 * `prefactor` rescales every output (e.g. 138.935458 kJ mol^-1 nm e^-2 for
 * GROMACS units gives prefactor = 4 pi * 138.935458).
 *
 * Conventions
 *  - Positions: N x 3 array-of-structs (x0 y0 z0 x1 ...), any real values;
 *    they are wrapped into [0, L). Forces: N x 3, same layout. Potential: N.
 *    Outputs are in the caller's atom order.
 *  - `where` = ESP_HOST: pointers are host memory; the call copies, computes
 *    and returns after the results are in the caller's buffers.
 *    `where` = ESP_DEVICE: pointers are device memory of the plan's device;
 *    the call enqueues the work on the plan's stream and returns without
 *    waiting (use esp_synchronize). `energy` is then a device double.
 *  - The caller owns every buffer it passes; the library copies inputs and
 *    never keeps a caller pointer after a call returns.
 *  - Errors: every call returns an esp_status; esp_last_error() gives a
 *    thread-local message for the last failing call on this thread. No call
 *    aborts the process. Device-side faults detected by the kernels (a
 *    non-finite coordinate, an out-of-range tile index) set a flag that is
 *    reported by the next synchronising call as ESP_ERR_NONFINITE or
 *    ESP_ERR_INTERNAL.
 *  - Thread safety: a plan is used by one thread at a time. Distinct plans
 *    may be used concurrently from distinct threads.
 */
#ifndef ESP_GB300_H
#define ESP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esp_plan_s* esp_plan_t;

typedef enum {
  ESP_OK = 0,
  ESP_ERR_INVALID_ARG = 1,     /* bad pointer, size, tolerance or option     */
  ESP_ERR_CUTOFF_TOO_LARGE = 2,/* r_c >= L/2 (minimum image would fail)       */
  ESP_ERR_NOT_NEUTRAL = 3,     /* sum q != 0 and allow_background == 0        */
  ESP_ERR_NONFINITE = 4,       /* a position or charge is NaN or infinite     */
  ESP_ERR_OOM = 5,             /* device allocation failed                    */
  ESP_ERR_CUDA = 6,            /* CUDA runtime error                          */
  ESP_ERR_CUFFT = 7,           /* cuFFT error                                 */
  ESP_ERR_TIMEOUT = 8,         /* a device wait exceeded the plan deadline    */
  ESP_ERR_BUSY = 9,            /* admission refused (memory budget)           */
  ESP_ERR_UNSUPPORTED = 10,    /* a size beyond a compiled limit (e.g. P>16)
                                  or an option combination without a kernel
                                  (e.g. a triclinic cell in FP64)             */
  ESP_ERR_INTERNAL = 11,       /* a kernel bounds check failed                */
  ESP_ERR_NOT_READY = 12       /* positions or charges not set yet           */
} esp_status;

enum { ESP_KERNEL_PSWF = 0, ESP_KERNEL_GAUSS = 1 };
enum { ESP_WINDOW_PSWF = 0, ESP_WINDOW_BSPLINE = 1 };
enum { ESP_DIFF_AD = 0, ESP_DIFF_IK = 1 };
enum { ESP_FP32 = 0, ESP_FP64 = 1 };
enum { ESP_HOST = 0, ESP_DEVICE = 1 };

/* Cubic box: L[0] = L[1] = L[2] > 0 (non-cubic boxes are rejected). */
typedef struct { double L[3]; } esp_box;

/* Options. Zero-initialise (or call esp_plan_opts_init) and set what you
 * need; a zero field means "the planner chooses". */
typedef struct {
  double r_c;          /* cutoff of the local part; 0 = cost model           */
  int P;               /* stencil points per axis; 0 = Table 2 (P_esp)       */
  int n_f;             /* grid points per axis; 0 = Eq. pswfparameters rule
                          raised until the aliasing estimate is <= eps/2     */
  double c;            /* PSWF split shape; 0 = solve psi_0^c(1) = tolerance */
  double c1;           /* PSWF SI-kernel shape; 0 = minimise the aliasing
                          estimate over c1/c in [1.1, 1.4]                   */
  double alpha;        /* Gaussian split shape (kernel = GAUSS); 0 = ln(1/eps) */
  int kernel;          /* ESP_KERNEL_PSWF (default) or ESP_KERNEL_GAUSS      */
  int precision;       /* ESP_FP32 (production) or ESP_FP64 (plain mode)     */
  double prefactor;    /* scales u, E, F; 0 = 1                              */
  int device;          /* CUDA device ordinal                                */
  void* stream;        /* cudaStream_t to run on; NULL = plan-owned stream   */
  int allow_background;/* 1 = neutralising background for sum q != 0        */
  int brick_cells;     /* tuning: cells per spread/gather brick edge; 0 auto */
  double timeout_ms;   /* deadline of host waits; 0 = 60000                  */
  int cell_reach;      /* tuning: cell edge ~ r_c / cell_reach (2 or 3; 0 auto) */
  int window;          /* SI kernel: ESP_WINDOW_PSWF (default, Eq. pswf) or
                          ESP_WINDOW_BSPLINE (centred cardinal B-spline of
                          order P, default P 5, n_f = R_default^(1/3) c L /
                          (pi r_c) with Table 2's R_default: the "Default"
                          PME-style comparator of Tables 1 and 2, meant with
                          ESP_KERNEL_GAUSS)                                  */
  int near_variant;    /* tuning: local-part kernel, 1 = one thread per atom,
                          pairs evaluated in the scan, 2 = the same with pairs
                          queued per lane, 3 = one warp per cluster of 8 atoms,
                          every pair from both sides, 4 = the same, every pair
                          once (FP32 only for 3, 4); 0 = default (4 in FP32,
                          1 in FP64)                                          */
  int diff;            /* spectral forces (Methods, step 5): ESP_DIFF_AD
                          (default: analytic derivatives of the SI kernel's
                          polynomials) or ESP_DIFF_IK (the scaled spectrum
                          times 2 pi i k_a / L, three more inverse FFTs, the
                          gradients interpolated with the SI weights; the
                          Nyquist component of the differentiated axis is
                          zero). Potentials and energies are the same.      */
  int virial;          /* 1: every compute also forms the virial W_ab =
                          -dE/d eps_ab (esp_last_virial); needs the default
                          local-part kernel (near_variant 0 or 4 in FP32, 0
                          or 1 in FP64)                                       */
  int reserved[3];
} esp_plan_opts;

/* Parameters a plan chose (esp_plan_info). */
typedef struct {
  double L, r_c, h, c, c1, alpha, prefactor;
  double alias_estimate;   /* relative E_A of Eq. errorformula at (c1, n_f)  */
  double si_fit_error;     /* max |SI-kernel polynomial - psi| (FP64)        */
  double near_fit_error;   /* max error of the local-part polynomials        */
  int64_t N;
  int P, n_f, kernel, precision;
  int n_cells;             /* cell-list cells per axis (edge >= r_c/reach)   */
  int cell_reach;          /* neighbour cells per side in the local part     */
  int near_terms;          /* polynomial terms of the local-part corrections */
  int brick_cells;         /* cells per brick edge                           */
  int tile;                /* shared-memory tile edge in grid points         */
  int si_degree, near_degree;
  size_t device_bytes;     /* device memory held by the plan                 */
  int window;              /* ESP_WINDOW_PSWF or ESP_WINDOW_BSPLINE          */
  int diff;                /* ESP_DIFF_AD or ESP_DIFF_IK                     */
  int virial;              /* 1 when computes form the virial                */
  int triclinic;           /* 1 for a plan of esp_plan_cell (L is then the
                              longest cell vector, n_cells counts cells of
                              fractional coordinates per axis)               */
} esp_plan_params;

/* Fill opts with defaults (all planner choices, FP32, PSWF, device 0). */
void esp_plan_opts_init(esp_plan_opts* opts);

/* Create a plan for N charges in `box` at relative RMS force tolerance
 * `tolerance` (Eq. Deltadef; 1e-15 < tolerance < 0.1). Allocates all device
 * memory and cuFFT plans. opts may be NULL. On success *out owns everything. */
esp_status esp_plan(const esp_box* box, int64_t N, double tolerance,
                    const esp_plan_opts* opts, esp_plan_t* out);

esp_status esp_plan_info(esp_plan_t plan, esp_plan_params* out);

/* Run the planner only (host FP64, no device allocation, no GPU needed) and
 * report the parameters esp_plan would choose; device_bytes is an estimate
 * that excludes the cuFFT work areas. */
esp_status esp_plan_query(const esp_box* box, int64_t N, double tolerance,
                          const esp_plan_opts* opts, esp_plan_params* out);

/* Triclinic (or orthorhombic) periodic cell: the cell vectors a, b, c in the
 * reduced orientation a = (ax, 0, 0), b = (bx, by, 0), c = (cx, cy, cz) with
 * ax, by, cz > 0 (the truncated-octahedral and rhombic-dodecahedral boxes of
 * Table 1 take this form). Images of r are r + n_a a + n_b b + n_c c. */
typedef struct { double a[3], b[3], c[3]; } esp_cell;

/* Plan for N charges in a triclinic cell (Eq. task on the lattice of the
 * cell). The n_f^3 grid and the cell list are laid over fractional
 * coordinates s = H^-1 r (H = [a b c]); spread and interpolation use the SI
 * kernel per fractional axis, the influence function is Eq. pk with
 * |xi(k)| = 2 pi |H^-T k| and Phi in grid units, forces are
 * -q H^-T grad_s u~ plus the local part over every image within r_c.
 * n_f, c, c1 and P follow the cubic rules on the longest cell vector.
 * Errors: ESP_ERR_INVALID_ARG for a cell not in the reduced orientation,
 * ESP_ERR_CUTOFF_TOO_LARGE unless r_c is below half the smallest distance
 * between opposite faces, ESP_ERR_UNSUPPORTED for ESP_FP64, ESP_DIFF_IK, the
 * virial, a local-part variant other than 0/4, or n_f > 384. The plan is used
 * like any other (esp_set_*, esp_compute, esp_step, esp_destroy). */
esp_status esp_plan_cell(const esp_cell* cell, int64_t N, double tolerance,
                         const esp_plan_opts* opts, esp_plan_t* out);
esp_status esp_plan_query_cell(const esp_cell* cell, int64_t N, double tolerance,
                               const esp_plan_opts* opts, esp_plan_params* out);

/* The influence function p_k (Eq. pk) the plan of (box or cell, N,
 * tolerance, opts) would apply, in FP64 from the host planner (no GPU
 * needed): out[(kz * n_f + ky) * (n_f/2 + 1) + kx] for the half spectrum of
 * the forward transform sum_l b_l exp(-2 pi i k.l / n_f) of the grid
 * b[z][y][x] (x fastest), index i standing for k = i below n_f/2 and
 * i - n_f from n_f/2 on. Where a component is -n_f/2 the value is the
 * average over k and the representative of -k (equal for a cube). Pass
 * exactly one of box and cell. *len: in, the capacity of out; out, the
 * number of entries n_f^2 (n_f/2 + 1). out may be NULL to query *len only.
 * ESP_ERR_INVALID_ARG if the capacity is too small. */
esp_status esp_influence_query(const esp_box* box, const esp_cell* cell, int64_t N, double tolerance,
                               const esp_plan_opts* opts, double* out, int64_t* len);

/* Charges q[N] (double or float). Must be called before the first compute
 * and whenever charges change. */
esp_status esp_set_charges(esp_plan_t plan, const double* q, int where);
esp_status esp_set_charges_f32(esp_plan_t plan, const float* q, int where);

/* Positions xyz[N*3]: ingest (wrap, fixed-point conversion, finite check)
 * and bin sort (counting sort by cell) -- steps A0-A1 of the pipeline. */
esp_status esp_set_positions(esp_plan_t plan, const double* xyz, int where);
esp_status esp_set_positions_f32(esp_plan_t plan, const float* xyz, int where);

/* Exclusions: the listed pairs (caller indices; pair k is pairs[2k],
 * pairs[2k+1]) do not interact in the computes that follow: their direct
 * interaction q_i q_j / (4 pi r) (times the prefactor) is removed from the
 * energy, the potentials and the forces, while their other periodic images
 * still count (the bonded pairs of molecules in MD). The pair vector is the
 * image nearest in wrapped fractional coordinates, the minimum image for
 * pairs closer than half the smallest cell height. n_pairs = 0 clears the
 * list. pairs is a host array, copied; the call first waits for the plan's
 * stream. ESP_ERR_INVALID_ARG for an index outside [0, N), i = j, or a pair
 * listed more than once (in either order); ESP_ERR_UNSUPPORTED on a plan
 * made with opts.virial. */
esp_status esp_set_exclusions(esp_plan_t plan, const int32_t* pairs, int64_t n_pairs);

/* Spread, R2C FFT, fused influence scale + spectral energy, C2R FFT, gather,
 * local part, corrections and compensated FP64 energy. Any of energy,
 * forces, potential may be NULL; with forces and potential both NULL only
 * the energy is computed (the C2R FFT and the gather are skipped, and the
 * gathered spectral energy of esp_last_spectral_energy reads 0). */
esp_status esp_compute(esp_plan_t plan, double* energy, double* forces,
                       double* potential, int where);
esp_status esp_compute_f32(esp_plan_t plan, double* energy, float* forces,
                           float* potential, int where);

/* Wait (bounded by the plan deadline) for the plan's queued work; reports a
 * device-side error flag raised since the last call. */
esp_status esp_synchronize(esp_plan_t plan);

/* Per-phase device times (ms) of the last compute when timing is enabled:
 * [0] ingest+sort (with the local part's cluster lists), [1] spread,
 * [2] r2c, [3] scale, [4] c2r, [5] gather, [6] near (the pair kernel),
 * [7] finalize, [8] whole compute. enable = 1 records CUDA events
 * around the phases (the local part still overlaps the spectral part, so the
 * spectral phases include contention); enable = 2 also runs the local part on
 * the main stream so that every phase is timed alone; 0 turns timing off.
 * esp_phase_times waits for the last compute and returns ESP_ERR_NOT_READY
 * when timing is off. */
esp_status esp_set_timing(esp_plan_t plan, int enable);
esp_status esp_phase_times(esp_plan_t plan, float* ms, int n);

/* Spectral energy 1/2 sum_k p_k |bh_k|^2 of the last compute (host double). */
esp_status esp_last_spectral_energy(esp_plan_t plan, double* e_fourier, double* e_gather);

/* One step: esp_set_positions(xyz) followed by esp_compute, in one call.
 * With host buffers the call copies the positions in (positions in
 * page-locked host memory mapped into the device's address space, e.g. from
 * cudaHostAlloc, are read in place by the ingest kernel instead), computes,
 * copies the results out and waits once; after its first run the sort and the compute
 * replay as one captured CUDA graph (per position source and output
 * pointers, as for esp_compute). Errors as for the two calls (a non-finite
 * position is reported as ESP_ERR_NONFINITE by this call with host
 * buffers, by the next synchronising call otherwise). */
esp_status esp_step(esp_plan_t plan, const double* xyz, double* energy, double* forces,
                    double* potential, int where);

/* Virial of the last compute of a plan made with opts.virial = 1: W_ab =
 * -dE/d eps_ab under the homogeneous deformation r -> (1 + eps) r of atoms
 * and box (the grid deforms with the box), in energy units (times the
 * prefactor); pressure = (kinetic term + trace W) / (3 V). Spectral part
 * sum_k 1/2 |bh_k|^2 [p_k delta_ab + p'_k k_a k_b / |k|^2] with p'_k the
 * derivative of Eq. pk's Shat with respect to ln|k|, local part the pair
 * terms of Eq. localpart, and the neutralising background's energy on the
 * diagonal. virial[6] receives (xx, yy, zz, xy, xz, yz) on the host; the
 * call waits (bounded) for the compute. ESP_ERR_NOT_READY without
 * opts.virial or before the first compute. */
esp_status esp_last_virial(esp_plan_t plan, double* virial);

esp_status esp_destroy(esp_plan_t plan);

/* Autotuner. The paper has no counterpart (its kernels are CPU code): the
 * shapes this implementation is free to choose -- cell-list reach (cell edge
 * r_c/2 or r_c/3), local-part kernel (near_variant 3: every pair from both
 * sides; 4: every pair once) and the brick edge of spread/gather (the
 * planner's choice and one cell either side) -- are timed on the caller's own
 * system: for each candidate a plan is made, charges q[N] and positions
 * xyz[N*3] (FP64, host or device per `where`) are set, one warm-up compute
 * runs, then `reps` timed computes (0 = 5); the median whole-compute time
 * decides. Options fixed in `opts` (non-zero) are kept. *out receives opts
 * with the winning shapes (and the planner's r_c); *best_ms its time. Results
 * are cached per process by (N, L, tolerance, r_c, precision, kernel,
 * device), so a second call returns at once. Allocates and frees a plan per
 * candidate; synchronous. */
esp_status esp_autotune(const esp_box* box, int64_t N, double tolerance, const esp_plan_opts* opts,
                        const double* xyz, const double* q, int where, int reps,
                        esp_plan_opts* out, double* best_ms);

/* ------------------------------------------------------------------ batches
 * Many independent systems (each its own cubic box, charges and positions)
 * solved together in one step: the same pipeline as esp_compute runs once
 * over all systems, with per-system cell lists, grids and influence
 * functions, one batched cuFFT plan per grid size, and after the first call
 * the whole step replayed from a CUDA graph. The paper treats one system at
 * a time (Methods); the batch is the data-parallel form of that method for
 * ensembles of small boxes, where one system cannot fill the GPU.
 *
 * Planning: every system is planned as by esp_plan with the same tolerance
 * and options; r_c must be given (opts->r_c > 0) and be below L/2 of every
 * box. The SI-kernel shape c1 is made common (the value most systems chose
 * when planned alone) and each grid is raised to the next size of a ladder
 * of FFT-friendly sizes >= 12% apart, so systems of similar size share a
 * batched FFT; both only lower each system's aliasing estimate.
 *
 * Layout: the systems' atoms are concatenated in system order. Charges q
 * (sum N[s]), positions xyz (sum N[s] x 3), forces (sum N[s] x 3) and
 * potential (sum N[s]) use that order; energies has one entry per system.
 * All FP64. `where` as for plans; outputs may be NULL. */
typedef struct esp_batch_s* esp_batch_t;

esp_status esp_batch_create(const esp_box* boxes, const int64_t* N, int n_systems,
                            double tolerance, const esp_plan_opts* opts, esp_batch_t* out);
/* Planner only (host, no GPU needed): the parameters esp_batch_create
 * would choose, one esp_plan_params per system in out[n_systems]
 * (device_bytes is 0). */
esp_status esp_batch_query(const esp_box* boxes, const int64_t* N, int n_systems,
                           double tolerance, const esp_plan_opts* opts, esp_plan_params* out);
/* Parameters chosen for system `sys` (0-based). */
esp_status esp_batch_info(esp_batch_t batch, int sys, esp_plan_params* out);
/* Charges of all systems; rejects a non-neutral system when
 * allow_background is 0. */
esp_status esp_batch_set_charges(esp_batch_t batch, const double* q, int where);
/* One step on positions xyz: ingest and bin sort, local and spectral parts,
 * corrections, per-system compensated energies. With `where` = ESP_HOST it
 * returns after the outputs are copied; with ESP_DEVICE it only enqueues. */
esp_status esp_batch_compute(esp_batch_t batch, const double* xyz, double* energies,
                             double* forces, double* potential, int where);
esp_status esp_batch_synchronize(esp_batch_t batch);
/* Phase timing as esp_set_timing / esp_phase_times; while timing is on the
 * step runs as direct launches instead of the graph. */
esp_status esp_batch_set_timing(esp_batch_t batch, int enable);
esp_status esp_batch_phase_times(esp_batch_t batch, float* ms, int n);
/* Virials of the last batch compute (opts.virial = 1): virial[6 * s + c],
 * c = xx, yy, zz, xy, xz, yz, for every system s (as esp_last_virial). */
esp_status esp_batch_last_virial(esp_batch_t batch, double* virial);
esp_status esp_batch_destroy(esp_batch_t batch);

/* ------------------------------------------------------------------ server
 * Request server on one device. The paper treats one solve at a time; the
 * server is the serving form of the same solve: systems are registered once
 * (box, N, charges, copied), and each request (system id, tolerance,
 * positions N x 3 FP64, copied at submit) is answered with the energy, forces
 * and potential of esp_compute for that system.
 *  - Plans: one per (system, tolerance), created on the first request and
 *    kept resident (sorted bins, grids, FFT plans) for the next ones. A plan
 *    that would exceed memory_budget first evicts idle plans, least recently
 *    used first; a request whose plan cannot fit waits until running requests
 *    finish, and fails with ESP_ERR_BUSY if it could never fit.
 *  - Continuous batching: a worker thread keeps up to max_inflight requests
 *    on the device at once, each on its plan's own streams (copies and
 *    kernels asynchronous through pinned host buffers); a request submitted
 *    while others run starts as soon as a slot and its plan are free. Two
 *    requests for the same plan run one after the other.
 *  - Results equal those of esp_plan + esp_compute on the same inputs up to
 *    FP32 rounding (atomic summation order).
 * The server is internally synchronized: submit, poll and wait may be called
 * from any thread. Latency = completion - submission, in ms. */
typedef struct esp_server_s* esp_server_t;

typedef struct {
  size_t memory_budget;  /* device bytes the server's plans may hold; 0 = 80% of free */
  int device;            /* CUDA device ordinal                                        */
  int max_inflight;      /* requests on the device at once; 0 = 8                      */
  double r_c;            /* cutoff of every plan (required, > 0)                        */
  int precision;         /* ESP_FP32 (default) or ESP_FP64                             */
  int kernel;            /* ESP_KERNEL_PSWF (default) or ESP_KERNEL_GAUSS              */
  double timeout_ms;     /* deadline of a running request and of waits; 0 = 60000    */
  int reserved[8];
} esp_server_opts;

typedef struct {
  int64_t completed, failed, pending, running;
  double atoms_done;          /* atoms of completed requests                          */
  int64_t plans_resident, plans_created, evictions;
  size_t device_bytes;        /* bytes held by resident plans                         */
  size_t memory_budget;
  double latency_p50_ms, latency_p99_ms, latency_max_ms;
  double wall_ms;             /* first submission to last completion                  */
  /* Overlap on the device, from events recorded on each request's stream
   * before its first copy and after its last: every completed request's
   * device interval [start, done]. */
  int64_t peak_inflight;      /* most requests admitted to the device at once         */
  int64_t peak_concurrent;    /* most device intervals that overlap at one instant    */
  double overlap_ms;          /* device time with two or more requests in flight      */
} esp_server_counters;

void esp_server_opts_init(esp_server_opts* opts);
esp_status esp_server_create(const esp_server_opts* opts, esp_server_t* out);
/* Register a system; q[N] host FP64 (copied). *id is the handle of requests. */
esp_status esp_server_add_system(esp_server_t server, const esp_box* box, int64_t N,
                                 const double* q, int* id);
/* Queue a request; xyz[3N] host FP64 (copied before return). */
esp_status esp_server_submit(esp_server_t server, int id, double tolerance, const double* xyz,
                             int64_t* ticket);
/* *done = 1 once the request has finished (successfully or not). */
esp_status esp_server_poll(esp_server_t server, int64_t ticket, int* done);
/* Wait (at most timeout_ms; 0 = the server deadline) and copy the results to
 * host buffers (any may be NULL); the ticket is released unless the wait or
 * the request timed out. Returns the request's status. */
esp_status esp_server_wait(esp_server_t server, int64_t ticket, double timeout_ms, double* energy,
                           double* forces, double* potential, double* latency_ms);
esp_status esp_server_stats(esp_server_t server, esp_server_counters* out);
/* Clear the completion counters and latencies (resident plans stay). */
esp_status esp_server_reset_stats(esp_server_t server);
/* Stop the worker, wait for running requests, free every plan. */
esp_status esp_server_destroy(esp_server_t server);

/* Local part without device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (code running
 * while a framework's caching allocator owns the device heap, inside regions
 * where an allocation would synchronise the device, or under a fixed device
 * memory budget).
 *
 * For N charges q[N] at xyz[N*3] (both FP64, in device memory of
 * opts->device) it computes what esp_compute returns minus the spectral part:
 * the direct pair sum of the split within r_c, the self term and, when
 * sum q != 0 and allow_background is set, the neutralising background:
 *   potential[i] = u^l_i - q_i chi(0)/(4 pi r_c) + background,
 *   forces[i]    = F^l_i,
 *   *energy      = 1/2 sum q_i u^l_i + E_self + E_bg,
 * all FP64 in device memory (any of them may be NULL). opts selects the
 * split, precision, cutoff r_c (required here: 0 picks the planner's cost
 * model) and stream (NULL = the legacy default stream); the grid options are
 * ignored.
 *
 * Working memory comes from one 6 MiB array in the library's device image,
 * which every GPU that loads the library holds until the process exits:
 * about 65k atoms in FP32 mode and 32k in FP64 mode fit; larger systems are
 * rejected with ESP_ERR_UNSUPPORTED before any device work. xyz, q and every
 * non-NULL output must be device (or managed) memory of opts->device, else
 * ESP_ERR_INVALID_ARG before any launch. The first call on a device looks up
 * the array's address with that device current; make that first call before
 * any stream capture. The call reads the charges back to the host (a
 * synchronising copy), enqueues its kernels on the stream and waits for them
 * to read their error flag: a NaN or infinite position gives
 * ESP_ERR_NONFINITE (the outputs are then not valid), a failed bounds check
 * ESP_ERR_INTERNAL. Every call shares the array, and each call clears what it
 * reads before writing it; calls whose device work overlaps (on different
 * streams or host threads) race on the array and must be serialised by the
 * caller. */
esp_status esp_local_part_static(const esp_box* box, int64_t N, double tolerance,
                                 const esp_plan_opts* opts, const double* xyz,
                                 const double* q, double* energy, double* forces,
                                 double* potential);

/* Thread-local message of the last failing call ("" if none). */
const char* esp_last_error(void);

/* Library build identification (compile-time arch list and version). */
const char* esp_version(void);

/* ------------------------------------------------------------ MD loop
 * A workload around the solve: velocity Verlet for flexible SPC/E-shaped
 * water, the plan's atoms being consecutive (O, H, H) molecules. Forces:
 * the plan's ESP solve with the three intramolecular pairs of every molecule
 * excluded (esp_md_create sets the plan's exclusion list), harmonic O-H
 * bonds and H-O-H angle, O-O Lennard-Jones within a cutoff (shifted to zero
 * there). Units nm, ps, amu, kJ/mol: make the plan with
 * opts.prefactor = 4 pi 138.935458 so that its energy is in kJ/mol for
 * charges in e. Cubic plans, charges set before esp_md_create. */
typedef struct esp_md_s* esp_md_t;
typedef struct {
  double dt;                 /* time step, ps                                    */
  double k_bond, r0;         /* bonds k (r - r0)^2 / 2: kJ mol^-1 nm^-2, nm       */
  double k_angle, theta0;    /* angle k (theta - theta0)^2 / 2: kJ mol^-1 rad^-2, rad */
  double lj_sigma, lj_epsilon, lj_cutoff; /* O-O: nm, kJ/mol, nm (< L/2)      */
  double mass_O, mass_H;     /* amu                                              */
  int reserved[8];
} esp_md_params;

/* Defaults: dt 0.0005 ps, k_b 3.45e5, r0 0.1, k_theta 383, theta0 109.47 deg,
 * SPC/E sigma 0.316557 nm and epsilon 0.650194 kJ/mol, cutoff 1.0 nm,
 * masses 15.9994 and 1.008. */
void esp_md_params_init(esp_md_params* params);

/* Bind an MD state to `plan` (which it then drives; destroy the MD state
 * before the plan): positions xyz and velocities vel (host, N x 3, nm and
 * nm/ps) are copied to the device. ESP_ERR_INVALID_ARG for N not a multiple
 * of 3 or bad parameters, ESP_ERR_UNSUPPORTED for a triclinic plan. */
esp_status esp_md_create(esp_plan_t plan, const esp_md_params* params, const double* xyz, const double* vel,
                         esp_md_t* out);

/* n_steps velocity-Verlet steps. energies (host, nullable) receives
 * (n_steps + 1) rows (Coulomb, bonded, Lennard-Jones, kinetic) in kJ/mol:
 * the state before the first step, then after every step. */
esp_status esp_md_run(esp_md_t md, int n_steps, double* energies);

/* Current positions and velocities (host, N x 3; either may be NULL). */
esp_status esp_md_state(esp_md_t md, double* xyz, double* vel);
/* Free the MD state and clear the plan's exclusion list (the intramolecular
 * pairs esp_md_create set), so later computes on the plan count every pair. */
esp_status esp_md_destroy(esp_md_t md);

#ifdef __cplusplus
}
#endif
#endif /* ESP_GB300_H */
