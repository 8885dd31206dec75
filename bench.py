"""Benchmark: atoms/s of the ESP long-range electrostatics solve on one GB300.

Workload (default): SPC/E-shaped water, 1e5 molecules = 3e5 atoms, L = 14.413
nm (33.4 molecules/nm^3), r_c = 1.0 nm, tolerance 1e-4 relative RMS force
error, FP32 production path with FP64 corrections and energy.

One step = the whole hot path, one esp_step call: ingest + bin sort, then
spread, R2C FFT, fused scale + spectral energy, C2R FFT, gather, local part,
corrections and energy. `value` times steps with inputs and outputs resident
in device memory; `e2e` times the same call with pinned host buffers
(host->device positions, device->host energy, forces, potential).

The inputs (3.6 MB) fit in L2, so L2 is flushed (a 512 MB write) between timed
steps, outside the timed events.

`--impl reference` times the FP64 CPU oracle instead (see --help).
Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of the
workload (the single-system solve has no data-parallel split without an
exchange step), no collective on the data path; value = total atoms / max
rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atoms/s long-range forces at 1e-4 err: batched+served vs plain; p50/p99 ms"
UNIT = "atoms/s"
WORKLOAD = dict(workload="spce_water_1e5_molecules", molecules=100_000, atoms=300_000,
                density_per_nm3=33.4, r_c_nm=1.0, tolerance=1e-4, seed=2505)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--molecules", type=int, default=WORKLOAD["molecules"])
    ap.add_argument("--tolerance", type=float, default=WORKLOAD["tolerance"],
                    help="relative RMS force tolerance of the main line (profiling other stencil widths)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64, Gaussian, batched and served comparison lines")
    ap.add_argument("--served-full", action="store_true",
                    help="served line on the full 256-system, 1e4-request stream (minutes of setup)")
    return ap.parse_args()


def dist_env():
    from paper_2505_09727_gb300 import replicas
    return replicas.dist_env()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"esp_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# flops of one unordered pair evaluation: difference 3, r^2 5, rsqrt 1,
# polynomial argument 2, two 9-term Horner polynomials 2 x 18, potentials
# 2 + 2, r^-3 terms 4, forces on both atoms 2 x (1 + 6)
NEAR_FLOPS_PER_PAIR = 71
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "near_cluster_water3e5_traffic.md")
NEAR_SOURCE = os.path.join(ROOT, "paper_2505_09727_gb300", "csrc", "esp_near_cluster.cuh")


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of the local-part kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    import hashlib
    if kernel != "near" or not os.path.exists(TRAFFIC_PROFILE):
        return None
    fields = {}
    for line in open(TRAFFIC_PROFILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            fields[k.strip().strip("-* `")] = v.strip().strip("`")
    with open(NEAR_SOURCE, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    if fields.get("source_sha256") != digest:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def roofline(phases: dict, info: dict, n_atoms: int, L: float, clocks, n_steps: int):
    """Roofline of the dominant kernel (largest average serialised duration).

    Algorithmic work per launch:
      near    FP32 ALU: unique pairs within r_c (N * 4/3 pi r_c^3 rho / 2) x
              NEAR_FLOPS_PER_PAIR, against 152 SMs x 128 FP32 lanes x 2 flop x
              the median SM clock seen during the run
      spread  HBM: 16 B/atom (sorted atoms) + 4 B per grid point (grid write)
      gather  HBM: 16 B/atom in + 16 B/atom out + 4 B per grid point
      scale   HBM: 16 B per complex mode (read + write)
    """
    rho = n_atoms / L ** 3
    pairs = 0.5 * n_atoms * 4.0 / 3.0 * math.pi * info["r_c"] ** 3 * rho
    n_f = info["n_f"]
    grid = n_f ** 3
    modes = n_f * n_f * (n_f // 2 + 1)
    algo = {
        "near": ("alu", pairs * NEAR_FLOPS_PER_PAIR, "TFLOP/s"),
        "spread": ("hbm", 16.0 * n_atoms + 4.0 * grid, "GB/s"),
        "gather": ("hbm", 32.0 * n_atoms + 4.0 * grid, "GB/s"),
        "scale": ("hbm", 16.0 * modes, "GB/s"),
    }
    kernel = max(algo, key=lambda k: phases.get(k, 0.0))
    bound, work, unit = algo[kernel]
    t = phases[kernel] * 1e-3
    peaks, source = measured_peaks()
    if bound == "alu":
        mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1492.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        achieved = work / t / 1e12
        peak_note = (f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz (median SM clock in the "
                     f"run); no measured FP32 peak in MEASURED_PEAKS.json")
    else:
        peak = peaks["hbm_gbs"]
        achieved = work / t / 1e9
        peak_note = f"{source} HBM copy bandwidth"
    return {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": profiled_traffic(kernel), "peak_source": peak_note,
            "algorithmic_per_launch": work, "avg_launch_ms": phases[kernel]}


def phase_rooflines(phases: dict, info: dict, n_atoms: int, L: float, clocks) -> dict:
    """Every phase (serialised CUDA-event time) against each resource: its
    algorithmic DRAM bytes over the measured HBM copy bandwidth and, for the
    arithmetic phases, its FP32 flops over the derived FP32 peak.

    Bytes per step: sort 24 B/atom FP64 positions in + 36 B/atom sorted
    records, pair records and permutation out; spread 16 B/atom + 4 B per
    grid point; R2C and C2R 4 B per grid point + 8 B per mode; scale 16 B per
    mode; gather 32 B/atom + 4 B per grid point; local part 32 B/atom;
    finalize 52 B/atom in + 32 B/atom out. Flops per atom: spread 2 P^3
    (weighted adds) + 6 P (SI_DEGREE + 1) (1-D weights); gather 8 P^3 + 12 P
    (SI_DEGREE + 1) (potential, three derivatives); local part as in
    roofline()."""
    rho = n_atoms / L ** 3
    pairs = 0.5 * n_atoms * 4.0 / 3.0 * math.pi * info["r_c"] ** 3 * rho
    n_f, P, deg = info["n_f"], info["P"], info.get("si_degree", 9)
    grid = n_f ** 3
    modes = n_f * n_f * (n_f // 2 + 1)
    peaks, source = measured_peaks()
    hbm = peaks["hbm_gbs"]
    mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1492.0)
    fp32 = 152 * 128 * 2 * mhz * 1e6 / 1e12
    work = {
        "ingest_sort": (60.0 * n_atoms, 0.0),
        "spread": (16.0 * n_atoms + 4.0 * grid, n_atoms * (2.0 * P ** 3 + 6.0 * P * (deg + 1))),
        "fft_r2c": (4.0 * grid + 8.0 * modes, 0.0),
        "scale": (16.0 * modes, 0.0),
        "fft_c2r": (4.0 * grid + 8.0 * modes, 0.0),
        "gather": (32.0 * n_atoms + 4.0 * grid, n_atoms * (8.0 * P ** 3 + 12.0 * P * (deg + 1))),
        "near": (32.0 * n_atoms, pairs * NEAR_FLOPS_PER_PAIR),
        "finalize": (84.0 * n_atoms, 0.0),
    }
    out = {"hbm_peak_gbs": hbm, "hbm_peak_source": source, "fp32_peak_tflops": fp32}
    for k, (b, f) in work.items():
        t = phases.get(k, 0.0) * 1e-3
        if t <= 0:
            continue
        row = {"ms": round(phases[k], 5), "hbm_gbs": round(b / t / 1e9, 2), "hbm_frac": round(b / t / 1e9 / hbm, 5)}
        if f:
            row["fp32_tflops"] = round(f / t / 1e12, 3)
            row["fp32_frac"] = round(f / t / 1e12 / fp32, 5)
        out[k] = row
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, world, rank, local):
    import torch
    from paper_2505_09727_gb300 import esp, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.spce_water(args.molecules, seed=WORKLOAD["seed"])
    N, L = s.n, s.L
    # one explicit stream for the plan, the tensors and the timing events
    # (torch's default stream is the legacy NULL stream, which the plan does
    # not adopt)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h = esp.esp_plan(L, N, args.tolerance, r_c=WORKLOAD["r_c_nm"], device=local,
                     stream=stream.cuda_stream)
    info = esp.esp_plan_info(h)
    q = torch.tensor(s.q, device=dev)
    x = torch.tensor(s.pos, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    esp.esp_set_charges(h, q)

    def step():
        esp.esp_step(h, x, e, f, u)               # positions in, compute (one graph after the first run)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    from paper_2505_09727_gb300 import replicas

    def barrier():
        replicas.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)

    # second timed region: phases serialised and bracketed by CUDA events on
    # the stream each kernel runs on (per-kernel durations for the roofline)
    esp.esp_set_timing(h, 2)
    phase_acc = {k: 0.0 for k in esp.PHASES}
    for i in range(args.steps):
        flush.zero_()
        step()
        for k, v in esp.esp_phase_times(h).items():
            phase_acc[k] += v
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    esp.esp_set_timing(h, 0)

    # end to end through the C-ABI with pinned host buffers
    xh = torch.tensor(s.pos).pin_memory()
    fh = torch.zeros((N, 3), dtype=torch.float64).pin_memory()
    uh = torch.zeros(N, dtype=torch.float64).pin_memory()
    eh = np.zeros(1)
    for _ in range(3):
        esp.esp_step(h, xh, eh, fh, uh, esp.ESP_HOST)
    torch.cuda.synchronize(dev)
    e2e_steps = max(5, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        esp.esp_step(h, xh, eh, fh, uh, esp.ESP_HOST)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    esp.esp_destroy(h)

    extras = {}
    if not args.no_extras and world == 1:
        extras["plain_fp64"] = single_variant(args, local, stream, flush, s, precision=esp.ESP_FP64)
        extras["gaussian"] = single_variant(args, local, stream, flush, s, kernel=esp.ESP_KERNEL_GAUSS)
        # the ik force method (Methods, step 5): three more inverse FFTs
        extras["ik"] = single_variant(args, local, stream, flush, s, diff=esp.ESP_DIFF_IK)
        # the same compute with the virial (local pair terms and spectral modes)
        extras["virial"] = single_variant(args, local, stream, flush, s, virial=1)
        # the "Default" comparator of Table 1: Gaussian split, cardinal B-spline window
        extras["default_bspline"] = single_variant(args, local, stream, flush, s, kernel=esp.ESP_KERNEL_GAUSS,
                                                   window=esp.ESP_WINDOW_BSPLINE)
        extras["batched"] = batched(args, local, stream, flush)
        extras["served"] = served(args, local)
        extras["large"] = large(args, local, stream, flush)
        # a triclinic cell: the same water density in a truncated
        # octahedron; last, and guarded, so that it cannot cost the lines above
        try:
            extras["triclinic"] = triclinic(args, local, stream, flush)
        except Exception as exc:         # reported in the JSON line
            extras["triclinic"] = {"error": f"{type(exc).__name__}: {exc}"}
        # the MD loop workload (velocity Verlet around the solve), likewise
        try:
            extras["md"] = md_loop(args, local, stream)
        except Exception as exc:         # reported in the JSON line
            extras["md"] = {"error": f"{type(exc).__name__}: {exc}"}

    total_ms, e2e_s = replicas.max_over_ranks([total_ms, e2e_s], device=dev)
    phases = {k: v / args.steps for k, v in phase_acc.items()}
    return dict(N=N, L=L, info=info, total_ms=total_ms, step_ms=step_ms, e2e_s=e2e_s,
                e2e_steps=e2e_steps, phases=phases, clocks=clocks, energy=float(e.cpu()[0]), extras=extras)


# ------------------------------------------------------------------ extras
def time_steps(step, stream, steps: int, flush) -> list:
    """Per-step device ms of `step` (CUDA events on `stream`, L2 flushed between steps)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def single_variant(args, local, stream, flush, s, tolerance=None, **opts):
    """atoms/s of the single-system path with other plan options."""
    import torch
    from paper_2505_09727_gb300 import esp
    dev = torch.device("cuda", local)
    tol = WORKLOAD["tolerance"] if tolerance is None else tolerance
    h = esp.esp_plan(s.L, s.n, tol, r_c=WORKLOAD["r_c_nm"], device=local, stream=stream.cuda_stream, **opts)
    info = esp.esp_plan_info(h)
    x = torch.tensor(s.pos, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
    esp.esp_set_charges(h, torch.tensor(s.q, device=dev))

    def step():
        esp.esp_step(h, x, e, f, None)

    for _ in range(3):
        step()
    ms = time_steps(step, stream, max(3, min(args.steps, 20)), flush)
    esp.esp_destroy(h)
    t = statistics.median(ms)
    return {"value": s.n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "n_f": info["n_f"], "P": info["P"],
            "window": ("pswf", "bspline")[info["window"]], "diff": ("ad", "ik")[info["diff"]],
            "tolerance": tol, "steps": len(ms)}


TRICLINIC = dict(workload="spce_water_1e5_molecules_truncated_octahedron", molecules=100_000, atoms=300_000,
                 density_per_nm3=33.4, r_c_nm=1.0, tolerance=1e-4, seed=2505)


def triclinic(args, local, stream, flush):
    """atoms/s of a triclinic plan (esp_plan_cell): 1e5 SPC/E-shaped water
    molecules in a truncated octahedron of the headline box's volume."""
    import torch
    from paper_2505_09727_gb300 import esp, inputs
    dev = torch.device("cuda", local)
    s = inputs.spce_water_cell(TRICLINIC["molecules"], density=TRICLINIC["density_per_nm3"], seed=TRICLINIC["seed"])
    h = esp.esp_plan_cell(s.H, s.n, TRICLINIC["tolerance"], r_c=TRICLINIC["r_c_nm"], device=local,
                          stream=stream.cuda_stream)
    info = esp.esp_plan_info(h)
    x = torch.tensor(s.pos, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
    esp.esp_set_charges(h, torch.tensor(s.q, device=dev))

    def step():
        esp.esp_step(h, x, e, f, None)

    for _ in range(3):
        step()
    ms = time_steps(step, stream, max(3, min(args.steps, 20)), flush)
    esp.esp_destroy(h)
    t = statistics.median(ms)
    return {"value": s.n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "n_f": info["n_f"], "P": info["P"],
            "n_cells": info["n_cells"], "steps": len(ms),
            "config": dict(TRICLINIC, cell="truncated_octahedron", cell_vectors_nm=s.H.T.round(6).tolist())}


MD_LOOP = dict(workload="spce_water_1e5_molecules_md", molecules=100_000, atoms=300_000, density_per_nm3=33.4,
               r_c_nm=1.0, lj_cutoff_nm=1.0, tolerance=1e-4, dt_ps=0.0005, temperature_K=300.0, seed=2505)


def md_loop(args, local, stream):
    """ns/day and energy change of the MD loop (esp_md_*): 1e5 flexible
    SPC/E-shaped water molecules, FP32 solve, velocity Verlet."""
    import torch
    from paper_2505_09727_gb300 import esp, inputs
    s = inputs.spce_water(MD_LOOP["molecules"], seed=MD_LOOP["seed"])
    v = inputs.water_velocities(MD_LOOP["molecules"], MD_LOOP["temperature_K"], seed=MD_LOOP["seed"])
    n_steps = max(10, min(args.steps, 50))
    with esp.Plan(s.L, s.n, MD_LOOP["tolerance"], r_c=MD_LOOP["r_c_nm"], device=local, stream=stream.cuda_stream,
                  prefactor=esp.MD_PREFACTOR) as p:
        p.set_charges(s.q)
        with esp.MD(p.handle, s.pos, v, dt=MD_LOOP["dt_ps"], lj_cutoff=MD_LOOP["lj_cutoff_nm"]) as sim:
            sim.run(3)                                   # graph capture, first forces
            torch.cuda.synchronize(torch.device("cuda", local))
            t0 = time.perf_counter()
            e = sim.run(n_steps)                         # ends with a device sync
            secs = time.perf_counter() - t0
    tot = e.sum(axis=1)
    ns_per_day = n_steps * MD_LOOP["dt_ps"] * 1e-3 / secs * 86400.0
    return {"value": ns_per_day, "unit": "ns/day", "ms_per_step": 1e3 * secs / n_steps, "steps": n_steps,
            "energy_change_kj_mol_per_atom": float(tot[-1] - tot[0]) / s.n,
            "max_energy_excursion_over_kinetic": float(np.max(np.abs(tot - tot[0])) / np.mean(e[:, 3])),
            "config": dict(MD_LOOP, L_nm=s.L)}


LARGE = dict(workload="spce_water_1e6_molecules", molecules=1_000_000, atoms=3_000_000, density_per_nm3=33.4,
             r_c_nm=1.0, tolerance=1e-5, seed=2505)


def large(args, local, stream, flush):
    """3e6-atom water box at 1e-5: PSWF split against the Gaussian split on
    the same machinery (the grid ratio is the method's point)."""
    from paper_2505_09727_gb300 import inputs
    s = inputs.spce_water(LARGE["molecules"], seed=LARGE["seed"])
    pswf = single_variant(args, local, stream, flush, s, tolerance=LARGE["tolerance"])
    gauss = single_variant(args, local, stream, flush, s, tolerance=LARGE["tolerance"], kernel=1)
    return {"value": pswf["value"], "unit": UNIT, "pswf": pswf, "gaussian": gauss,
            "grid_points_ratio": (gauss["n_f"] / pswf["n_f"]) ** 3, "speedup_vs_gaussian": pswf["value"] / gauss["value"],
            "config": dict(LARGE, L_nm=s.L)}


BATCH = dict(workload="electrolyte_batch_64", systems=64, atoms_lo=3000, atoms_hi=200_000,
             density_per_nm3=100.0, r_c_nm=1.0, tolerance=1e-4, seed=9727)


def batched(args, local, stream, flush):
    """64 independent electrolyte boxes, sizes log-uniform in [3e3, 2e5], one
    batch: bucketed batched FFTs, whole step replayed from a CUDA graph."""
    import torch
    from paper_2505_09727_gb300 import esp, inputs
    dev = torch.device("cuda", local)
    sizes = inputs.batch_sizes(BATCH["systems"], BATCH["atoms_lo"], BATCH["atoms_hi"], seed=BATCH["seed"])
    systems = inputs.electrolyte_batch(sizes, seed=BATCH["seed"])
    pos, q = inputs.concat(systems)
    n = int(pos.shape[0])
    t0 = time.perf_counter()
    b = esp.esp_batch_create([s.L for s in systems], [s.n for s in systems], BATCH["tolerance"],
                             r_c=BATCH["r_c_nm"], device=local, stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    grids = sorted({esp.esp_batch_info(b, i)["n_f"] for i in range(len(systems))})
    esp.esp_batch_set_charges(b, q)
    x = torch.tensor(pos, device=dev)
    e = torch.zeros(len(systems), dtype=torch.float64, device=dev)
    f = torch.zeros((n, 3), dtype=torch.float64, device=dev)

    def step():
        esp.esp_batch_compute(b, x, e, f, None)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    ms = time_steps(step, stream, max(3, min(args.steps, 20)), flush)
    # phases (direct launches, serialised) for the breakdown
    esp.esp_batch_set_timing(b, 2)
    step()
    phases = esp.esp_batch_phase_times(b)
    esp.esp_batch_set_timing(b, 0)
    # end to end with pinned host buffers
    xh = torch.tensor(pos).pin_memory()
    fh = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    eh = torch.zeros(len(systems), dtype=torch.float64).pin_memory()
    esp.esp_batch_compute(b, xh, eh, fh, None, esp.ESP_HOST)
    k = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(k):
        esp.esp_batch_compute(b, xh, eh, fh, None, esp.ESP_HOST)
    e2e_s = (time.perf_counter() - t0) / k
    esp.esp_batch_destroy(b)
    t = statistics.median(ms)
    return {"value": n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "atoms": n, "systems": len(systems),
            "grid_sizes": grids, "create_s": round(t_create, 3), "steps": len(ms),
            "phases_ms": {k2: round(v, 5) for k2, v in phases.items()},
            "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * 24,
                    "d2h_bytes_per_step": n * 24 + 8 * len(systems)},
            "config": BATCH}


SERVE = dict(workload="served_electrolyte", systems=64, atoms_lo=1000, atoms_hi=200_000, requests=2000,
             tolerances=[1e-3, 1e-4, 1e-5], sigma_nm=0.01, density_per_nm3=100.0, r_c_nm=1.0,
             budget_gb=150.0, loads=[0.5, 0.8, 0.95], seed=1000)
SERVE_FULL = dict(SERVE, systems=256, atoms_hi=1_000_000, requests=10_000)


def served(args, local):
    """Request server: resident systems, Poisson arrivals, p50/p99 latency.

    Saturation: every request submitted at once (closed loop); then Poisson
    arrivals at the given fractions of the saturated request rate."""
    import threading
    from paper_2505_09727_gb300 import esp, inputs
    cfg = SERVE_FULL if args.served_full else SERVE
    rng = np.random.default_rng(cfg["seed"])
    sizes = inputs.batch_sizes(cfg["systems"], cfg["atoms_lo"], cfg["atoms_hi"], seed=cfg["seed"])
    systems = inputs.electrolyte_batch(sizes, seed=cfg["seed"])
    nmax = int(max(sizes))
    noise = [rng.normal(0.0, cfg["sigma_nm"], size=(nmax, 3)) for _ in range(4)]
    reqs = []
    for k in range(cfg["requests"]):
        i = int(rng.integers(len(systems)))
        reqs.append((i, float(rng.choice(cfg["tolerances"])), k % len(noise)))

    def positions(i, k):
        s = systems[i]
        return np.mod(s.pos + noise[k][: s.n], s.L)

    srv = esp.Server(cfg["r_c_nm"], memory_budget=int(cfg["budget_gb"] * 1e9), device=local, max_inflight=8)
    ids = [srv.add_system(s.L, s.q) for s in systems]
    # plans for every (system, tolerance) the stream uses, created before timing
    t0 = time.perf_counter()
    for i, eps in sorted({(i, e) for i, e, _ in reqs}):
        srv.wait(srv.submit(ids[i], eps, systems[i].pos), forces=False, potential=False)
    t_plans = time.perf_counter() - t0
    pos_cache = {}

    def run(rate):
        """rate None: closed loop with 64 requests outstanding; else Poisson."""
        import queue
        esp.esp_server_reset_stats(srv.handle)
        window = threading.Semaphore(64 if rate is None else 512)
        pending = queue.Queue()

        def waiter():
            while True:
                t = pending.get()
                if t is None:
                    return
                srv.wait(t, forces=False, potential=False)
                window.release()

        th = threading.Thread(target=waiter)
        th.start()
        t_start = time.perf_counter()
        next_t = t_start
        for i, eps, k in reqs:
            if rate:
                next_t += rng.exponential(1.0 / rate)
                d = next_t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            window.acquire()
            pending.put(srv.submit(ids[i], eps, pos_cache[(i, k)]))
        pending.put(None)
        th.join()
        wall = time.perf_counter() - t_start
        st = srv.stats()
        return dict(wall_s=wall, requests_per_s=len(reqs) / wall, atoms_per_s=st["atoms_done"] / wall,
                    p50_ms=st["latency_p50_ms"], p99_ms=st["latency_p99_ms"])

    for i, eps, k in reqs:                        # positions prepared outside the timed runs
        pos_cache.setdefault((i, k), positions(i, k))
    sat = run(None)
    loads = {}
    for f in cfg["loads"]:
        r = run(f * sat["requests_per_s"])
        loads[str(f)] = {k: round(v, 4) for k, v in r.items()}
    st = srv.stats()
    srv.close()
    atoms = float(sum(systems[i].n for i, _, _ in reqs))
    return {"value": sat["atoms_per_s"], "unit": UNIT, "requests": len(reqs), "atoms_per_pass": atoms,
            "saturated": {k: round(v, 4) for k, v in sat.items()}, "poisson": loads,
            "plans": st["plans_created"], "evictions": st["evictions"],
            "device_gb": round(st["device_bytes"] / 1e9, 3), "plan_setup_s": round(t_plans, 2),
            "config": dict(cfg, scaled=not args.served_full)}


# --------------------------------------------------------------- CPU oracle
def cpu_baseline(molecules: int, budget_atoms: int = 1500):
    """Time the FP64 CPU oracle on a bounded sample of the workload.

    Per step the oracle spreads all N atoms and runs the FFT pair (timed in
    full); interpolation and the local pair sum are per atom (timed on
    `budget_atoms` sampled atoms and scaled to N).
    """
    from oracle import esp as oesp
    from oracle import params as oparams
    from oracle import pswf
    from paper_2505_09727_gb300 import inputs

    s = inputs.spce_water(molecules, seed=WORKLOAD["seed"])
    eps, r_c = WORKLOAD["tolerance"], WORKLOAD["r_c_nm"]
    pl = oparams.plan(eps, s.L, r_c)
    p = oesp.ESPParams(eps, r_c, pl["P"], pl["n_f"], pl["c"], pl["c1"])
    split = p.split()
    window = pswf.PSWFWindow(p.c1, p.P)
    idx = np.sort(np.random.default_rng(0).choice(s.n, size=min(budget_atoms, s.n), replace=False))
    t0 = time.perf_counter()
    oesp.far_field(s.pos, s.q, s.L, p.n_f, r_c, split, window, idx[:0])
    t_fixed = time.perf_counter() - t0                 # spread of all atoms + FFT pair
    t0 = time.perf_counter()
    oesp.far_field(s.pos, s.q, s.L, p.n_f, r_c, split, window, idx)
    t_gather = max(time.perf_counter() - t0 - t_fixed, 0.0)
    t0 = time.perf_counter()
    oesp.near_field(s.pos, s.q, s.L, r_c, split, idx)
    t_near = time.perf_counter() - t0
    t_step = t_fixed + (t_gather + t_near) / len(idx) * s.n
    return {"value": s.n / t_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, same {s.n}-atom water box and parameters: spread of all "
                       f"atoms + FFT pair timed in full ({t_fixed:.2f} s); interpolation and local part "
                       f"timed on {len(idx)} sampled atoms ({t_gather + t_near:.2f} s) and scaled to N; "
                       f"single-threaded"),
            "seconds_per_step": t_step}


# --------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = []
        base = None
        for _ in range(max(1, min(args.steps, 3))):
            base = cpu_baseline(args.molecules)
            vals.append(base["value"])
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
                "steps": len(vals), "warmup": args.warmup, "ms_per_step": base["seconds_per_step"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(WORKLOAD, molecules=args.molecules),
                "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    from paper_2505_09727_gb300 import replicas
    if world > 1:
        replicas.init("nccl")
    r = run_gpu(args, world, rank, local)
    N = r["N"]
    value = replicas.whole_job_rate(N * args.steps, world, r["total_ms"] * 1e-3)
    e2e_value = replicas.whole_job_rate(N * r["e2e_steps"], world, r["e2e_s"])
    # our kernels per step (cuFFT's own and memsets not counted): ingest, 3 scan
    # passes, scatter, local part (column clusters, 3 scan passes, cluster
    # list, pair kernel), spread, scale, gather, finalize, energy
    kernels_per_step = 16
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, molecules=args.molecules, tolerance=args.tolerance, atoms=N, L_nm=r["L"], n_f=r["info"]["n_f"],
                       P=r["info"]["P"], c=r["info"]["c"], c1=r["info"]["c1"], l2="flushed_between_steps",
                       parallelism=f"replicas{world}"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * 3 * 8,
                "d2h_bytes_per_step": N * 3 * 8 + N * 8 + 8},
        "gpu_launches": kernels_per_step * args.steps,
        "phases_ms": {k: round(v, 5) for k, v in r["phases"].items()},
        "step_ms_p50": statistics.median(r["step_ms"]),
        "step_ms_p99": float(np.percentile(r["step_ms"], 99)),
        "clocks": r["clocks"],
    }
    line.update(r["extras"])
    if "default_bspline" in line:
        d = line["default_bspline"]
        d["grid_points_ratio"] = (d["n_f"] / r["info"]["n_f"]) ** 3
        d["esp_speedup"] = value / world / d["value"]
    line["roofline"] = roofline(r["phases"], r["info"], N, r["L"], r["clocks"], args.steps)
    line["phase_roofline"] = phase_rooflines(r["phases"], r["info"], N, r["L"], r["clocks"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.molecules)
        line["cpu_baseline"] = {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line))
    replicas.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
