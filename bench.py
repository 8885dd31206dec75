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
    """SM clocks and clock-event reasons while the timed steps run.

    NVML read-only queries (through ctypes, from a thread) every 5 ms, so a
    timed region of a few tens of milliseconds still holds several samples;
    without NVML, nvidia-smi every 200 ms. Nothing is ever set.
    """
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of NVML
    NVML_REASONS = ((0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
                    (0x40, "hw_thermal_slowdown"))
    NVML_CLOCK_SM = 1
    PERIOD_S = 0.005

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.thread = None
        self.path = os.path.join(tempfile.gettempdir(), f"esp_bench_clocks_rank{index}.csv")

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        handle = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(handle)) == 0
        except (AttributeError, RuntimeError, ImportError):
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(handle)) != 0:
            return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, handle, reasons

    def _poll(self, lib, handle, reasons_fn):
        import ctypes
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(clk)) == 0 and \
                    reasons_fn(handle, ctypes.byref(rs)) == 0:
                self.samples.append((clk.value, rs.value))
            time.sleep(self.PERIOD_S)

    def start(self):
        import threading
        try:
            nv = self._nvml_handle()
        except (OSError, AttributeError):
            nv = None
        if nv is not None:
            import ctypes
            lib, handle, reasons_fn = nv
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(
                handle, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0 else None
            self.samples = []
            self.stop_flag = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=nv, daemon=True)
            self.thread.start()
            return
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
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            if not self.samples:
                return None
            sm = [float(c) for c, _ in self.samples]
            reasons = {name for c, r in self.samples for bit, name in self.NVML_REASONS if r & bit}
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz or max(sm),
                    "sm_min_mhz": min(sm), "reasons": sorted(reasons), "samples": len(sm),
                    "source": "NVML every 5 ms"}
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
                "samples": len(sm), "source": "nvidia-smi every 200 ms"}


# ------------------------------------------------------------------ roofline
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work of one unordered pair of the local part (the count the
# roofline uses): about 30 flop, i.e. difference 3, r^2 5, 1/r 1, the split
# function and its derivative ~10, potential and force terms on both atoms ~11.
NEAR_FLOPS_PER_PAIR = 30
# What the kernel itself issues per evaluated pair (reported beside it):
# difference 3, r^2 5, rsqrt 1, polynomial argument 2, two Horner polynomials
# of about 9 terms 2 x 18, potentials 2 + 2, r^-3 terms 4, forces on both
# atoms 2 x (1 + 6); the packed f32x2 form does two pairs per instruction.
NEAR_ISSUED_FLOPS_PER_PAIR = 71
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


def measure_peaks(device: int, reps: int = 5) -> dict:
    """FP32 and shared-memory throughput of this GPU at its current clocks,
    from the microbenchmarks of libesp_peaks.so (independent FFMA and packed
    FFMA2 chains on every SM; shared atomicAdd and read-add-write to
    conflict-free addresses). Best of `reps` launches each."""
    import ctypes
    from paper_2505_09727_gb300 import _build
    lib = ctypes.CDLL(_build.PEAKS_LIB)
    out = (ctypes.c_double * 6)()
    if lib.esp_measure_peaks(int(device), int(reps), out) != 0:
        raise RuntimeError("peak microbenchmarks failed")
    return {"fp32_ffma_tflops": out[0] / 1e12, "fp32_ffma2_tflops": out[1] / 1e12,
            "fp32_tflops": max(out[0], out[1]) / 1e12, "shared_atomic_gops": out[2] / 1e9,
            "shared_rmw_gops": out[3] / 1e9, "sms": int(out[4])}


def roofline(phases: dict, info: dict, n_atoms: int, L: float, peaks_gpu: dict):
    """Roofline of the dominant kernel (largest average serialised duration).

    Algorithmic work per launch:
      near    FP32: unique pairs within r_c (N * 4/3 pi r_c^3 rho / 2) x
              NEAR_FLOPS_PER_PAIR, against the FP32 multiply-add peak measured
              in this run (the larger of the scalar and packed rates)
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
    out = {"kernel": kernel, "bound": bound}
    if bound == "alu":
        peak = peaks_gpu["fp32_tflops"]
        achieved = work / t / 1e12
        out.update(achieved=achieved, peak=peak, unit=unit, frac=achieved / peak,
                   peak_source=(f"measured in this run: FP32 multiply-add microbenchmark on all "
                                f"{peaks_gpu['sms']} SMs (scalar {peaks_gpu['fp32_ffma_tflops']:.1f}, packed f32x2 "
                                f"{peaks_gpu['fp32_ffma2_tflops']:.1f} TFLOP/s; the larger)"),
                   flops_per_pair=NEAR_FLOPS_PER_PAIR, pairs_per_launch=pairs,
                   issued_flops_per_pair=NEAR_ISSUED_FLOPS_PER_PAIR,
                   issued_tflops=pairs * NEAR_ISSUED_FLOPS_PER_PAIR / t / 1e12)
    else:
        peak = peaks["hbm_gbs"]
        achieved = work / t / 1e9
        out.update(achieved=achieved, peak=peak, unit=unit, frac=achieved / peak,
                   peak_source=f"{source} HBM copy bandwidth (MEASURED_PEAKS.json)")
    out.update(traffic=profiled_traffic(kernel), algorithmic_per_launch=work, avg_launch_ms=phases[kernel])
    return out


def phase_rooflines(phases: dict, info: dict, n_atoms: int, L: float, peaks_gpu: dict) -> dict:
    """Every phase (serialised CUDA-event time) against each resource: its
    algorithmic DRAM bytes over the measured HBM copy bandwidth; for the
    arithmetic phases its FP32 flops over the measured FP32 peak; for the
    spread its P^3 shared-memory read-add-writes per atom over the measured
    shared read-add-write rate.

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
    fp32 = peaks_gpu["fp32_tflops"]
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
    out = {"hbm_peak_gbs": hbm, "hbm_peak_source": source, "fp32_peak_tflops": fp32,
           "shared_rmw_peak_gops": peaks_gpu["shared_rmw_gops"], "fp32_peak_source": "measured in this run"}
    for k, (b, f) in work.items():
        t = phases.get(k, 0.0) * 1e-3
        if t <= 0:
            continue
        row = {"ms": round(phases[k], 5), "hbm_gbs": round(b / t / 1e9, 2), "hbm_frac": round(b / t / 1e9 / hbm, 5)}
        if f:
            row["fp32_tflops"] = round(f / t / 1e12, 3)
            row["fp32_frac"] = round(f / t / 1e12 / fp32, 5)
        if k == "spread":
            rmw = n_atoms * P ** 3 / t / 1e9
            row["shared_rmw_gops"] = round(rmw, 2)
            row["shared_rmw_frac"] = round(rmw / peaks_gpu["shared_rmw_gops"], 5)
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
    esp.esp_set_timing(h, 0)
    # roofline denominators, measured at the clocks of this run (still sampled)
    peaks_gpu = measure_peaks(local)
    clocks = sampler.stop()
    # the error of this result: the last step's forces and energy against the
    # eps = 1e-10 reference
    ref = reference_solve(s, local, stream)
    delta = stated_error(f.cpu().numpy(), float(e.cpu()[0]), ref, WORKLOAD["tolerance"])

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
        extras["plain_fp64"] = single_variant(args, local, stream, flush, s, ref=ref, precision=esp.ESP_FP64)
        extras["gaussian"] = single_variant(args, local, stream, flush, s, ref=ref, kernel=esp.ESP_KERNEL_GAUSS)
        # the ik force method (Methods, step 5): three more inverse FFTs
        extras["ik"] = single_variant(args, local, stream, flush, s, ref=ref, diff=esp.ESP_DIFF_IK)
        # the same compute with the virial (local pair terms and spectral modes)
        extras["virial"] = single_variant(args, local, stream, flush, s, ref=ref, virial=1)
        # the "Default" comparator of Tables 1 and 2: Gaussian split, B-spline window of order 5
        extras["default_bspline"] = single_variant(args, local, stream, flush, s, ref=ref,
                                                   kernel=esp.ESP_KERNEL_GAUSS, window=esp.ESP_WINDOW_BSPLINE)
        extras["batched"] = batched(args, local, stream, flush)
        extras["served"] = served(args, local)
        extras["large"] = large(args, local, stream, flush, peaks_gpu)
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
                e2e_steps=e2e_steps, phases=phases, clocks=clocks, energy=float(e.cpu()[0]), extras=extras,
                peaks=peaks_gpu, delta=delta)


# ------------------------------------------------------------ stated errors
REFERENCE_EPS = 1e-10


def reference_solve(s, local, stream, r_c=None) -> dict:
    """The reference each result's error is stated against: the same method
    at eps = 1e-10 parameters in FP64 (the paper's reference for systems
    where classical Ewald is out of reach), same r_c, on the GPU's FP64
    path (which the tests hold to the CPU oracle to 1e-9 and to converged
    Ewald to 1e-9)."""
    from paper_2505_09727_gb300 import esp
    with esp.Plan(s.L, s.n, REFERENCE_EPS, r_c=r_c or WORKLOAD["r_c_nm"], precision=esp.ESP_FP64, device=local,
                  stream=stream.cuda_stream) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, _ = p.compute()
        info = p.info
    return {"energy": e, "forces": f, "n_f": info["n_f"], "P": info["P"]}


def stated_error(forces, energy, ref: dict, tolerance: float) -> dict:
    """Relative RMS force error over all atoms (Eq. Deltadef) and relative
    energy error against `ref`."""
    f = np.asarray(forces, dtype=np.float64)
    d = float(np.sqrt(np.sum((f - ref["forces"]) ** 2) / np.sum(ref["forces"] ** 2)))
    return {"force_rel_rms": d, "energy_rel": abs(energy - ref["energy"]) / abs(ref["energy"]),
            "tolerance": tolerance, "within_tolerance": d <= tolerance,
            "reference": (f"FP64 ESP at eps={REFERENCE_EPS:g} parameters (P {ref['P']}, n_f {ref['n_f']}), "
                          f"same r_c, all atoms")}


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


def single_variant(args, local, stream, flush, s, tolerance=None, ref=None, peaks_gpu=None, **opts):
    """atoms/s of the single-system path with other plan options (and the
    error of its last step against `ref`); with peaks_gpu, also its
    serialised phase times and every phase against the measured peaks."""
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
    phases = None
    if peaks_gpu is not None:
        # second pass: phases serialised and bracketed by CUDA events
        esp.esp_set_timing(h, 2)
        phases = {k: 0.0 for k in esp.PHASES}
        n_ph = max(3, min(args.steps, 10))
        for _ in range(n_ph):
            flush.zero_()
            step()
            for k, v in esp.esp_phase_times(h).items():
                phases[k] += v / n_ph
        torch.cuda.synchronize(dev)
        esp.esp_set_timing(h, 0)
    esp.esp_destroy(h)
    t = statistics.median(ms)
    out = {"value": s.n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "n_f": info["n_f"], "P": info["P"],
           "window": ("pswf", "bspline")[info["window"]], "diff": ("ad", "ik")[info["diff"]],
           "tolerance": tol, "steps": len(ms)}
    if phases is not None:
        out["phases_ms"] = {k: round(v, 5) for k, v in phases.items()}
        out["phase_roofline"] = phase_rooflines(phases, info, s.n, s.L, peaks_gpu)
    if ref is not None:
        out["delta"] = stated_error(f.cpu().numpy(), float(e.cpu()[0]), ref, tol)
    return out


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
    # reference: triclinic cells run in FP32 only, so the same method at
    # eps = 1e-6 parameters in FP32 (its own error and rounding ~1e-6)
    with esp.Plan(s.H, s.n, 1e-6, r_c=TRICLINIC["r_c_nm"], device=local, stream=stream.cuda_stream) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e_ref, f_ref, _ = p.compute()
        rinfo = p.info
    delta = stated_error(f.cpu().numpy(), float(e.cpu()[0]), {"energy": e_ref, "forces": f_ref, "P": rinfo["P"],
                                                             "n_f": rinfo["n_f"]}, TRICLINIC["tolerance"])
    delta["reference"] = (f"FP32 ESP on the same cell at eps=1e-6 parameters (P {rinfo['P']}, n_f "
                          f"{rinfo['n_f']}), all atoms (triclinic cells have no FP64 path)")
    return {"value": s.n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "n_f": info["n_f"], "P": info["P"],
            "n_cells": info["n_cells"], "steps": len(ms), "delta": delta,
            "config": dict(TRICLINIC, cell="truncated_octahedron", cell_vectors_nm=s.H.T.round(6).tolist())}


MD_LOOP = dict(workload="spce_water_1e5_molecules_md", molecules=100_000, atoms=300_000, density_per_nm3=33.4,
               r_c_nm=1.0, lj_cutoff_nm=1.0, tolerance=1e-4, dt_ps=0.0005, temperature_K=300.0, seed=2505)
MD_DRIFT = dict(MD_LOOP, workload="spce_water_1e4_molecules_md_drift", molecules=10_000, atoms=30_000, steps=20_000)


def md_loop(args, local, stream):
    """ns/day of the MD loop (esp_md_*: 1e5 flexible SPC/E-shaped water
    molecules, FP32 solve, velocity Verlet, every step one CUDA graph), and
    the energy drift over 2e4 steps (10 ps) of a 1e4-molecule box: the slope
    of a least-squares line through the total energy, per atom."""
    import torch
    from paper_2505_09727_gb300 import esp, inputs

    def run(cfg, n_steps):
        s = inputs.spce_water(cfg["molecules"], seed=cfg["seed"])
        v = inputs.water_velocities(cfg["molecules"], cfg["temperature_K"], seed=cfg["seed"])
        with esp.Plan(s.L, s.n, cfg["tolerance"], r_c=cfg["r_c_nm"], device=local, stream=stream.cuda_stream,
                      prefactor=esp.MD_PREFACTOR) as p:
            p.set_charges(s.q)
            with esp.MD(p.handle, s.pos, v, dt=cfg["dt_ps"], lj_cutoff=cfg["lj_cutoff_nm"]) as sim:
                sim.run(3)                                   # graph capture, first forces
                torch.cuda.synchronize(torch.device("cuda", local))
                t0 = time.perf_counter()
                e = sim.run(n_steps)                         # ends with a device sync
                secs = time.perf_counter() - t0
        return s, e, secs

    n_steps = max(50, min(4 * args.steps, 200))
    s, e, secs = run(MD_LOOP, n_steps)
    tot = e.sum(axis=1)
    ns_per_day = n_steps * MD_LOOP["dt_ps"] * 1e-3 / secs * 86400.0
    out = {"value": ns_per_day, "unit": "ns/day", "ms_per_step": 1e3 * secs / n_steps, "steps": n_steps,
           "energy_change_kj_mol_per_atom": float(tot[-1] - tot[0]) / s.n,
           "max_energy_excursion_over_kinetic": float(np.max(np.abs(tot - tot[0])) / np.mean(e[:, 3])),
           "config": dict(MD_LOOP, L_nm=s.L)}
    sd, ed, secs_d = run(MD_DRIFT, MD_DRIFT["steps"])
    totd = ed.sum(axis=1)
    t_ns = np.arange(len(totd)) * MD_DRIFT["dt_ps"] * 1e-3
    slope = float(np.polyfit(t_ns, totd, 1)[0])
    out["drift"] = {"kj_mol_per_ns_per_atom": slope / sd.n, "steps": MD_DRIFT["steps"],
                    "simulated_ps": MD_DRIFT["steps"] * MD_DRIFT["dt_ps"],
                    "max_excursion_over_kinetic": float(np.max(np.abs(totd - totd[0])) / np.mean(ed[:, 3])),
                    "ms_per_step": 1e3 * secs_d / MD_DRIFT["steps"], "config": dict(MD_DRIFT, L_nm=sd.L)}
    return out


LARGE = dict(workload="spce_water_1e6_molecules", molecules=1_000_000, atoms=3_000_000, density_per_nm3=33.4,
             r_c_nm=1.0, tolerance=1e-5, seed=2505)


def large(args, local, stream, flush, peaks_gpu=None):
    """3e6-atom water box at 1e-5: PSWF split against the Gaussian split on
    the same machinery (the grid ratio is the method's point); the PSWF
    solve's phases against the measured peaks (n_f = 144, P = 8: the grid
    is 12 MB, so the spread and gather tiles come from L2 and HBM)."""
    from paper_2505_09727_gb300 import inputs
    s = inputs.spce_water(LARGE["molecules"], seed=LARGE["seed"])
    ref = reference_solve(s, local, stream)
    pswf = single_variant(args, local, stream, flush, s, tolerance=LARGE["tolerance"], ref=ref,
                          peaks_gpu=peaks_gpu)
    gauss = single_variant(args, local, stream, flush, s, tolerance=LARGE["tolerance"], ref=ref, kernel=1)
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
    # stated error: every system against an FP64 batch at eps = 1e-10 parameters
    fh_np = fh.numpy().copy()
    rb = esp.esp_batch_create([s.L for s in systems], [s.n for s in systems], REFERENCE_EPS, r_c=BATCH["r_c_nm"],
                              precision=esp.ESP_FP64, device=local, stream=stream.cuda_stream)
    esp.esp_batch_set_charges(rb, q)
    f_ref = np.zeros((n, 3))
    e_ref = np.zeros(len(systems))
    esp.esp_batch_compute(rb, pos, e_ref, f_ref, None, esp.ESP_HOST)
    esp.esp_batch_destroy(rb)
    per_sys, a0 = [], 0
    for sy in systems:
        sl = slice(a0, a0 + sy.n)
        per_sys.append(float(np.sqrt(np.sum((fh_np[sl] - f_ref[sl]) ** 2) / np.sum(f_ref[sl] ** 2))))
        a0 += sy.n
    delta = stated_error(fh_np, float(eh.sum()), {"energy": float(e_ref.sum()), "forces": f_ref, "P": "13",
                                                  "n_f": "per system"}, BATCH["tolerance"])
    delta.update(max_system_force_rel_rms=max(per_sys), systems_within_tolerance=sum(d <= BATCH["tolerance"]
                                                                                         for d in per_sys),
                 reference=f"FP64 batch of the same systems at eps={REFERENCE_EPS:g} parameters, all atoms")
    return {"value": n / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "atoms": n, "systems": len(systems),
            "delta": delta,
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

    def run(rate, clients=4):
        """rate None: closed loop with 64 requests outstanding; else Poisson
        arrivals. Requests are handed to `clients` submitting threads (each
        submission copies the request's positions into the server's pinned
        buffers, so one thread caps the request rate); one thread collects."""
        import queue
        esp.esp_server_reset_stats(srv.handle)
        window = threading.Semaphore(64 if rate is None else 512)
        arrivals = queue.Queue()
        pending = queue.Queue()

        def client():
            while True:
                item = arrivals.get()
                if item is None:
                    return
                i, eps, k = item
                window.acquire()
                pending.put(srv.submit(ids[i], eps, pos_cache[(i, k)]))

        def waiter():
            while True:
                t = pending.get()
                if t is None:
                    return
                srv.wait(t, forces=False, potential=False)
                window.release()

        subs = [threading.Thread(target=client) for _ in range(clients)]
        th = threading.Thread(target=waiter)
        for t in subs:
            t.start()
        th.start()
        t_start = time.perf_counter()
        next_t = t_start
        for item in reqs:
            if rate:
                next_t += rng.exponential(1.0 / rate)
                d = next_t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            arrivals.put(item)
        for _ in subs:
            arrivals.put(None)
        for t in subs:
            t.join()
        pending.put(None)
        th.join()
        wall = time.perf_counter() - t_start
        st = srv.stats()
        return dict(wall_s=wall, requests_per_s=len(reqs) / wall, atoms_per_s=st["atoms_done"] / wall,
                    p50_ms=st["latency_p50_ms"], p99_ms=st["latency_p99_ms"],
                    peak_concurrent=st["peak_concurrent"], overlap_ms=st["overlap_ms"])

    for i, eps, k in reqs:                        # positions prepared outside the timed runs
        pos_cache.setdefault((i, k), positions(i, k))
    sat = run(None)
    loads = {}
    for f in cfg["loads"]:
        r = run(f * sat["requests_per_s"])
        loads[str(f)] = {k: round(v, 4) for k, v in r.items()}
    st = srv.stats()
    # stated errors: the two largest systems' requests at each tolerance,
    # served with forces, against FP64 plans at eps = 1e-10 parameters
    delta = {}
    for eps in cfg["tolerances"]:
        picks = sorted({(systems[i].n, i, k) for i, e2, k in reqs if e2 == eps})[-2:]
        worst = 0.0
        for _, i, k in picks:
            pos = pos_cache[(i, k)]
            _, f_got, _, _ = srv.wait(srv.submit(ids[i], eps, pos), potential=False)
            sy = systems[i]
            with esp.Plan(sy.L, sy.n, REFERENCE_EPS, r_c=cfg["r_c_nm"], precision=esp.ESP_FP64, device=local) as p:
                p.set_charges(sy.q)
                p.set_positions(pos)
                _, f_ref, _ = p.compute()
            worst = max(worst, float(np.sqrt(np.sum((f_got - f_ref) ** 2) / np.sum(f_ref ** 2))))
        delta[str(eps)] = {"force_rel_rms_max": worst, "requests": len(picks), "within_tolerance": worst <= eps}
    delta["reference"] = (f"FP64 ESP at eps={REFERENCE_EPS:g} parameters on the request's positions, all atoms; "
                          f"the two largest systems requested at each tolerance")
    srv.close()
    atoms = float(sum(systems[i].n for i, _, _ in reqs))
    return {"value": sat["atoms_per_s"], "unit": UNIT, "requests": len(reqs), "atoms_per_pass": atoms,
            "delta": delta, "saturated": {k: round(v, 4) for k, v in sat.items()}, "poisson": loads,
            "plans": st["plans_created"], "evictions": st["evictions"],
            "device_gb": round(st["device_bytes"] / 1e9, 3), "plan_setup_s": round(t_plans, 2),
            "config": dict(cfg, scaled=not args.served_full)}


# --------------------------------------------------------------- CPU oracle
# The CPU baseline: whole steps of the FP64 oracle (every atom's potential
# and forces, and the energy) on all host cores, on a water box of the
# headline workload's density, cutoff and tolerance, 5e3 molecules (1.5e4
# atoms) so that a step takes about a second; atoms/s is per-atom work, the
# same per atom as at 3e5 atoms up to the FFT share.
CPU_SAMPLE = dict(WORKLOAD, workload="spce_water_5e3_molecules", molecules=5_000, atoms=15_000)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)


def _oracle_chunk(task):
    """Oracle ESP (spread of all atoms, transforms, interpolation and local
    part for the chunk's atoms) in a worker process."""
    pos, q, L, p, idx = task
    from oracle import esp as oesp
    r = oesp.esp(pos, q, L, p, idx)
    return idx, r["potential"], r["forces"]


class OracleStepper:
    """Whole oracle steps over a process pool (spawned: safe after CUDA use)."""

    def __init__(self, molecules: int):
        import multiprocessing as mp
        from oracle import esp as oesp
        from oracle import params as oparams
        from paper_2505_09727_gb300 import inputs
        self.s = inputs.spce_water(molecules, seed=WORKLOAD["seed"])
        eps, r_c = WORKLOAD["tolerance"], WORKLOAD["r_c_nm"]
        pl = oparams.plan(eps, self.s.L, r_c)
        self.p = oesp.ESPParams(eps, r_c, pl["P"], pl["n_f"], pl["c"], pl["c1"])
        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init)
        self.chunks = np.array_split(np.arange(self.s.n), 2 * self.cores)

    def step(self):
        s = self.s
        u = np.zeros(s.n)
        f = np.zeros((s.n, 3))
        tasks = [(s.pos, s.q, s.L, self.p, idx) for idx in self.chunks]
        for idx, ui, fi in self.pool.map(_oracle_chunk, tasks):
            u[idx] = ui
            f[idx] = fi
        return 0.5 * float(np.dot(s.q, u)), f, u

    def describe(self, n_steps: int, seconds: float) -> dict:
        return {"value": self.s.n * n_steps / seconds, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "cpu_model": cpu_model(),
                "sample": (f"whole steps of the FP64 NumPy/SciPy oracle (spread, FFTs, influence, interpolation, "
                           f"local part, energy for every atom) on a {self.s.n}-atom SPC/E-shaped water box of the "
                           f"headline density, r_c and tolerance (n_f {self.p.n_f}, P {self.p.P}); atoms split "
                           f"over {self.cores} worker processes; {n_steps} timed steps, "
                           f"{seconds / n_steps:.2f} s per step")}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(steps: int = 3, warmup: int = 1) -> dict:
    st = OracleStepper(CPU_SAMPLE["molecules"])
    try:
        for _ in range(warmup):
            st.step()
        t0 = time.perf_counter()
        for _ in range(steps):
            st.step()
        secs = time.perf_counter() - t0
        return st.describe(steps, secs)
    finally:
        st.close()


# --------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        # this tier's reference arm: the CPU oracle on the host cores, whole
        # steps of a bounded sample of the workload (CPU_SAMPLE), exactly
        # --warmup untimed and --steps timed steps; rank 0 only
        if rank != 0:
            return 0
        st = OracleStepper(CPU_SAMPLE["molecules"])
        try:
            for _ in range(args.warmup):
                st.step()
            times = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                st.step()
                times.append(time.perf_counter() - t0)
        finally:
            st.close()
        base = st.describe(args.steps, sum(times))
        value = base["value"]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": CPU_SAMPLE,
                "cpu_baseline": base,
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
    line["delta"] = r["delta"]
    line["measured_peaks"] = r["peaks"]
    line["roofline"] = roofline(r["phases"], r["info"], N, r["L"], r["peaks"])
    line["phase_roofline"] = phase_rooflines(r["phases"], r["info"], N, r["L"], r["peaks"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    replicas.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
