"""The high-accuracy large box at full size, and the reference the benchmark
states its errors against.

* 1e6 SPC/E-shaped water molecules (3e6 atoms, L = 31.05 nm) at 1e-5 with
  r_c = 1 nm, the benchmark's `large` configuration (P = 8, n_f = 144): the
  FP32 solve equals the oracle at the plan's parameters on sampled atoms
  (FP32 parity bound), and its relative RMS force error over all atoms
  against the FP64 solve at eps = 1e-10 parameters is at most 1e-5 (the
  paper's reference for systems where Ewald is out of reach: the same
  method at raised parameters).
* That reference: the FP64 solve at eps = 1e-10 parameters matches
  converged classical Ewald to 1e-9 on a water box small enough for Ewald.
* The batched workload at full size (64 electrolyte boxes, 3.24e6 atoms):
  sampled atoms of three systems against the oracle at their batch
  parameters, every system against an FP64 batch at 1e-10 parameters.
"""
import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald, metrics
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_PARITY = 5e-6


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def solve(esp, s, eps, **opts):
    with esp.Plan(s.L, s.n, eps, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, u = p.compute()
        info = p.info
    return e, f, u, info


def test_reference_solve_matches_converged_ewald(esp):
    s = inputs.spce_water(1000, seed=11)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    e, f, u, _ = solve(esp, s, 1e-10, r_c=1.0, precision=esp.ESP_FP64)
    assert metrics.relative_rms_force_error(f, ref["forces"]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])


def test_large_water_box_at_full_size(esp):
    s = inputs.spce_water(1_000_000, seed=2505)
    e, f, u, info = solve(esp, s, 1e-5, r_c=1.0)
    assert info["P"] == 8 and info["n_f"] == 144
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(u))
    # sampled atoms against the oracle at the plan's parameters
    idx = np.sort(np.random.default_rng(3).choice(s.n, size=64, replace=False))
    p = oesp.ESPParams(1e-5, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"])
    ref = oesp.esp(s.pos, s.q, s.L, p, idx)
    assert metrics.relative_rms_force_error(f[idx], ref["forces"]) <= FP32_PARITY
    assert float(np.sqrt(np.sum((u[idx] - ref["potential"]) ** 2) / np.sum(ref["potential"] ** 2))) <= FP32_PARITY
    # every atom against the eps = 1e-10 reference
    e_ref, f_ref, _, _ = solve(esp, s, 1e-10, r_c=1.0, precision=esp.ESP_FP64)
    delta = metrics.relative_rms_force_error(f, f_ref)
    assert delta <= 1e-5, delta
    assert abs(e - e_ref) <= 1e-5 * abs(e_ref)


def test_batched_workload_at_full_size(esp):
    """The 64-box electrolyte batch of the benchmark (3.24e6 atoms, sizes
    log-uniform in [3e3, 2e5], seed 9727, one launch per kernel, graph
    replay): sampled atoms of the smallest, a middle and the largest system
    against the oracle at that system's batch parameters (FP32 parity bound),
    and every system's force error over all atoms against an FP64 batch at
    eps = 1e-10 parameters within the tolerance."""
    sizes = inputs.batch_sizes(64, 3000, 200_000, seed=9727)
    systems = inputs.electrolyte_batch(sizes, seed=9727)
    pos, q = inputs.concat(systems)
    with esp.Batch([s.L for s in systems], [s.n for s in systems], 1e-4, r_c=1.0) as b:
        b.set_charges(q)
        for _ in range(2):                                  # direct run, then the captured graph
            e, f, u = b.compute(pos)
        infos = [b.info(i) for i in range(len(systems))]
        off = b.offsets
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(e))
    order = np.argsort(sizes)
    rng = np.random.default_rng(5)
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        s, info = systems[i], infos[i]
        idx = np.sort(rng.choice(s.n, size=min(48, s.n), replace=False))
        p = oesp.ESPParams(1e-4, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"])
        ref = oesp.esp(s.pos, s.q, s.L, p, idx)
        fs = f[off[i]:off[i + 1]][idx]
        us = u[off[i]:off[i + 1]][idx]
        assert metrics.relative_rms_force_error(fs, ref["forces"]) <= FP32_PARITY, i
        assert float(np.sqrt(np.sum((us - ref["potential"]) ** 2) / np.sum(ref["potential"] ** 2))) <= FP32_PARITY
    with esp.Batch([s.L for s in systems], [s.n for s in systems], 1e-10, r_c=1.0, precision=esp.ESP_FP64) as rb:
        rb.set_charges(q)
        _, f_ref, _ = rb.compute(pos)
    for i in range(len(systems)):
        sl = slice(off[i], off[i + 1])
        assert metrics.relative_rms_force_error(f[sl], f_ref[sl]) <= 1e-4, i
