"""Batches of independent systems through esp_batch_* against single plans
and the oracle.

Every system of a batch must give what a single plan gives for that system
at the batch's parameters (same P, c1, n_f, r_c): the batch changes only how
the work is laid out (concatenated atoms and cell lists, pooled grids,
batched FFTs, a replayed CUDA graph), not the arithmetic of any system. The
graph is captured on the second call, so three calls in a row with moved
atoms check that replays read the new positions.
"""
import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald, metrics
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_PARITY = 5e-6          # the FP32 bound of the single-plan parity tests
SIZES = [3000, 4600, 3300, 9000, 3100, 5200]


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def single(esp, s, eps, info, precision):
    with esp.Plan(s.L, s.n, eps, r_c=info["r_c"], P=info["P"], n_f=info["n_f"], c=info["c"],
                  c1=info["c1"], precision=precision) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        return p.compute()


def split(arr, offsets, s):
    return arr[offsets[s]:offsets[s + 1]]


@pytest.mark.parametrize("precision,bound", [(0, FP32_PARITY), (1, 1e-10)])
def test_batch_matches_single_plans(esp, precision, bound):
    systems = inputs.electrolyte_batch(SIZES, seed=40)
    eps = 1e-4
    with esp.Batch([s.L for s in systems], [s.n for s in systems], eps, r_c=1.0,
                   precision=precision) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        for step in range(3):           # direct run, capture + replay, replay
            moved = [inputs.perturb(s, 0.02, seed=100 * step + i) for i, s in enumerate(systems)]
            pos, _ = inputs.concat(moved)
            e, f, u = b.compute(pos)
            for i, s in enumerate(moved):
                info = b.info(i)
                e1, f1, u1 = single(esp, s, eps, info, precision)
                fs, us = split(f, b.offsets, i), split(u, b.offsets, i)
                assert rel_rms(fs, f1) <= bound, (step, i)
                assert rel_rms(us, u1) <= bound, (step, i)
                assert abs(e[i] - e1) <= bound * max(abs(e1), 1.0), (step, i)


def test_batch_fp64_matches_oracle(esp):
    systems = inputs.electrolyte_batch([3000, 3500], seed=50)
    eps = 1e-5
    with esp.Batch([s.L for s in systems], [s.n for s in systems], eps, r_c=1.0,
                   precision=esp.ESP_FP64) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        e, f, u = b.compute(pos)
        for i, s in enumerate(systems):
            info = b.info(i)
            p = oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"])
            ref = oesp.esp(s.pos, s.q, s.L, p)
            assert metrics.relative_rms_force_error(split(f, b.offsets, i), ref["forces"]) <= 1e-9
            assert rel_rms(split(u, b.offsets, i), ref["potential"]) <= 1e-9
            assert abs(e[i] - ref["energy"]) <= 1e-10 * abs(ref["energy"])


def test_batch_ik_fp64_matches_oracle(esp):
    """The ik force method on a batch: two grid-size buckets, FP64 against
    the oracle at each system's parameters."""
    systems = inputs.electrolyte_batch([3000, 9000], seed=55)
    eps = 1e-4
    with esp.Batch([s.L for s in systems], [s.n for s in systems], eps, r_c=1.0,
                   precision=esp.ESP_FP64, diff=esp.ESP_DIFF_IK) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        for _ in range(2):               # direct run, then the captured graph
            e, f, u = b.compute(pos)
        for i, s in enumerate(systems):
            info = b.info(i)
            assert info["diff"] == esp.ESP_DIFF_IK
            p = oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"], diff="ik")
            ref = oesp.esp(s.pos, s.q, s.L, p)
            assert metrics.relative_rms_force_error(split(f, b.offsets, i), ref["forces"]) <= 1e-9
            assert rel_rms(split(u, b.offsets, i), ref["potential"]) <= 1e-9


def test_batch_fp32_within_tolerance_of_ewald(esp):
    systems = inputs.electrolyte_batch([3000, 4000, 3200], seed=60)
    refs = [ewald.ewald(s.pos, s.q, s.L, acc=1e-14) for s in systems]
    for eps in (1e-3, 1e-4):
        with esp.Batch([s.L for s in systems], [s.n for s in systems], eps, r_c=1.0) as b:
            pos, q = inputs.concat(systems)
            b.set_charges(q)
            e, f, u = b.compute(pos)
            for i, ref in enumerate(refs):
                delta = metrics.relative_rms_force_error(split(f, b.offsets, i), ref["forces"])
                assert delta <= eps, (eps, i, delta)


def test_batch_device_buffers_match_host(esp):
    import torch
    systems = inputs.electrolyte_batch([3000, 6000, 3400], seed=70)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    with esp.Batch([s.L for s in systems], [s.n for s in systems], 1e-4, r_c=1.0,
                   stream=stream.cuda_stream) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        e_h, f_h, u_h = b.compute(pos)
        n = pos.shape[0]
        with torch.cuda.stream(stream):
            x = torch.tensor(pos, device=dev)
            e = torch.zeros(len(systems), dtype=torch.float64, device=dev)
            f = torch.zeros((n, 3), dtype=torch.float64, device=dev)
            u = torch.zeros(n, dtype=torch.float64, device=dev)
        stream.synchronize()
        for _ in range(2):
            esp.esp_batch_compute(b.handle, x, e, f, u)
            esp.esp_batch_synchronize(b.handle)
        assert rel_rms(f.cpu().numpy(), f_h) <= 1e-6
        assert rel_rms(u.cpu().numpy(), u_h) <= 1e-6
        assert np.allclose(e.cpu().numpy(), e_h, rtol=1e-6, atol=0)


def test_batch_rejects_non_neutral_system(esp):
    systems = inputs.electrolyte_batch([3000, 3000], seed=80)
    pos, q = inputs.concat(systems)
    q = q.copy()
    q[systems[0].n + 5] += 1.0                     # system 1 is not neutral
    with esp.Batch([s.L for s in systems], [s.n for s in systems], 1e-4, r_c=1.0,
                   allow_background=0) as b:
        with pytest.raises(esp.EspError) as exc:
            b.set_charges(q)
        assert exc.value.status == 3
        assert "system 1" in esp.esp_last_error()


def test_batch_phase_timing(esp):
    systems = inputs.electrolyte_batch([3000, 5000], seed=90)
    with esp.Batch([s.L for s in systems], [s.n for s in systems], 1e-4, r_c=1.0) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        e0, f0, _ = b.compute(pos)
        esp.esp_batch_set_timing(b.handle, 2)
        e1, f1, _ = b.compute(pos)
        t = esp.esp_batch_phase_times(b.handle)
        assert t["total"] > 0 and t["near"] > 0 and t["spread"] > 0
        assert rel_rms(f1, f0) <= 1e-6
        esp.esp_batch_set_timing(b.handle, 0)
        e2, f2, _ = b.compute(pos)                 # back on the graph
        assert rel_rms(f2, f0) <= 1e-6
