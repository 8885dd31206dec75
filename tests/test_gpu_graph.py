"""Graph replay of a single plan's compute.

After its first direct run, a plan replays its compute as a captured CUDA
graph for the same output pointers and re-captures when they change. Every
replayed result must equal a fresh plan's direct result for the same
positions (up to the FP32 atomic summation order), with new positions each
step, host outputs, and device outputs alternating between two buffers.
"""
import numpy as np
import pytest

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


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def fresh(esp, s, pos):
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        p.set_positions(pos)
        return p.compute()


def test_host_outputs_replayed(esp):
    s = inputs.spce_water(2000, seed=41)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        for k in range(5):                       # direct, capture, replays
            pos = inputs.perturb(s, 0.02, seed=400 + k).pos
            p.set_positions(pos)
            e, f, u = p.compute()
            e0, f0, u0 = fresh(esp, s, pos)
            assert rel_rms(f, f0) <= FP32_PARITY
            assert rel_rms(u, u0) <= FP32_PARITY
            assert abs(e - e0) <= FP32_PARITY * abs(e0)


def test_device_outputs_alternating_buffers(esp):
    import torch
    dev = torch.device("cuda:0")
    s = inputs.electrolyte(6000, seed=42)
    h = esp.esp_plan(s.L, s.n, 1e-4, r_c=1.0)
    try:
        esp.esp_set_charges(h, torch.tensor(s.q, device=dev))
        bufs = [(torch.zeros(1, dtype=torch.float64, device=dev), torch.zeros((s.n, 3), dtype=torch.float64, device=dev),
                 torch.zeros(s.n, dtype=torch.float64, device=dev)) for _ in range(2)]
        for k in range(7):                       # keys change every step: re-captures, then direct runs
            pos = inputs.perturb(s, 0.02, seed=500 + k).pos
            e, f, u = bufs[k % 2]
            esp.esp_set_positions(h, torch.tensor(pos, device=dev))
            esp.esp_compute(h, e, f, u)
            torch.cuda.synchronize()
            e0, f0, u0 = fresh(esp, s, pos)
            assert rel_rms(f.cpu().numpy(), f0) <= FP32_PARITY
            assert rel_rms(u.cpu().numpy(), u0) <= FP32_PARITY
            assert abs(float(e.cpu()[0]) - e0) <= FP32_PARITY * abs(e0)
    finally:
        esp.esp_destroy(h)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energy_only_matches_full_compute(esp, prec):
    """Forces and potential NULL: the energy alone, from the spectral sum of
    the scale kernel and the local part (no inverse FFT, no gather)."""
    import torch
    dev = torch.device("cuda:0")
    precision = esp.ESP_FP32 if prec == "fp32" else esp.ESP_FP64
    s = inputs.spce_water(1500, seed=43)
    h = esp.esp_plan(s.L, s.n, 1e-4, r_c=1.0, precision=precision)
    try:
        esp.esp_set_charges(h, torch.tensor(s.q, device=dev))
        esp.esp_set_positions(h, torch.tensor(s.pos, device=dev))
        e_full = torch.zeros(1, dtype=torch.float64, device=dev)
        f = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
        esp.esp_compute(h, e_full, f, None)
        for _ in range(3):                       # direct, captured, replayed
            e = torch.zeros(1, dtype=torch.float64, device=dev)
            esp.esp_compute(h, e, None, None)
            torch.cuda.synchronize()
            bound = 1e-6 if prec == "fp32" else 1e-13
            assert abs(float(e.cpu()[0]) - float(e_full.cpu()[0])) <= bound * abs(float(e_full.cpu()[0]))
    finally:
        esp.esp_destroy(h)


def test_step_matches_set_positions_and_compute(esp):
    """esp_step (positions in, compute, results out in one call; sort and
    compute replayed as one graph) equals fresh plans, host and device."""
    import torch
    dev = torch.device("cuda:0")
    s = inputs.spce_water(2000, seed=44)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        for k in range(4):                       # direct run, capture, replays
            pos = inputs.perturb(s, 0.02, seed=600 + k).pos
            e = np.zeros(1)
            f = np.zeros((s.n, 3))
            u = np.zeros(s.n)
            esp.esp_step(p.handle, np.ascontiguousarray(pos), e, f, u)
            e0, f0, u0 = fresh(esp, s, pos)
            assert rel_rms(f, f0) <= FP32_PARITY and rel_rms(u, u0) <= FP32_PARITY
            assert abs(e[0] - e0) <= FP32_PARITY * abs(e0)
        x = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
        ed = torch.zeros(1, dtype=torch.float64, device=dev)
        fd = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
        for k in range(3):                       # device buffers, the same source pointer
            pos = inputs.perturb(s, 0.02, seed=700 + k).pos
            x.copy_(torch.tensor(pos))
            esp.esp_step(p.handle, x, ed, fd, None)
            torch.cuda.synchronize()
            e0, f0, _ = fresh(esp, s, pos)
            assert rel_rms(fd.cpu().numpy(), f0) <= FP32_PARITY
            assert abs(float(ed.cpu()[0]) - e0) <= FP32_PARITY * abs(e0)
        bad = s.pos.copy()
        bad[3, 0] = np.inf
        with pytest.raises(esp.EspError) as exc:
            esp.esp_step(p.handle, bad, np.zeros(1), np.zeros((s.n, 3)), None)
        assert exc.value.status == 4
