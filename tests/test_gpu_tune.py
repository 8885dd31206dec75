"""Autotuner (esp_autotune): the chosen shapes are valid plan options, give
the same results as the planner's defaults (within the FP32 parity bound),
and a second call is answered from the per-process cache."""
import time

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


def solve(esp, s, eps, **opts):
    with esp.Plan(s.L, s.n, eps, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        return p.compute()


def test_autotune_picks_valid_equivalent_shapes(esp):
    s = inputs.electrolyte(20000, seed=400)
    chosen, ms = esp.esp_autotune(s.L, 1e-4, s.pos, s.q, reps=3, r_c=1.0)
    assert ms > 0
    assert chosen["cell_reach"] in (2, 3) and chosen["near_variant"] in (3, 4)
    assert 1 <= chosen["brick_cells"] <= 8 and chosen["r_c"] == 1.0
    e0, f0, u0 = solve(esp, s, 1e-4, r_c=1.0)
    e1, f1, u1 = solve(esp, s, 1e-4, r_c=1.0, cell_reach=chosen["cell_reach"],
                       near_variant=chosen["near_variant"], brick_cells=chosen["brick_cells"])
    assert np.sqrt(np.sum((f1 - f0) ** 2) / np.sum(f0 ** 2)) <= FP32_PARITY
    assert abs(e1 - e0) <= FP32_PARITY * abs(e0)
    t0 = time.perf_counter()
    again, ms2 = esp.esp_autotune(s.L, 1e-4, s.pos, s.q, reps=3, r_c=1.0)
    assert time.perf_counter() - t0 < 0.05
    assert again == chosen and ms2 == ms


def test_autotune_keeps_fixed_options(esp):
    s = inputs.electrolyte(6000, seed=401)
    chosen, _ = esp.esp_autotune(s.L, 1e-3, s.pos, s.q, reps=2, r_c=1.0, cell_reach=2, near_variant=4)
    assert chosen["cell_reach"] == 2 and chosen["near_variant"] == 4
