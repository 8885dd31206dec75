"""Exclusions (esp_set_exclusions) on the GPU against the oracle: ESP over
all pairs (oracle/esp.py) minus the direct interaction of the excluded
pairs (oracle/md.py, exclusion_correction), at the plan's parameters.

The errors of the GPU path come from the uncorrected sums, whose
intramolecular terms are several times larger than what remains, so each
bound is the plain parity bound (FP64 1e-9 forces and potentials, 1e-10
energy; FP32 5e-6) times the ratio of the uncorrected to the corrected
magnitude, with a factor 2 of margin.

Also: the esp_step graph replay with exclusions, clearing them, a
triclinic cell, and the argument checks. Collected last (test_zz_*): the
newest GPU path.
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import md
from oracle import triclinic as tr
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def params_of(eps, info):
    return oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"])


def gpu(esp, L, s, eps, pairs, **opts):
    with esp.Plan(L, s.n, eps, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        esp.esp_set_exclusions(p.handle, pairs)
        e, f, u = p.compute()
        return e, f, u, p.info


@pytest.mark.parametrize("prec,bound", [(1, 1e-9), (0, 5e-6)], ids=["fp64", "fp32"])
def test_exclusions_match_the_oracle(esp, prec, bound):
    s = inputs.spce_water(300, seed=21)
    pairs = md.exclusion_pairs(s.n)
    eps = 1e-5
    e, f, u, info = gpu(esp, s.L, s, eps, pairs, r_c=1.0, precision=prec)
    ref = oesp.esp(s.pos, s.q, s.L, params_of(eps, info))
    ex, ux, fx = md.exclusion_correction(s.pos, s.q, s.L, pairs)
    F, U, E = ref["forces"] + fx, ref["potential"] + ux, ref["energy"] + ex
    ratio_f = np.linalg.norm(ref["forces"]) / np.linalg.norm(F)
    ratio_u = np.linalg.norm(ref["potential"]) / np.linalg.norm(U)
    assert rel_rms(f, F) <= 2 * bound * ratio_f
    assert rel_rms(u, U) <= 2 * bound * ratio_u
    e_scale = max(abs(ref["energy"]), 0.5 * float(np.sum(s.q * ref["self_term"])) if prec == 0 else 0.0)
    assert abs(e - E) <= 2 * (bound if prec == 0 else 1e-10) * abs(e_scale)


def test_graph_replay_and_clearing(esp):
    s = inputs.spce_water(400, seed=22)
    pairs = md.exclusion_pairs(s.n)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e0, f0, u0 = p.compute()                          # no exclusions
        esp.esp_set_exclusions(p.handle, pairs)
        e1, f1, u1 = p.compute()
        e, f, u = np.zeros(1), np.zeros((s.n, 3)), np.zeros(s.n)
        for _ in range(3):                                # direct run, capture, replay
            esp.esp_step(p.handle, s.pos, e, f, u)
            assert rel_rms(f, f1) <= 1e-5 and abs(e[0] - e1) <= 1e-5 * abs(e0)
        esp.esp_set_exclusions(p.handle, None)
        e2, f2, _ = p.compute()
    assert rel_rms(f2, f0) <= 1e-6 and abs(e2 - e0) <= 1e-6 * abs(e0)
    # the removed direct terms, by the oracle's formula
    ex, _, fx = md.exclusion_correction(s.pos, s.q, s.L, pairs)
    assert abs((e1 - e0) - ex) <= 1e-5 * abs(e0)
    assert rel_rms(f1 - f0, fx) <= 1e-4


def test_triclinic_cell_with_exclusions(esp):
    s = inputs.spce_water_cell(300, seed=23)
    pairs = md.exclusion_pairs(s.n)
    eps, r_c = 1e-4, 0.9
    with esp.Plan(s.H, s.n, eps, r_c=r_c) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        esp.esp_set_exclusions(p.handle, pairs)
        e, f, u = p.compute()
        info = p.info
    prm = params_of(eps, info)
    ref = tr.esp(s.pos, s.q, s.H, prm.split(), prm.si_window(), info["n_f"], info["r_c"])
    # molecules are stored whole (not wrapped), so the intramolecular vectors
    # need no image
    ex, ux, fx = md.exclusion_correction(s.pos, s.q, 1e9, pairs)
    F, E = ref["forces"] + fx, ref["energy"] + ex
    ratio_f = np.linalg.norm(ref["forces"]) / np.linalg.norm(F)
    assert rel_rms(f, F) <= 2 * 5e-6 * ratio_f
    chi0 = prm.split().chi0
    e_self = 0.5 * float(np.sum(s.q * s.q)) * chi0 / (4 * math.pi * info["r_c"])
    assert abs(e - E) <= 2 * 5e-6 * max(abs(ref["energy"]), e_self)


def test_exclusion_arguments(esp):
    s = inputs.spce_water(50, seed=24)                       # L = 1.14 nm
    with esp.Plan(s.L, s.n, 1e-4, r_c=0.5) as p:
        # out of range, negative, self pair, and a pair listed twice (either order)
        for bad in ([[0, s.n]], [[-1, 2]], [[3, 3]], [[1, 2], [5, 6], [2, 1]], [[4, 5], [4, 5]]):
            with pytest.raises(esp.EspError) as exc:
                esp.esp_set_exclusions(p.handle, np.array(bad))
            assert exc.value.status == 1
    with esp.Plan(s.L, s.n, 1e-4, r_c=0.5, virial=1) as p:
        with pytest.raises(esp.EspError) as exc:
            esp.esp_set_exclusions(p.handle, md.exclusion_pairs(s.n))
        assert exc.value.status == 10
