"""Pins for oracle.esp (plain CPU ESP) and oracle.params (the paper's rules).

The exact result is classical Ewald (itself pinned in test_oracle_ewald.py);
ESP must reach it within the requested tolerance (Eq. Deltadef), satisfy the
exact discrete energy identity, converge to Ewald when the Gaussian split is
used with generous parameters, and respect the invariances of Eq. task.
"""
import math

import numpy as np
import pytest

from golden_io import rows
from oracle import esp, ewald, metrics, params, pswf
from paper_2505_09727_gb300 import inputs


@pytest.fixture(scope="module")
def water():
    s = inputs.spce_water(1000, seed=11)
    return s, ewald.ewald(s.pos, s.q, s.L, acc=1e-14)


@pytest.fixture(scope="module")
def ions():
    s = inputs.uniform_charges(300, 5.0, 7)
    return s, ewald.ewald(s.pos, s.q, s.L)


def planned(eps, L, r_c, kind="pswf"):
    p = params.plan(eps, L, r_c, kind)
    return esp.ESPParams(eps, r_c, p["P"], p["n_f"], p["c"], p["c1"], kind, p["alpha"])


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_water_force_error_within_tolerance(water, eps):
    s, ref = water
    r = esp.esp(s.pos, s.q, s.L, planned(eps, s.L, 1.0))
    delta = metrics.relative_rms_force_error(r["forces"], ref["forces"])
    assert delta <= eps, delta
    # energy and potentials at the same order
    assert abs(r["energy"] - ref["energy"]) <= eps * abs(ref["energy"])
    du = np.sqrt(np.mean((r["potential"] - ref["potential"]) ** 2) / np.mean(ref["potential"] ** 2))
    assert du <= eps


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_ions_force_error_within_tolerance(ions, eps):
    s, ref = ions
    r = esp.esp(s.pos, s.q, s.L, planned(eps, s.L, 1.2))
    assert metrics.relative_rms_force_error(r["forces"], ref["forces"]) <= eps


def test_discrete_energy_identity(ions):
    # sum_i q_i u~_i = sum_k p_k |bh_k|^2 exactly (any parameters)
    s, _ = ions
    r = esp.esp(s.pos, s.q, s.L, esp.ESPParams(1e-3, 1.2, 5, 12))
    lhs = 0.5 * float(np.dot(s.q, r["spectral_potential"]))
    assert abs(lhs - r["fourier_energy"]) < 1e-13 * abs(lhs)


def test_gaussian_split_converges_to_ewald(ions):
    # Gaussian split with alpha = 30 (erfc(sqrt(30)) ~ 2e-14), a wide stencil and a
    # fine grid: the five-step method reproduces Ewald with g = sqrt(alpha)/r_c.
    s, ref = ions
    alpha, r_c = 30.0, 2.2
    n_f = params.round_grid(2.0 * math.sqrt(alpha * 32.0) * s.L / (math.pi * r_c))
    p = esp.ESPParams(1e-13, r_c, 16, n_f, c=12.0, c1=36.0, kind="gauss", alpha=alpha)
    r = esp.esp(s.pos, s.q, s.L, p)
    assert metrics.relative_rms_force_error(r["forces"], ref["forces"]) < 1e-9
    assert abs(r["energy"] - ref["energy"]) < 1e-10 * abs(ref["energy"])


def test_nacl_madelung_through_esp():
    s = inputs.nacl_lattice(4)          # 512 ions, L = 4, d = 0.5
    (m, *_), = rows("nacl_madelung.txt")
    e_closed = -(s.n / 2) * float(m) / (4 * np.pi * 0.5)
    r = esp.esp(s.pos, s.q, s.L, planned(1e-10, s.L, 1.9))
    assert abs(r["energy"] - e_closed) < 1e-9 * abs(e_closed)
    assert np.max(np.abs(r["forces"])) < 1e-9


def test_invariances(ions):
    s, ref = ions
    p = planned(1e-4, s.L, 1.2)
    r = esp.esp(s.pos, s.q, s.L, p)
    # translation: ESP is translation invariant to within its tolerance
    t = esp.esp(s.pos + np.array([0.123, 1.7, -0.9]), s.q, s.L, p)
    assert metrics.relative_rms_force_error(t["forces"], r["forces"]) < 1e-4
    # linearity (exact up to rounding)
    d = esp.esp(s.pos, 2 * s.q, s.L, p)
    assert abs(d["energy"] - 4 * r["energy"]) < 1e-12 * abs(r["energy"])
    assert np.max(np.abs(d["forces"] - 4 * r["forces"])) < 1e-11 * np.max(np.abs(r["forces"]))
    # net force is O(eps) of the force scale, not exactly zero (AD forces)
    rms = np.sqrt(np.sum(ref["forces"] ** 2))
    assert np.linalg.norm(r["forces"].sum(axis=0)) < 1e-4 * rms


def test_sampled_targets_match_full(ions):
    s, _ = ions
    p = planned(1e-4, s.L, 1.2)
    full = esp.esp(s.pos, s.q, s.L, p)
    idx = np.array([3, 99, 298])
    part = esp.esp(s.pos, s.q, s.L, p, targets=idx)
    assert np.max(np.abs(part["forces"] - full["forces"][idx])) < 1e-13
    assert np.max(np.abs(part["potential"] - full["potential"][idx])) < 1e-13


def test_non_neutral_background_matches_ewald():
    s = inputs.uniform_charges(100, 5.0, 3)
    q = s.q.copy()
    q[:3] += 0.4
    ref = ewald.ewald(s.pos, q, s.L)
    r = esp.esp(s.pos, q, s.L, planned(1e-6, s.L, 1.5))
    assert abs(r["energy"] - ref["energy"]) < 1e-5 * abs(ref["energy"])
    assert np.max(np.abs(r["potential"] - ref["potential"])) < 1e-5 * np.max(np.abs(ref["potential"]))


# ----------------------------------------------------------------- params
def test_table1_grid_spacing_rule():
    # Eq. pswfparameters with Table 2's c reproduces Table 1's ESP spacing at 1e-5.
    for name, L, eps, r_c, P, h in rows("table1_esp_rows.txt"):
        L, eps, r_c, P, h = float(L), float(eps), float(r_c), int(P), float(h)
        c = pswf.c_from_tolerance(eps)
        n_f = math.ceil(params.pswf_grid_min(c, L, r_c))
        assert abs(L / n_f - h) <= 0.0051, (name, L / n_f)
        assert params.stencil_width(eps) == P


def test_table2_stencil_widths():
    for eps, _a, _c, P, _r in rows("table2_optimal_values.txt"):
        assert params.stencil_width(float(eps)) == int(P)


def test_round_grid():
    for n in (11.2, 14.0, 57.3, 143.9, 159.0):
        m = params.round_grid(n)
        assert m >= n and m % 2 == 0 and params.is_smooth(m)
        assert all(not (k % 2 == 0 and params.is_smooth(k)) for k in range(math.ceil(n), m))


def test_gauss_grid_rule_and_mode_ratio():
    # Eq. cemparameters vs Eq. pswfparameters: the Gaussian needs more modes,
    # 8x in the small-eps limit and ~3.6x at 1e-4 (Fig. 3 caption).
    L, r_c = 14.413, 1.0
    assert params.gauss_grid_min(1e-4, L, r_c) == 2 * math.ceil(math.log(1e4) * L / (math.pi * r_c))
    c = pswf.c_from_tolerance(1e-4)
    ratio = (params.gauss_grid_min(1e-4, L, r_c) / params.pswf_grid_min(c, L, r_c)) ** 3
    assert 3.3 < ratio < 4.0
    # the ratio (2 ln(1/eps) / c)^3 grows toward 8 as eps -> 0
    ratios = [(2 * math.log(1 / e) / pswf.c_from_tolerance(e)) ** 3 for e in (1e-4, 1e-8, 1e-11, 1e-14)]
    assert all(a < b < 8.0 for a, b in zip(ratios, ratios[1:]))


# ------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(ions, monkeypatch):
    """Each plausible slip in the oracle fails one of the checks above."""
    s, ref = ions
    p = planned(1e-4, s.L, 1.2)

    def delta(res):
        return metrics.relative_rms_force_error(res["forces"], ref["forces"])

    def du(res):
        return np.sqrt(np.mean((res["potential"] - ref["potential"]) ** 2) / np.mean(ref["potential"] ** 2))

    good = esp.esp(s.pos, s.q, s.L, p)
    assert delta(good) < 1e-4 and du(good) < 1e-4

    # (a) forgetting the self term shifts every potential
    monkeypatch.setattr(pswf.PSWFSplit, "chi0", property(lambda self: 0.0))
    assert du(esp.esp(s.pos, s.q, s.L, p)) > 1e-2
    monkeypatch.undo()

    # (b) the wrong FFT normalisation (dividing by N_f) breaks the spectral part
    orig = np.fft.ifftn
    monkeypatch.setattr(np.fft, "ifftn", lambda a: orig(a) / a.size)
    assert delta(esp.esp(s.pos, s.q, s.L, p)) > 1e-2
    monkeypatch.undo()

    # (c) deconvolving by Phi instead of Phi^2 (Eq. pk)
    orig_inf = esp.influence

    def once(L, n_f, r_c, split, window):
        k = np.fft.fftfreq(n_f, d=1.0 / n_f)
        ph = window.Phi(2 * math.pi * k / n_f)
        return orig_inf(L, n_f, r_c, split, window) * np.abs(ph[:, None, None] * ph[None, :, None] * ph[None, None, :])
    monkeypatch.setattr(esp, "influence", once)
    assert delta(esp.esp(s.pos, s.q, s.L, p)) > 1e-2
    monkeypatch.undo()

    # (d) a sign slip in the local force
    orig_near = esp.near_field
    monkeypatch.setattr(esp, "near_field", lambda *a: (lambda u, f: (u, -f))(*orig_near(*a)))
    assert delta(esp.esp(s.pos, s.q, s.L, p)) > 1e-2
