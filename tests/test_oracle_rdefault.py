"""Pin of the "Default" comparator and of the ESP planner against Table 2.

Table 2's last row, R_default, is the ratio of the total number of Fourier
grid points the default PME needs (Gaussian split of Eq. cem with
alpha_G = ln(1/eps), cardinal B-spline window of order P = 5, the packages'
default, n_f raised until the force error meets eps) to the number ESP needs
at the same error. This test repeats that experiment with the oracle on a
synthetic SPC/E-shaped water box: for every tolerance of Table 2 it finds
the smallest even n_f at which the B-spline comparator's relative RMS force
error (Eq. Deltadef, against the ESP solve at eps = 1e-10 parameters, which
the Ewald pins hold to 1e-9) is at most eps, and sets its cube against
ESP's Eq. pswfparameters grid c L / (pi r_c). The measured ratio must land
within a factor 1.5 of the printed R_default at every tolerance and grow
with the precision as the printed row does; a wrong window order (P = 4),
shape alpha, window transform or error metric moves it by several times.

The same measurement pins the ESP planner (the relative aliasing estimate of
Eq. errorformula and its acceptance): its grid meets eps and is no larger
than 1.25 times the Eq. pswfparameters value.
"""
import math

import numpy as np
import pytest

from golden_io import rows
from oracle import bspline, esp, metrics, params, pswf
from paper_2505_09727_gb300 import inputs

R_C = 0.5


@pytest.fixture(scope="module")
def water():
    s = inputs.spce_water(2000, seed=5)            # 6000 atoms, L = 3.91 nm, L / r_c = 7.8
    c = pswf.c_from_tolerance(1e-10)
    ref_p = esp.ESPParams(1e-10, R_C, 13, params.round_grid(1.25 * c * s.L / (math.pi * R_C)))
    return s, esp.esp(s.pos, s.q, s.L, ref_p)["forces"]


def forces(s, split, window, n_f, near):
    _, grad, _ = esp.far_field(s.pos, s.q, s.L, n_f, R_C, split, window, np.arange(s.n))
    return -s.q[:, None] * grad + near


def smallest_grid(s, f_ref, eps, split, window, n_lo):
    """Smallest even n_f >= n_lo with Delta <= eps (Delta falls with n_f)."""
    _, near = esp.near_field(s.pos, s.q, s.L, R_C, split, np.arange(s.n))

    def ok(n):
        return metrics.relative_rms_force_error(forces(s, split, window, n, near), f_ref) <= eps

    lo, hi = n_lo, n_lo
    while not ok(hi):
        lo, hi = hi + 2, 2 * hi
    while lo < hi:                                  # invariant: ok(hi), not ok(n) for n < lo
        mid = 2 * ((lo + hi) // 4)
        if mid < lo:
            mid = lo
        if ok(mid):
            hi = mid
        else:
            lo = mid + 2
    return hi


def test_default_comparator_reproduces_r_default(water):
    s, f_ref = water
    table = {float(r[0]): (float(r[2]), float(r[4])) for r in rows("table2_optimal_values.txt")}
    measured = []
    for eps in sorted(table, reverse=True):
        c, r_default = table[eps]
        alpha = math.log(1.0 / eps)
        n_def = smallest_grid(s, f_ref, eps, pswf.GaussianSplit(alpha), bspline.BSplineWindow(5),
                              params.gauss_grid_min(eps, s.L, R_C))
        R = (n_def / params.pswf_grid_min(c, s.L, R_C)) ** 3
        measured.append(R)
        assert r_default / 1.5 <= R <= r_default * 1.5, (eps, R, r_default)
    assert all(b > a for a, b in zip(measured, measured[1:]))


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_esp_planner_grid_meets_the_tolerance_without_waste(water, eps):
    s, f_ref = water
    pl = params.plan(eps, s.L, R_C)
    p = esp.ESPParams(eps, R_C, pl["P"], pl["n_f"], c=pl["c"], c1=pl["c1"])
    delta = metrics.relative_rms_force_error(esp.esp(s.pos, s.q, s.L, p)["forces"], f_ref)
    assert delta <= eps
    assert pl["n_f"] <= 1.25 * params.pswf_grid_min(pl["c"], s.L, R_C)


def test_comparator_planner_grid_meets_the_tolerance(water):
    s, f_ref = water
    for eps in (1e-3, 1e-4, 1e-5):
        pl = params.plan_bspline(eps, s.L, R_C)
        p = esp.ESPParams(eps, R_C, pl["P"], pl["n_f"], kind="gauss", alpha=pl["alpha"], window="bspline")
        delta = metrics.relative_rms_force_error(esp.esp(s.pos, s.q, s.L, p)["forces"], f_ref)
        assert delta <= eps, (eps, delta)
