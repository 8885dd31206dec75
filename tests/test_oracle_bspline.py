"""Pins for oracle.bspline (the cardinal B-spline SI window of the Default
comparator) and for the comparator's plan: Gaussian split, B-spline window,
grid raised until the aliasing estimate meets the tolerance.

The window is pinned by facts of the B-spline that do not depend on the
implementation: two independent constructions agree, the integer
translates form a partition of unity, the closed-form transform equals the
numerical transform of the function, the derivative equals a finite
difference; the comparator's solution reaches classical Ewald within the
tolerance."""
import math

import numpy as np
import pytest

from oracle import bspline, esp, ewald, metrics, params
from paper_2505_09727_gb300 import inputs

ORDERS = [2, 3, 4, 5, 6, 7, 8]


@pytest.mark.parametrize("P", ORDERS)
def test_two_constructions_agree(P):
    x = np.linspace(-0.5, P + 0.5, 2001)
    a = bspline.cardinal(P, x)
    b = bspline.cardinal_recursive(P, x)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("P", ORDERS)
def test_partition_of_unity_on_the_stencil(P):
    w = bspline.BSplineWindow(P)
    t = np.random.default_rng(P).uniform(-50, 50, 500)
    l0 = np.ceil(t - 0.5 * P)
    total = sum(w.phi(t - (l0 + a)) for a in range(P))
    assert np.max(np.abs(total - 1.0)) < 1e-12
    # and the derivative weights sum to zero
    dtot = sum(w.dphi(t - (l0 + a)) for a in range(P))
    assert np.max(np.abs(dtot)) < 1e-11


@pytest.mark.parametrize("P", [4, 6, 8])
def test_transform_matches_numerical_transform(P):
    w = bspline.BSplineWindow(P)
    gx, gw = np.polynomial.legendre.leggauss(40)
    theta = np.linspace(0.0, 3.0 * math.pi, 37)
    num = np.zeros_like(theta)
    for piece in range(P):                       # exact per polynomial piece
        a, b = -0.5 * P + piece, -0.5 * P + piece + 1
        t = 0.5 * (b - a) * gx + 0.5 * (a + b)
        num += 0.5 * (b - a) * (np.cos(np.outer(theta, t)) @ (gw * w.phi(t)))
    assert np.max(np.abs(num - w.Phi(theta))) < 1e-13


@pytest.mark.parametrize("P", [3, 4, 6])
def test_derivative_matches_finite_difference(P):
    w = bspline.BSplineWindow(P)
    t = np.random.default_rng(1).uniform(-0.5 * P + 0.01, 0.5 * P - 0.01, 200)
    d = 1e-6
    fd = (w.phi(t + d) - w.phi(t - d)) / (2 * d)
    assert np.max(np.abs(fd - w.dphi(t))) < 1e-7


def test_comparator_needs_a_finer_grid_than_esp():
    b = params.plan_bspline(1e-4, 14.4129, 1.0)
    e = params.plan(1e-4, 14.4129, 1.0)
    assert b["P"] == 5 and b["n_f"] > 2 * e["n_f"]
    # the grid ratio is Table 2's R_default (up to the FFT-friendly rounding)
    R = (b["n_f"] / params.pswf_grid_min(params.TABLE2[1e-4][1], 14.4129, 1.0)) ** 3
    assert 14.32 <= R <= 14.32 * 1.08 ** 3


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_comparator_reaches_ewald_within_tolerance(eps):
    s = inputs.uniform_charges(300, 5.0, 7)
    ref = ewald.ewald(s.pos, s.q, s.L)
    pl = params.plan_bspline(eps, s.L, 1.2)
    p = esp.ESPParams(eps, 1.2, pl["P"], pl["n_f"], kind="gauss", alpha=pl["alpha"], window="bspline")
    r = esp.esp(s.pos, s.q, s.L, p)
    delta = metrics.relative_rms_force_error(r["forces"], ref["forces"])
    assert delta <= eps, delta
    # the discrete energy identity holds for any window
    assert abs(r["fourier_energy"] - 0.5 * float(np.dot(s.q, r["spectral_potential"]))) <= 1e-10 * abs(r["energy"])
