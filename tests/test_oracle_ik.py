"""Pins of the oracle's ik force method (Methods: multiply the scaled
spectrum by 2 pi i k / L and transform back, instead of differentiating the
SI kernel).

* ik_gradient on a single real Fourier mode returns its closed-form
  derivative on the grid, and zero for the Nyquist mode of the
  differentiated axis (the reading for even n_f).
* The ik method changes nothing but the spectral gradients: potentials and
  energies equal the AD run's exactly.
* ik forces match converged Ewald within the tolerance, and the AD forces to
  the same order.
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald, metrics
from paper_2505_09727_gb300 import inputs


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, -3), (3, -1, 2), (-5, 4, 1)])
def test_ik_gradient_of_a_single_mode(m):
    n, L = 12, 3.7
    l = np.arange(n)
    X, Y, Z = np.meshgrid(l, l, l, indexing="ij")
    phase = 2 * math.pi * (m[0] * X + m[1] * Y + m[2] * Z) / n + 0.3
    c = np.cos(phase)
    ch = np.fft.ifftn(c)                         # c = fftn(ch), the oracle's step-4 convention
    grads = oesp.ik_gradient(ch, L)
    for a in range(3):
        exact = -(2 * math.pi * m[a] / L) * np.sin(phase)
        assert np.max(np.abs(grads[a] - exact)) < 1e-12


def test_ik_gradient_drops_the_nyquist_mode_of_its_axis():
    n, L = 8, 2.0
    l = np.arange(n)
    X, Y, Z = np.meshgrid(l, l, l, indexing="ij")
    c = np.cos(math.pi * X) * np.cos(2 * math.pi * Y / n)   # Nyquist along x
    gx, gy, gz = oesp.ik_gradient(np.fft.ifftn(c), L)
    assert np.max(np.abs(gx)) < 1e-12
    exact_y = -(2 * math.pi / L) * np.cos(math.pi * X) * np.sin(2 * math.pi * Y / n)
    assert np.max(np.abs(gy - exact_y)) < 1e-12
    assert np.max(np.abs(gz)) < 1e-12


def _params(eps, L, r_c, diff):
    p = oesp.default_params(eps, L, r_c)
    p.diff = diff
    return p


def test_ik_changes_only_the_spectral_gradient():
    s = inputs.uniform_charges(200, 4.0, 17)
    ad = oesp.esp(s.pos, s.q, s.L, _params(1e-4, s.L, 1.2, "ad"))
    ik = oesp.esp(s.pos, s.q, s.L, _params(1e-4, s.L, 1.2, "ik"))
    assert np.array_equal(ad["potential"], ik["potential"])
    assert ad["energy"] == ik["energy"]
    assert np.array_equal(ad["local_forces"], ik["local_forces"])
    assert not np.array_equal(ad["spectral_forces"], ik["spectral_forces"])


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_ik_forces_within_tolerance_of_ewald(eps):
    s = inputs.spce_water(300, seed=19)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    ik = oesp.esp(s.pos, s.q, s.L, _params(eps, s.L, 0.9, "ik"))
    ad = oesp.esp(s.pos, s.q, s.L, _params(eps, s.L, 0.9, "ad"))
    d_ik = metrics.relative_rms_force_error(ik["forces"], ref["forces"])
    d_ad = metrics.relative_rms_force_error(ad["forces"], ref["forces"])
    assert d_ik <= eps, d_ik
    assert metrics.relative_rms_force_error(ik["forces"], ad["forces"]) <= 2 * eps
    assert d_ad <= eps


def test_oracle_forces_are_the_energy_gradient():
    """The oracle's AD forces equal central differences of its energy."""
    s = inputs.uniform_charges(60, 3.0, 63)
    p = oesp.default_params(1e-6, s.L, 1.2)
    f = oesp.esp(s.pos, s.q, s.L, p)["forces"]
    h = 1e-5
    for i, a in [(0, 0), (11, 1), (42, 2)]:
        e = []
        for sgn in (1.0, -1.0):
            pos = s.pos.copy()
            pos[i, a] += sgn * h
            e.append(oesp.esp(pos, s.q, s.L, p)["energy"])
        assert abs(-(e[0] - e[1]) / (2 * h) - f[i, a]) <= 1e-7 * np.max(np.abs(f))
