"""Pins of the oracle's virial W_ab = -dE/d eps_ab (homogeneous deformation
of atoms and box).

* Trace: a central finite difference of the energy under the isotropic
  scaling r -> s r, L -> s L equals -tr W (ESP with both splits, Ewald).
* Full tensor: the ESP virial (general per-mode form) matches the textbook
  Ewald virial within the tolerance's order, and an isolated dipole in a
  large box has the bare Coulomb pair virial q1 q2 d d^T / (4 pi r^3).
* Index consistency: swapping the x and y coordinates of every atom swaps
  the corresponding rows and columns of W.
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald
from paper_2505_09727_gb300 import inputs


def _fd_trace(energy_at, h=1e-6):
    return (energy_at(1.0 + h) - energy_at(1.0 - h)) / (2.0 * h)


def test_ewald_virial_trace_is_the_scaling_derivative():
    s = inputs.spce_water(100, seed=5)
    W = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)["virial"]
    d = _fd_trace(lambda f: ewald.ewald(s.pos * f, s.q, s.L * f, acc=1e-14)["energy"])
    assert abs(d + np.trace(W)) <= 1e-8 * abs(np.trace(W))


@pytest.mark.parametrize("kind", ["pswf", "gauss"])
def test_esp_virial_trace_is_the_scaling_derivative(kind):
    s = inputs.uniform_charges(120, 3.0, 23)
    p = oesp.default_params(1e-4, s.L, 1.1, kind=kind)
    W = oesp.esp(s.pos, s.q, s.L, p)["virial"]
    d = _fd_trace(lambda f: oesp.esp(s.pos * f, s.q, s.L * f, p)["energy"])
    assert abs(d + np.trace(W)) <= 1e-7 * np.max(np.abs(W))


def test_non_neutral_background_enters_the_virial():
    s = inputs.uniform_charges(60, 3.0, 29)
    q = s.q.copy()
    q[0] += 0.5                                    # net charge: background term
    p = oesp.default_params(1e-4, s.L, 1.1)
    W = oesp.esp(s.pos, q, s.L, p)["virial"]
    d = _fd_trace(lambda f: oesp.esp(s.pos * f, q, s.L * f, p)["energy"])
    assert abs(d + np.trace(W)) <= 1e-7 * np.max(np.abs(W))


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
@pytest.mark.parametrize("kind", ["pswf", "gauss"])
def test_esp_virial_matches_ewald_tensor(kind, eps):
    s = inputs.spce_water(300, seed=3)
    W_ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)["virial"]
    W = oesp.esp(s.pos, s.q, s.L, oesp.default_params(eps, s.L, 0.9, kind=kind))["virial"]
    assert np.max(np.abs(W - W_ref)) <= 10 * eps * np.max(np.abs(W_ref))


def test_isolated_dipole_has_the_pair_virial():
    d = np.array([0.3, 0.2, -0.1])
    L = 12.0
    pos = np.array([[6.0, 6.0, 6.0], [6.0, 6.0, 6.0] + d])
    q = np.array([1.0, -1.0])
    W = oesp.esp(pos, q, L, oesp.default_params(1e-6, L, 1.5))["virial"]
    # force on atom 0 from atom 1 times (r_0 - r_1): q0 q1 (r_0 - r_1)(r_0 - r_1)^T / (4 pi r^3)
    r = np.linalg.norm(d)
    W_pair = q[0] * q[1] * np.outer(d, d) / (4.0 * math.pi * r ** 3)
    assert np.max(np.abs(W - W_pair)) <= 1e-3 * np.max(np.abs(W_pair))


def test_axis_swap_permutes_the_virial():
    s = inputs.uniform_charges(80, 3.0, 31)
    p = oesp.default_params(1e-4, s.L, 1.1)
    W = oesp.esp(s.pos, s.q, s.L, p)["virial"]
    swapped = s.pos[:, [1, 0, 2]]
    Ws = oesp.esp(swapped, s.q, s.L, p)["virial"]
    perm = [1, 0, 2]
    assert np.max(np.abs(Ws - W[np.ix_(perm, perm)])) <= 1e-12 * np.max(np.abs(W))
