"""Pins of the oracle's MD workload (oracle/md.py).

* Bonded terms: zero at the equilibrium geometry, (1/2) k delta^2 and a
  force k delta along the bond for a stretched bond, (1/2) k_theta dtheta^2
  for an opened angle, no net force and no net torque.
* Lennard-Jones: no force at r = 2^(1/6) sigma, zero energy at the cutoff.
* Exclusions: a single molecule in a cubic box keeps, after the direct
  intramolecular pairs are removed, only its interaction with its own
  images: -|p|^2 / (6 V) for the dipole p under tinfoil boundary conditions
  (the simple-cubic dipole lattice sum vanishes), with corrections of
  relative order (molecule size / L)^2.
* Forces are central differences of the total energy (bonded, LJ, ESP with
  exclusions).
* Velocity Verlet: the energy error falls as dt^2 (forces consistent with
  the energy), and the integration runs backwards to the start when the
  velocities are reversed.
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import md
from paper_2505_09727_gb300 import inputs

MODEL = md.WaterModel()


def _molecule(theta=MODEL.theta0, r1=MODEL.r0, r2=MODEL.r0):
    """One molecule in the xz plane around O at (1, 1, 1)."""
    o = np.array([1.0, 1.0, 1.0])
    h1 = o + r1 * np.array([math.sin(theta / 2), 0.0, math.cos(theta / 2)])
    h2 = o + r2 * np.array([-math.sin(theta / 2), 0.0, math.cos(theta / 2)])
    return np.stack([o, h1, h2])


def test_bonded_terms_closed_forms():
    e, f = md.bonded(_molecule(), 5.0, MODEL)
    assert abs(e) < 1e-20 and np.max(np.abs(f)) < 1e-9
    delta = 0.003
    pos = _molecule(r1=MODEL.r0 + delta)
    e, f = md.bonded(pos, 5.0, MODEL)
    assert e == pytest.approx(0.5 * MODEL.k_bond * delta ** 2, rel=1e-12)
    axis = (pos[1] - pos[0]) / np.linalg.norm(pos[1] - pos[0])
    assert np.allclose(f[1], -MODEL.k_bond * delta * axis, rtol=1e-12, atol=1e-9)
    assert np.allclose(f[2], 0.0, atol=1e-9)
    dth = 0.05
    pos = _molecule(theta=MODEL.theta0 + dth)
    e, f = md.bonded(pos, 5.0, MODEL)
    assert e == pytest.approx(0.5 * MODEL.k_angle * dth ** 2, rel=1e-12)
    assert np.allclose(f.sum(axis=0), 0.0, atol=1e-9)
    torque = np.cross(pos - pos[0], f).sum(axis=0)
    assert np.allclose(torque, 0.0, atol=1e-9)


def test_lennard_jones_minimum_and_cutoff():
    a, b = _molecule(), _molecule()
    r_min = 2 ** (1 / 6) * MODEL.sigma
    b = b + np.array([r_min, 0.0, 0.0])
    pos = np.concatenate([a, b])
    e, f = md.lennard_jones_oxygen(pos, 5.0, 1.2, MODEL)
    shift = 4 * MODEL.epsilon * ((MODEL.sigma / 1.2) ** 12 - (MODEL.sigma / 1.2) ** 6)
    assert e == pytest.approx(-MODEL.epsilon - shift, rel=1e-12)
    assert np.max(np.abs(f)) < 1e-9
    pos[3:] += np.array([1.2 - r_min - 1e-9, 0.0, 0.0])
    e, _ = md.lennard_jones_oxygen(pos, 5.0, 1.2, MODEL)
    assert abs(e) < 1e-9


@pytest.mark.parametrize("L", [2.0, 3.0, 4.0, 6.0])
def test_exclusions_leave_the_image_dipole_energy(L):
    rng = np.random.default_rng(1)
    pos, q = inputs._water_sites(rng, np.full((1, 3), L / 2))
    p = oesp.default_params(1e-9, L, 0.4 * L).resolved()
    e_esp = oesp.esp(pos, q, L, p)["energy"]
    e_ex, _, _ = md.exclusion_correction(pos, q, L, md.exclusion_pairs(3))
    dip = q @ pos
    want = -float(dip @ dip) / (6.0 * L ** 3)
    # leading order in (size / L): the quadrupole terms are ~4e-3 at L = 2 nm
    assert abs((e_esp + e_ex) / want - 1.0) <= 0.03 / L ** 2


def _water_box():
    s = inputs.spce_water(8, density=5.0, seed=3)
    p = oesp.default_params(1e-8, s.L, 0.55).resolved()
    return s, md.WaterForceField(s.q, s.L, p, 0.55)


def test_forces_are_the_energy_gradient():
    s, ff = _water_box()
    _, f = ff(s.pos)
    h = 1e-6
    for i, a in [(0, 0), (1, 2), (5, 1), (12, 0), (22, 2)]:
        e = []
        for sgn in (1.0, -1.0):
            pos = s.pos.copy()
            pos[i, a] += sgn * h
            e.append(ff(pos)[0])
        assert abs(-(e[0] - e[1]) / (2 * h) - f[i, a]) <= 1e-6 * np.max(np.abs(f))


def test_velocity_verlet_energy_error_scales_as_dt_squared():
    s, ff = _water_box()
    m = MODEL.masses(s.n)
    v = md.maxwell_boltzmann(m, 300.0, 7)
    err = []
    for dt, n in [(4e-4, 40), (2e-4, 80)]:                 # the same 16 fs
        tr = md.velocity_verlet(s.pos, v, m, dt, n, ff)
        e = tr["e_pot"] + tr["e_kin"]
        err.append(np.max(np.abs(e - e[0])))
    assert 3.6 <= err[0] / err[1] <= 4.4


def test_velocity_verlet_is_time_reversible():
    s, ff = _water_box()
    m = MODEL.masses(s.n)
    v = md.maxwell_boltzmann(m, 300.0, 8)
    fwd = md.velocity_verlet(s.pos, v, m, 4e-4, 25, ff)
    back = md.velocity_verlet(fwd["pos"], -fwd["vel"], m, 4e-4, 25, ff)
    assert np.max(np.abs(back["pos"] - s.pos)) < 1e-12
    assert np.max(np.abs(back["vel"] + v)) < 1e-9
