"""Pins for oracle.ewald (classical Ewald) and oracle.images (brute force)."""
import numpy as np
import pytest

from golden_io import rows
from oracle import ewald, images
from paper_2505_09727_gb300 import inputs


@pytest.fixture(scope="module")
def nacl():
    s = inputs.nacl_lattice(8)
    return s, ewald.ewald(s.pos, s.q, s.L)


def test_nacl_madelung(nacl):
    s, r = nacl
    (m, cells, a, n, d, e_ref, u_unit), = rows("nacl_madelung.txt")
    assert s.n == int(n)
    e_closed = -(int(n) / 2) * float(m) / (4 * np.pi * float(d))
    assert abs(e_closed - float(e_ref)) < 1e-10
    assert abs(r["energy"] - e_closed) / abs(e_closed) < 1e-12
    assert np.max(np.abs(r["potential"] - s.q * float(u_unit))) < 1e-12
    assert np.max(np.abs(r["forces"])) < 1e-12            # inversion symmetry


@pytest.mark.parametrize("seed", [3, 4])
def test_matches_brute_force_image_sums(seed):
    rng = np.random.default_rng(seed)
    L = 1.0
    pos = rng.uniform(0, L, (4, 3))
    q = np.array([1.0, -1.0, 0.5, -0.5])
    r = ewald.ewald(pos, q, L)
    e_s, f_s = images.surface_terms(pos, q, L)
    e_b, f_b = images.extrapolated(pos, q, L, R=16)
    assert abs(e_b - (r["energy"] + e_s)) < 1e-8 * abs(r["energy"])
    assert np.max(np.abs(f_b - (r["forces"] + f_s))) < 1e-7 * np.max(np.abs(r["forces"]))


def test_splitting_parameter_independence():
    s = inputs.uniform_charges(200, 5.0, 1)
    a = ewald.ewald(s.pos, s.q, s.L)
    b = ewald.ewald(s.pos, s.q, s.L, g=a["g"] * 1.4)
    assert abs(a["energy"] - b["energy"]) < 1e-12 * abs(a["energy"])
    assert np.max(np.abs(a["forces"] - b["forces"])) < 1e-11 * np.max(np.abs(a["forces"]))
    assert np.max(np.abs(a["potential"] - b["potential"])) < 1e-11 * np.max(np.abs(a["potential"]))


def test_invariants():
    s = inputs.uniform_charges(100, 4.0, 5)
    r = ewald.ewald(s.pos, s.q, s.L)
    rms = np.sqrt(np.mean(r["forces"] ** 2))
    assert np.max(np.abs(r["forces"].sum(axis=0))) < 1e-12 * rms * s.n
    # energy = 1/2 sum q u
    assert abs(r["energy"] - 0.5 * np.dot(s.q, r["potential"])) < 1e-14 * abs(r["energy"]) * s.n
    # translation
    t = ewald.ewald(s.pos + np.array([0.37, -1.1, 2.9]), s.q, s.L)
    assert abs(t["energy"] - r["energy"]) < 1e-12 * abs(r["energy"])
    assert np.max(np.abs(t["forces"] - r["forces"])) < 1e-11 * rms
    # linearity: q -> 2q gives E x 4, F x 4
    d = ewald.ewald(s.pos, 2 * s.q, s.L)
    assert abs(d["energy"] - 4 * r["energy"]) < 1e-12 * abs(r["energy"])
    # 90-degree rotation about z: (x, y, z) -> (-y, x, z) permutes force components
    rot = np.stack([-s.pos[:, 1], s.pos[:, 0], s.pos[:, 2]], axis=1)
    o = ewald.ewald(rot, s.q, s.L)
    f_rot = np.stack([-r["forces"][:, 1], r["forces"][:, 0], r["forces"][:, 2]], axis=1)
    assert np.max(np.abs(o["forces"] - f_rot)) < 1e-11 * rms


def test_two_ions_near_coulomb():
    # +-1 at distance d << L: force approaches 1/(4 pi d^2) along the axis
    L, d = 20.0, 0.2
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + d, 5.0, 5.0]])
    q = np.array([1.0, -1.0])
    r = ewald.ewald(pos, q, L)
    f = r["forces"][0, 0]
    assert abs(f - 1.0 / (4 * np.pi * d * d)) / (1.0 / (4 * np.pi * d * d)) < 1e-3
    assert abs(r["forces"][0, 1]) < 1e-12


def test_sampled_targets_match_full():
    s = inputs.uniform_charges(200, 5.0, 2)
    full = ewald.ewald(s.pos, s.q, s.L)
    idx = np.array([0, 17, 150, 199])
    part = ewald.ewald(s.pos, s.q, s.L, targets=idx)
    assert np.max(np.abs(part["forces"] - full["forces"][idx])) < 1e-13
    assert np.max(np.abs(part["potential"] - full["potential"][idx])) < 1e-13


def test_background_matches_textbook():
    # non-neutral: the Ewald result is g-independent only with the background
    s = inputs.uniform_charges(60, 4.0, 9)
    q = s.q.copy()
    q[0] += 0.5
    a = ewald.ewald(s.pos, q, s.L)
    b = ewald.ewald(s.pos, q, s.L, g=a["g"] * 1.3)
    assert abs(a["energy"] - b["energy"]) < 1e-11 * abs(a["energy"])
