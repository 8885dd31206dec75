"""Pins of the oracle's triclinic boxes (oracle/triclinic.py).

* H = L I reproduces the cubic oracle (ESP and Ewald) to rounding.
* Rock salt in its primitive (rhombohedral, 60 degree) cell: the Ewald energy
  per ion pair is the Madelung value -M / (4 pi d), d the nearest-neighbour
  distance, M = 1.747564594633...; ESP on a 3 x 3 x 3 supercell reaches it
  within the tolerance.
* A sheared description of the cubic lattice (b = a + b_cubic) has the same
  Ewald energy and forces as the cubic cell.
* ESP on a sheared box matches triclinic Ewald within the tolerance, and its
  forces are the energy gradient (central differences).
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald as cubic_ewald
from oracle import params as prm
from oracle import pswf
from oracle import triclinic as tr
from paper_2505_09727_gb300 import inputs

MADELUNG = 1.747564594633182


def _esp_params(eps, H, r_c):
    """ESP parameters from the cubic rules applied to the longest cell vector
    (a conservative grid for the sheared cell)."""
    L_eff = float(np.max(np.linalg.norm(H, axis=0)))
    c, c1, P, n_f = prm.pswf_parameters(eps, L_eff, r_c)
    return pswf.PSWFSplit(c), pswf.PSWFWindow(c1, P), n_f


def _rel_rms(f, ref):
    return float(np.sqrt(np.sum((f - ref) ** 2) / np.sum(ref ** 2)))


def _fcc_rock_salt(reps: int, a_c: float = 1.0):
    """Primitive rock-salt cell (d = a_c / sqrt 2 edges, 60 degree angles) in
    triangular form, repeated reps^3 times: (pos, q, H)."""
    d = a_c / math.sqrt(2.0)
    a = np.array([d, 0.0, 0.0])
    b = np.array([d / 2, d * math.sqrt(3.0) / 2, 0.0])
    c = np.array([d / 2, d / (2 * math.sqrt(3.0)), d * math.sqrt(2.0 / 3.0)])
    pos, q = [], []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                o = i * a + j * b + k * c
                pos += [o, o + 0.5 * (a + b + c)]
                q += [1.0, -1.0]
    H = tr.box_matrix(reps * a, reps * b, reps * c)
    return np.array(pos), np.array(q), H


def test_cubic_box_reproduces_the_cubic_oracle():
    s = inputs.uniform_charges(80, 3.0, 5)
    H = tr.box_matrix([3.0, 0, 0], [0, 3.0, 0], [0, 0, 3.0])
    et = tr.ewald_converged(s.pos, s.q, H)
    ec = cubic_ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    assert abs(et["energy"] - ec["energy"]) <= 1e-12 * abs(ec["energy"])
    assert np.max(np.abs(et["forces"] - ec["forces"])) <= 1e-12 * np.max(np.abs(ec["forces"]))
    p = oesp.default_params(1e-4, s.L, 1.1).resolved()
    rc = oesp.esp(s.pos, s.q, s.L, p)
    rt = tr.esp(s.pos, s.q, H, p.split(), p.si_window(), p.n_f, p.r_c)
    assert abs(rt["energy"] - rc["energy"]) <= 1e-12 * abs(rc["energy"])
    assert np.max(np.abs(rt["forces"] - rc["forces"])) <= 1e-12 * np.max(np.abs(rc["forces"]))


def test_rock_salt_primitive_cell_madelung():
    pos, q, H = _fcc_rock_salt(1)
    e = tr.ewald_converged(pos, q, H)["energy"]
    assert abs(e - (-MADELUNG / (4 * math.pi * 0.5))) <= 1e-11 * MADELUNG


def test_rock_salt_supercell_esp_reaches_madelung():
    pos, q, H = _fcc_rock_salt(3)
    eps = 1e-5
    split, window, n_f = _esp_params(eps, H, 0.8)
    r = tr.esp(pos, q, H, split, window, n_f, 0.8)
    e_ref = -27 * MADELUNG / (4 * math.pi * 0.5)
    assert abs(r["energy"] - e_ref) <= eps * abs(e_ref)
    assert np.max(np.abs(r["forces"])) <= eps * MADELUNG / (4 * math.pi * 0.25)   # forces vanish by symmetry


def test_sheared_description_of_a_cubic_lattice():
    s = inputs.uniform_charges(60, 3.0, 11)
    cube = tr.box_matrix([3.0, 0, 0], [0, 3.0, 0], [0, 0, 3.0])
    sheared = tr.box_matrix([3.0, 0, 0], [3.0, 3.0, 0], [0, 0, 3.0])
    # the sheared cell's shorter height shrinks the real-space cutoff, so
    # both sums are taken to 1e-18 truncation
    a = tr.ewald_converged(s.pos, s.q, cube, acc=1e-18)
    b = tr.ewald_converged(s.pos, s.q, sheared, acc=1e-18)
    assert abs(a["energy"] - b["energy"]) <= 1e-10 * abs(a["energy"])
    assert np.max(np.abs(a["forces"] - b["forces"])) <= 1e-9 * np.max(np.abs(a["forces"]))


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_esp_on_a_sheared_box_matches_ewald(eps):
    rng = np.random.default_rng(17)
    H = tr.box_matrix([3.2, 0, 0], [0.9, 3.0, 0], [-0.6, 0.7, 2.9])
    n = 120
    pos = rng.random((n, 3)) @ H.T
    q = np.repeat([1.0, -1.0], n // 2)
    ref = tr.ewald_converged(pos, q, H)
    split, window, n_f = _esp_params(eps, H, 1.1)
    r = tr.esp(pos, q, H, split, window, n_f, 1.1)
    assert _rel_rms(r["forces"], ref["forces"]) <= eps
    assert abs(r["energy"] - ref["energy"]) <= eps * abs(ref["energy"])


def test_triclinic_forces_are_the_energy_gradient():
    rng = np.random.default_rng(19)
    H = tr.box_matrix([3.0, 0, 0], [0.8, 2.8, 0], [0.5, -0.4, 3.1])
    n = 60
    pos = rng.random((n, 3)) @ H.T
    q = np.repeat([1.0, -1.0], n // 2)
    split, window, n_f = _esp_params(1e-6, H, 1.0)
    f = tr.esp(pos, q, H, split, window, n_f, 1.0)["forces"]
    h = 1e-5
    for i, a in [(0, 0), (17, 1), (44, 2)]:
        e = []
        for sgn in (1.0, -1.0):
            p2 = pos.copy()
            p2[i, a] += sgn * h
            e.append(tr.esp(p2, q, H, split, window, n_f, 1.0)["energy"])
        assert abs(-(e[0] - e[1]) / (2 * h) - f[i, a]) <= 1e-7 * np.max(np.abs(f))


def _deformation_fd(energy_of, H, pos, h=1e-6):
    """W_ab = -dE/d eps_ab by central differences under r -> (1 + eps) r,
    H -> (1 + eps) H with a symmetric eps."""
    W = np.zeros((3, 3))
    for a in range(3):
        for b in range(a, 3):
            e = []
            for sgn in (1.0, -1.0):
                eps = np.zeros((3, 3))
                eps[a, b] += sgn * h
                if a != b:
                    eps[b, a] += sgn * h
                D = np.eye(3) + eps
                e.append(energy_of(pos @ D.T, D @ H))
            W[a, b] = W[b, a] = -(e[0] - e[1]) / (2 * h) / (1.0 if a == b else 2.0)
    return W


def test_triclinic_virial_is_the_deformation_derivative():
    rng = np.random.default_rng(17)
    H = tr.box_matrix([3.2, 0, 0], [0.9, 3.0, 0], [-0.6, 0.7, 2.9])
    n = 60
    pos = rng.random((n, 3)) @ H.T
    q = np.repeat([1.0, -1.0], n // 2)
    q[0] += 0.3                                                  # background term too
    split, window, n_f = _esp_params(1e-4, H, 1.0)
    W = tr.esp(pos, q, H, split, window, n_f, 1.0, virial=True)["virial"]
    fd = _deformation_fd(lambda x, Hd: tr.esp(x, q, Hd, split, window, n_f, 1.0)["energy"], H, pos)
    assert np.max(np.abs(W - fd)) <= 1e-7 * np.max(np.abs(W))


def test_cube_virial_readings_against_the_deformation_derivative():
    """The cube's full virial tensor pinned by shearing it (the triclinic
    energy of the deformed cell): the "alias" Nyquist reading (the oracle's
    default, and the CUDA path's) is the exact derivative; the "component"
    reading (each Nyquist component averaged on its own) differs only in the
    off-diagonal terms of modes with two Nyquist components."""
    import dataclasses
    s = inputs.uniform_charges(80, 3.0, 5)
    p = oesp.default_params(1e-4, s.L, 1.1).resolved()
    H = s.L * np.eye(3)
    fd = _deformation_fd(lambda x, Hd: tr.esp(x, s.q, Hd, p.split(), p.si_window(), p.n_f, p.r_c)["energy"],
                         H, s.pos)
    W_alias = oesp.esp(s.pos, s.q, s.L, p)["virial"]
    W_comp = oesp.esp(s.pos, s.q, s.L, dataclasses.replace(p, virial_nyquist="component"))["virial"]
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(W_alias - fd)) <= 1e-7 * scale
    assert np.array_equal(np.diag(W_alias), np.diag(W_comp))
    assert 0 < np.max(np.abs(W_comp - W_alias)) <= 1e-5 * scale
