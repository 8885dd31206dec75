"""Triclinic cells (esp_plan_cell) on the GPU against the oracle's triclinic
ESP and Ewald.

* A diagonal cell L I gives the cube's results (same parameters; the pair
  sums run in another order, so to FP32 rounding).
* Sheared, truncated-octahedral, rhombic-dodecahedral and orthorhombic cells
  match the oracle's triclinic ESP at the plan's parameters within the FP32
  parity bound, and triclinic Ewald within the tolerance.
* Rock salt in its primitive (60 degree) cell, 3^3 cells: the Madelung
  energy within the tolerance and vanishing forces.
* Coordinates shifted by lattice vectors give the same results; esp_step
  (graph replay) equals esp_compute.

The triclinic path is among the newest on the GPU, so this file is
collected after the established ones (test_zz_*): a run that stops at the
first failure has run those first.
"""
import math

import numpy as np
import pytest

from oracle import esp as oesp
from oracle import triclinic as tr
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_PARITY = 5e-6          # the cube's FP32 parity bound (same arithmetic)
MADELUNG = 1.747564594633182


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def gpu_cell(esp, H, pos, q, eps, **opts):
    with esp.Plan(H, len(q), eps, **opts) as p:
        p.set_charges(q)
        p.set_positions(pos)
        e, f, u = p.compute()
        return dict(energy=e, forces=f, potential=u, info=p.info)


def oracle_cell(H, pos, q, eps, info):
    kind = "pswf" if info["kernel"] == 0 else "gauss"
    window = "bspline" if info["window"] == 1 else "pswf"
    p = oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"], kind=kind,
                       alpha=info["alpha"] if kind == "gauss" else None, window=window)
    return tr.esp(pos, q, H, p.split(), p.si_window(), info["n_f"], info["r_c"])


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def dodecahedron(d):
    return tr.box_matrix([d, 0, 0], [0, d, 0], [d / 2, d / 2, d * math.sqrt(2) / 2])


def octahedron(d):
    return tr.box_matrix([d, 0, 0], [d / 3, 2 * math.sqrt(2) * d / 3, 0],
                         [-d / 3, math.sqrt(2) * d / 3, math.sqrt(6) * d / 3])


def charges_in(H, n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) @ H.T
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)    # odd n: net charge +1 (background term)
    return pos, q


CELLS = {
    "sheared": (tr.box_matrix([4.2, 0, 0], [1.1, 4.0, 0], [-0.8, 0.9, 3.9]), 600, 1e-4, 1.2),
    "octahedron_eps1e-5": (octahedron(5.0), 500, 1e-5, 1.2),
    "dodecahedron_eps1e-3": (dodecahedron(5.5), 700, 1e-3, 1.1),
    "orthorhombic_ragged": (np.diag([4.0, 5.0, 6.5]), 611, 1e-4, 1.0),
    "sheared_many_bricks": (tr.box_matrix([6.4, 0, 0], [-1.5, 6.1, 0], [1.2, -1.9, 6.0]), 2000, 1e-4, 0.9),
}


def test_diagonal_cell_equals_the_cube(esp):
    s = inputs.spce_water(500, seed=4)
    cell = gpu_cell(esp, s.L * np.eye(3), s.pos, s.q, 1e-4, r_c=1.0)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, u = p.compute()
        info = p.info
    for k in ("n_f", "P", "c1", "n_cells"):
        assert cell["info"][k] == info[k], k
    assert rel_rms(cell["forces"], f) <= 1e-6
    assert abs(cell["energy"] - e) <= 1e-6 * abs(e)
    assert np.max(np.abs(cell["potential"] - u)) <= 1e-6 * np.max(np.abs(u))


@pytest.mark.parametrize("name", list(CELLS))
def test_cell_matches_the_oracle(esp, name):
    H, n, eps, r_c = CELLS[name]
    pos, q = charges_in(H, n, 31)
    g = gpu_cell(esp, H, pos, q, eps, r_c=r_c)
    assert g["info"]["triclinic"] == 1
    o = oracle_cell(H, pos, q, eps, g["info"])
    assert rel_rms(g["forces"], o["forces"]) <= FP32_PARITY
    # as for the cube: the FP32 spectral potential still holds each charge's
    # smooth self-interaction (removed afterwards in FP64), so its rounding
    # scales with the self energy, which for random charges exceeds |E|
    e_self = -0.5 * float(np.sum(q * q)) * oesp.ESPParams(
        eps, g["info"]["r_c"], g["info"]["P"], g["info"]["n_f"], c=g["info"]["c"]).split().chi0 \
        / (4 * math.pi * g["info"]["r_c"])
    assert abs(g["energy"] - o["energy"]) <= FP32_PARITY * max(abs(o["energy"]), abs(e_self))
    assert rel_rms(g["potential"], o["potential"]) <= FP32_PARITY


@pytest.mark.parametrize("name", ["sheared", "octahedron_eps1e-5"])
def test_cell_within_tolerance_of_ewald(esp, name):
    H, n, eps, r_c = CELLS[name]
    pos, q = charges_in(H, n, 31)
    g = gpu_cell(esp, H, pos, q, eps, r_c=r_c)
    ref = tr.ewald_converged(pos, q, H)
    assert rel_rms(g["forces"], ref["forces"]) <= eps
    assert abs(g["energy"] - ref["energy"]) <= eps * abs(ref["energy"])


def test_rock_salt_primitive_cells(esp):
    d = 1.0 / math.sqrt(2.0)
    a = np.array([d, 0.0, 0.0])
    b = np.array([d / 2, d * math.sqrt(3.0) / 2, 0.0])
    c = np.array([d / 2, d / (2 * math.sqrt(3.0)), d * math.sqrt(2.0 / 3.0)])
    reps = 3
    pos, q = [], []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                o = i * a + j * b + k * c
                pos += [o, o + 0.5 * (a + b + c)]
                q += [1.0, -1.0]
    H = tr.box_matrix(reps * a, reps * b, reps * c)
    eps = 1e-5
    g = gpu_cell(esp, H, np.array(pos), np.array(q), eps, r_c=0.8)
    e_ref = -27 * MADELUNG / (4 * math.pi * 0.5)
    assert abs(g["energy"] - e_ref) <= eps * abs(e_ref)
    assert np.max(np.abs(g["forces"])) <= eps * MADELUNG / (4 * math.pi * 0.25)


def test_lattice_shifts_and_graph_step(esp):
    H, n, eps, r_c = CELLS["sheared"]
    pos, q = charges_in(H, n, 32)
    rng = np.random.default_rng(5)
    shifted = pos + rng.integers(-3, 4, size=(n, 3)) @ H.T
    with esp.Plan(H, n, eps, r_c=r_c) as p:
        p.set_charges(q)
        p.set_positions(pos)
        e0, f0, u0 = p.compute()
        p.set_positions(shifted)
        e1, f1, u1 = p.compute()
        e = np.zeros(1)
        f = np.zeros((n, 3))
        u = np.zeros(n)
        for _ in range(2):                              # direct run, then the captured graph
            esp.esp_step(p.handle, pos, e, f, u)
            # the half-form pair sums add with atomics: equal to FP32 rounding
            assert rel_rms(f, f0) <= 1e-6 and abs(e[0] - e0) <= 1e-6 * abs(e0)
            assert np.max(np.abs(u - u0)) <= 1e-6 * np.max(np.abs(u0))
    assert rel_rms(f1, f0) <= 1e-6 and abs(e1 - e0) <= 1e-6 * abs(e0)
