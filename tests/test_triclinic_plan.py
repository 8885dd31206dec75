"""The triclinic planner (esp_plan_query_cell) without a GPU.

* A diagonal cell L I chooses the cube's parameters (c, c1, P, n_f, r_c and
  the cell list) and marks the plan triclinic.
* A sheared cell takes c, P and n_f from the cubic rules on its longest cell
  vector, and a cell list whose reach covers r_c across the smallest height.
* Cells outside the reduced orientation, cutoffs of half the smallest height
  or more, and options the triclinic path does not have are refused.
"""
import math

import numpy as np
import pytest

from oracle import params as oparams
from oracle import triclinic as tr


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09727_gb300 import _build, esp
    _build.build()
    return esp


SHEARED = tr.box_matrix([4.2, 0, 0], [1.1, 4.0, 0], [-0.8, 0.9, 3.9])


def _dodecahedron(d):
    """Rhombic dodecahedron (xy-square form) of nearest-image distance d."""
    return tr.box_matrix([d, 0, 0], [0, d, 0], [d / 2, d / 2, d * math.sqrt(2) / 2])


def _octahedron(d):
    """Truncated octahedron of nearest-image distance d."""
    return tr.box_matrix([d, 0, 0], [d / 3, 2 * math.sqrt(2) * d / 3, 0],
                         [-d / 3, math.sqrt(2) * d / 3, math.sqrt(6) * d / 3])


def test_diagonal_cell_chooses_the_cube_parameters(lib):
    L, N, eps = 6.0, 20_000, 1e-4
    cube = lib.esp_plan_query(L, N, eps, r_c=1.0)
    cell = lib.esp_plan_query_cell(L * np.eye(3), N, eps, r_c=1.0)
    for k in ("c", "c1", "P", "n_f", "r_c", "n_cells", "brick_cells", "tile", "cell_reach"):
        assert cell[k] == cube[k], k
    assert cell["triclinic"] == 1 and cube["triclinic"] == 0
    # the influence array covers the half spectrum instead of |k|^2
    n = cube["n_f"]
    assert cell["device_bytes"] - cube["device_bytes"] == 4 * (n * n * (n // 2 + 1) - (3 * (n // 2) ** 2 + 1)) \
        - 4 * (3 * (n // 2) ** 2 + 1)


@pytest.mark.parametrize("H", [SHEARED, _dodecahedron(5.0), _octahedron(5.5), np.diag([4.0, 5.0, 6.5])],
                         ids=["sheared", "dodecahedron", "octahedron", "orthorhombic"])
@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_cell_parameters_follow_the_longest_vector(lib, H, eps):
    r_c = 1.1
    got = lib.esp_plan_query_cell(H, 5000, eps, r_c=r_c)
    L_eff = float(np.max(np.linalg.norm(H, axis=0)))
    cube = lib.esp_plan_query(L_eff, 5000, eps, r_c=r_c)
    want = oparams.plan(eps, L_eff, r_c)
    assert abs(got["c"] - want["c"]) < 1e-9 * want["c"]
    assert got["P"] == want["P"] and got["n_f"] == cube["n_f"] and got["c1"] == cube["c1"]
    assert got["L"] == pytest.approx(L_eff, rel=1e-15)
    # every pair within r_c lies within cell_reach cells along each axis
    h_min = float(np.min(tr.heights(H)))
    assert got["n_cells"] * r_c <= got["cell_reach"] * h_min
    assert got["n_cells"] % got["brick_cells"] == 0


def test_automatic_cutoff_fits_the_cell(lib):
    H = _octahedron(4.0)
    got = lib.esp_plan_query_cell(H, 3000, 1e-4)
    assert 0 < got["r_c"] <= 0.45 * float(np.min(tr.heights(H))) + 1e-12


@pytest.mark.parametrize("H,kw,status", [
    (np.array([[4.0, 0, 0], [0.1, 4.0, 0], [0, 0, 4.0]]), {}, 1),     # a has a y component
    (SHEARED.T, {}, 1),                                                  # lower-triangular columns
    (np.diag([4.0, -4.0, 4.0]), {}, 1),
    (np.diag([4.0, 4.0, np.nan]), {}, 1),
    (SHEARED, dict(r_c=2.0), 2),                                         # beyond half the smallest height
    (SHEARED, dict(precision=1), 10),
    (SHEARED, dict(diff=1), 10),
    (SHEARED, dict(virial=1), 10),
    (SHEARED, dict(near_variant=2), 10),
])
def test_cell_refusals(lib, H, kw, status):
    kw = dict(dict(r_c=1.0), **kw)
    with pytest.raises(lib.EspError) as exc:
        lib.esp_plan_query_cell(H, 1000, 1e-4, **kw)
    assert exc.value.status == status


def _oracle_influence(H, n_f, info):
    """p_k from the oracle's split and window (Eq. pk on the lattice H) at
    the GPU layout's modes, averaged with the representative of -k where a
    component is -n_f/2 (the real part of the inverse transform)."""
    from oracle import esp as oesp
    p = oesp.ESPParams(1e-4, info["r_c"], info["P"], n_f, c=info["c"], c1=info["c1"])
    split, window = p.split(), p.si_window()
    V = abs(np.linalg.det(H))
    Hi = np.linalg.inv(H)
    half = n_f // 2
    comp = np.where(np.arange(n_f) < half, np.arange(n_f), np.arange(n_f) - n_f)

    def p_of(kx, ky, kz):
        K = np.stack([kx, ky, kz], axis=-1).astype(np.float64)
        xi = 2 * math.pi * K @ Hi
        x = np.sqrt(np.sum(xi * xi, axis=-1))
        Phi = window.Phi(2 * math.pi * np.stack([kx, ky, kz], -1) / n_f)
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(x > 0, split.chihat(info["r_c"] * x) / np.where(x > 0, x, 1.0) ** 2, 0.0)
        return s / (V * np.prod(Phi, axis=-1) ** 2)

    kz, ky, kx = np.meshgrid(comp, comp, comp[:half + 1], indexing="ij")
    kx = np.where(kx == half, -half, kx)
    neg = lambda k: np.where(k == -half, -half, -k)
    weight = np.prod(window.Phi(2 * math.pi * np.stack([kx, ky, kz], -1) / n_f), axis=-1) ** 2
    return 0.5 * (p_of(kx, ky, kz) + p_of(neg(kx), neg(ky), neg(kz))), weight


@pytest.mark.parametrize("H", [SHEARED, _dodecahedron(5.5), _octahedron(5.0), np.diag([4.0, 5.0, 6.5]),
                               4.6 * np.eye(3)], ids=["sheared", "dodecahedron", "octahedron", "orthorhombic", "cube"])
@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_influence_matches_the_oracle(lib, H, eps):
    """The planner's influence array (Hermite-tabulated chihat, per-axis
    window factors, the Nyquist average) against the oracle's Eq. pk."""
    r_c = 1.1
    got = lib.esp_influence_query(H, 700, eps, r_c=r_c)
    info = lib.esp_plan_query_cell(H, 700, eps, r_c=r_c)
    want, weight = _oracle_influence(H, info["n_f"], info)
    assert got.shape == want.shape
    # compared as Shat / V = p Phi^6: near the corner modes chihat is ~1e-12
    # of chihat(0), the two sides' quadratures differ there in the last
    # digits, and 1/Phi^6 (up to ~1e10 at P = 8) would magnify that; the
    # spread and gather multiply p_k by Phi^6 again, so this is the scale
    # that reaches the potentials
    err = np.max(np.abs(got - want) * weight)
    assert err <= 1e-10 * np.max(np.abs(want) * weight)
    # a cube plan applies the same values
    if np.allclose(H, H[0, 0] * np.eye(3)):
        cube = lib.esp_influence_query(H[0, 0], 700, eps, r_c=r_c)
        assert np.max(np.abs(cube - got) * weight) <= 1e-10 * np.max(np.abs(want) * weight)


def test_influence_query_arguments(lib):
    import ctypes
    so = lib.load_library()
    o = lib.make_opts(r_c=1.0)
    box = lib.esp_box((ctypes.c_double * 3)(5.0, 5.0, 5.0))
    cell = lib._cell(5.0 * np.eye(3))
    n = ctypes.c_int64(0)
    # exactly one of box and cell
    assert so.esp_influence_query(ctypes.byref(box), ctypes.byref(cell), 100, 1e-4, ctypes.byref(o), None,
                                  ctypes.byref(n)) == 1
    assert so.esp_influence_query(None, None, 100, 1e-4, ctypes.byref(o), None, ctypes.byref(n)) == 1
    assert so.esp_influence_query(ctypes.byref(box), None, 100, 1e-4, ctypes.byref(o), None, None) == 1
    # length query, then a buffer one entry short
    assert so.esp_influence_query(ctypes.byref(box), None, 100, 1e-4, ctypes.byref(o), None, ctypes.byref(n)) == 0
    n_f = lib.esp_plan_query(5.0, 100, 1e-4, r_c=1.0)["n_f"]
    assert n.value == n_f * n_f * (n_f // 2 + 1)
    short = ctypes.c_int64(n.value - 1)
    buf = np.zeros(n.value)
    assert so.esp_influence_query(ctypes.byref(box), None, 100, 1e-4, ctypes.byref(o),
                                  buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(short)) == 1
    # p_0 = 0 and p is even in k for a cube
    p = lib.esp_influence_query(5.0, 100, 1e-4, r_c=1.0)
    assert p[0, 0, 0] == 0.0
    assert np.allclose(p[1:, 1:, :], p[:0:-1, :0:-1, :], rtol=1e-14, atol=0)


def test_water_in_a_truncated_octahedron():
    """The triclinic bench input: volume n / density, SPC/E geometry, neutral,
    oxygens spread over the whole cell."""
    from paper_2505_09727_gb300 import inputs
    s = inputs.spce_water_cell(2000, seed=3)
    assert s.n == 6000 and abs(float(np.sum(s.q))) < 1e-12
    assert abs(np.linalg.det(s.H) - 2000 / inputs.WATER_DENSITY) < 1e-9
    h = tr.heights(s.H)
    assert np.allclose(h, h[0])                      # all faces of a truncated octahedron's cell alike
    o, h1, h2 = s.pos[0::3], s.pos[1::3], s.pos[2::3]
    assert np.allclose(np.linalg.norm(h1 - o, axis=1), 0.1) and np.allclose(np.linalg.norm(h2 - o, axis=1), 0.1)
    frac = np.linalg.solve(s.H, o.T).T
    assert frac.min() > -0.05 and frac.max() < 1.05
    assert np.all(np.ptp(frac, axis=0) > 0.9)
