"""The C-ABI library without a GPU: it builds, loads, exports every entry point
declared in include/*.h, validates its arguments, and its host planner makes
the same parameter choices as the oracle's reading of the paper's rules."""
import ctypes
import glob
import math
import os
import re

import pytest

from oracle import params as oparams

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09727_gb300 import _build, esp
    _build.build()
    return esp


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(esp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "esp_plan" in names and "esp_compute" in names and len(names) >= 15
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_version_and_opts(lib):
    assert "sm_103a" in lib.esp_version()
    o = lib.esp_plan_opts_init()
    assert o.precision == lib.ESP_FP32 and o.kernel == lib.ESP_KERNEL_PSWF and o.prefactor == 1.0


@pytest.mark.parametrize("L,N,eps,r_c", [
    (14.413, 300_000, 1e-4, 1.0),       # water 1e5 molecules
    (31.05, 3_000_000, 1e-5, 1.0),      # water 1e6 molecules
    (20.0, 1000, 1e-4, 5.0),            # uniform +-1 charges
    (8.0, 4096, 1e-4, 2.0),             # NaCl 8^3 cells
    (3.912, 6000, 1e-3, 1.0),
    (5.0, 300, 1e-5, 1.2),
])
def test_planner_matches_oracle_reading(lib, L, N, eps, r_c):
    got = lib.esp_plan_query(L, N, eps, r_c=r_c)
    want = oparams.plan(eps, L, r_c)
    assert abs(got["c"] - want["c"]) < 1e-9 * want["c"]
    assert got["P"] == want["P"]
    assert got["n_f"] == want["n_f"]
    assert abs(got["c1"] - want["c1"]) < 1e-9 * want["c1"]
    assert abs(got["alias_estimate"] - want["alias"]) < 1e-6 * want["alias"]
    assert got["h"] == pytest.approx(L / want["n_f"])
    # cell list: edge >= r_c / reach, bricks divide the cell grid
    assert L / got["n_cells"] >= r_c / got["cell_reach"]
    assert got["n_cells"] % got["brick_cells"] == 0
    # local-part polynomials: the fewest terms whose fit error stays 100x
    # below the tolerance (scaled by the correction's size, about 3)
    assert got["si_fit_error"] < 1e-8 and got["near_fit_error"] <= 0.01 * eps * 3.1
    assert got["near_terms"] in (8, 9, 10, 12)


def test_planner_gaussian_split(lib):
    got = lib.esp_plan_query(14.413, 300_000, 1e-4, r_c=1.0, kernel=lib.ESP_KERNEL_GAUSS)
    want = oparams.plan(1e-4, 14.413, 1.0, kind="gauss")
    assert got["n_f"] == want["n_f"] and abs(got["alpha"] - math.log(1e4)) < 1e-12


@pytest.mark.parametrize("L,N,eps,r_c", [
    (14.4129, 300_000, 1e-4, 1.0),      # water 1e5 molecules
    (5.0, 300, 1e-3, 1.2),
    (10.0, 100_000, 1e-5, 1.0),
])
def test_planner_bspline_window_matches_oracle(lib, L, N, eps, r_c):
    got = lib.esp_plan_query(L, N, eps, r_c=r_c, kernel=lib.ESP_KERNEL_GAUSS, window=lib.ESP_WINDOW_BSPLINE)
    want = oparams.plan_bspline(eps, L, r_c)
    assert got["window"] == lib.ESP_WINDOW_BSPLINE
    assert got["P"] == want["P"] == 5 and got["n_f"] == want["n_f"]
    assert abs(got["alias_estimate"] - want["alias"]) < 1e-6 * want["alias"]
    # the B-spline comparator needs a finer grid than the PSWF window
    assert got["n_f"] > lib.esp_plan_query(L, N, eps, r_c=r_c)["n_f"]


def test_planner_fp64_fits_to_rounding(lib):
    got = lib.esp_plan_query(20.0, 1000, 1e-10, r_c=5.0, precision=lib.ESP_FP64)
    # (the near-field correction K reaches ~35 at this shape: 1e-12 is ~3e-14 relative)
    assert got["si_fit_error"] < 1e-13 and got["near_fit_error"] < 1e-12
    assert got["P"] == oparams.stencil_width(1e-10)


@pytest.mark.parametrize("kw,status", [
    (dict(L=10.0, N=100, tol=1e-4, r_c=5.0), 2),       # r_c >= L/2
    (dict(L=10.0, N=100, tol=0.5, r_c=1.0), 1),        # tolerance out of range
    (dict(L=-1.0, N=100, tol=1e-4, r_c=1.0), 1),       # bad box
    (dict(L=10.0, N=-5, tol=1e-4, r_c=1.0), 1),        # bad N
    (dict(L=10.0, N=100, tol=1e-4, r_c=1.0, P=20), 10),  # P beyond compiled range
    (dict(L=10.0, N=100, tol=1e-4, r_c=1.0, n_f=31), 1),  # odd grid
])
def test_invalid_arguments_rejected(lib, kw, status):
    L, N, tol = kw.pop("L"), kw.pop("N"), kw.pop("tol")
    with pytest.raises(lib.EspError) as exc:
        lib.esp_plan_query(L, N, tol, **kw)
    assert exc.value.status == status
    assert lib.esp_last_error()


def test_non_cubic_box_rejected(lib):
    box = lib.esp_box((ctypes.c_double * 3)(10.0, 10.0, 11.0))
    p = lib.esp_plan_params()
    o = lib.esp_plan_opts_init()
    st = lib.load_library().esp_plan_query(ctypes.byref(box), 10, 1e-4, ctypes.byref(o), ctypes.byref(p))
    assert st == 1 and "cubic" in lib.esp_last_error()


def test_null_arguments(lib):
    so = lib.load_library()
    assert so.esp_plan_query(None, 10, 1e-4, None, None) == 1
    assert so.esp_destroy(None) == 0
    assert so.esp_plan_info(None, None) == 1


def test_server_argument_checks_without_device(lib):
    so = lib.load_library()
    o = lib.esp_server_opts_init()
    assert o.max_inflight == 8 and o.precision == lib.ESP_FP32
    out = ctypes.c_void_p()
    assert so.esp_server_create(ctypes.byref(o), ctypes.byref(out)) == 1     # r_c missing
    assert "r_c" in lib.esp_last_error()
    assert so.esp_server_create(None, None) == 1
    assert so.esp_server_destroy(None) == 0


def test_autotune_argument_checks(lib):
    so = lib.load_library()
    box = lib.esp_box((ctypes.c_double * 3)(5.0, 5.0, 5.0))
    out = lib.esp_plan_opts()
    assert so.esp_autotune(ctypes.byref(box), 10, 1e-4, None, None, None, 0, 3, ctypes.byref(out), None) == 1


def test_planner_ik_and_virial_options(lib):
    L, N, eps = 14.4129, 300_000, 1e-4
    base = lib.esp_plan_query(L, N, eps, r_c=1.0)
    ik = lib.esp_plan_query(L, N, eps, r_c=1.0, diff=lib.ESP_DIFF_IK)
    vir = lib.esp_plan_query(L, N, eps, r_c=1.0, virial=1)
    assert base["diff"] == lib.ESP_DIFF_AD and ik["diff"] == lib.ESP_DIFF_IK
    assert vir["virial"] == 1 and base["virial"] == 0
    # the ik method holds three more grids and spectra
    extra = 3 * (ik["n_f"] ** 3 * 4 + ik["n_f"] ** 2 * (ik["n_f"] // 2 + 1) * 8)
    assert ik["device_bytes"] - base["device_bytes"] == extra
    assert ik["n_f"] == base["n_f"] and ik["P"] == base["P"]


@pytest.mark.parametrize("kw,status", [
    (dict(diff=2), 1),
    (dict(virial=2), 1),
    (dict(virial=1, near_variant=2), 10),         # the virial needs the default local part
    (dict(virial=1, near_variant=3), 10),
])
def test_planner_rejects_bad_ik_and_virial_options(lib, kw, status):
    with pytest.raises(lib.EspError) as exc:
        lib.esp_plan_query(10.0, 1000, 1e-4, r_c=1.0, **kw)
    assert exc.value.status == status


def test_md_and_exclusion_entry_points_without_device(lib):
    """esp_md_* and esp_set_exclusions reject NULL handles before any device
    work; the MD defaults are the oracle's water model (oracle/md.py)."""
    import ctypes
    import math
    from oracle import md
    so = lib.load_library()
    assert so.esp_set_exclusions(None, None, 0) == 1
    p = lib.esp_md_params()
    so.esp_md_params_init(ctypes.byref(p))
    m = md.WaterModel()
    assert (p.k_bond, p.r0, p.k_angle, p.lj_sigma, p.lj_epsilon, p.mass_O, p.mass_H) == \
        (m.k_bond, m.r0, m.k_angle, m.sigma, m.epsilon, m.m_O, m.m_H)
    assert abs(p.theta0 - m.theta0) < 1e-15 and p.dt == 0.0005
    out = ctypes.c_void_p()
    assert so.esp_md_create(None, ctypes.byref(p), None, None, ctypes.byref(out)) == 1
    assert so.esp_md_run(None, 1, None) == 1
    assert so.esp_md_state(None, None, None) == 1
    assert so.esp_md_destroy(None) == 0
    assert abs(lib.MD_PREFACTOR - 4 * math.pi * md.COULOMB_F) < 1e-9
