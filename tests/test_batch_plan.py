"""Host planning of batches (no GPU): esp_batch_query.

A batch shares one SI kernel (P, c1) and groups grids into FFT-friendly
sizes; each system must still meet the tolerance, i.e. its aliasing estimate
(Eq. errorformula) stays at or below eps/2 as for a single plan.
"""
import pytest

from paper_2505_09727_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09727_gb300 import _build, esp
    _build.build()
    return esp


def boxes_of(sizes):
    return [(int(n) / 100.0) ** (1.0 / 3.0) for n in sizes]


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_batch_plan_meets_tolerance_with_common_kernel(lib, eps):
    sizes = inputs.batch_sizes(16, seed=5)
    L = boxes_of(sizes)
    got = lib.esp_batch_query(L, sizes, eps, r_c=1.0)
    assert len(got) == len(sizes)
    assert len({g["P"] for g in got}) == 1
    assert len({round(g["c1"], 12) for g in got}) == 1
    for g, Ls, n in zip(got, L, sizes):
        assert g["N"] == n and g["L"] == pytest.approx(Ls)
        assert g["alias_estimate"] <= 0.5 * eps
        alone = lib.esp_plan_query(Ls, n, eps, r_c=1.0, c1=g["c1"])
        assert g["n_f"] >= alone["n_f"]
        assert g["n_f"] <= 1.25 * alone["n_f"] + 2     # next ladder size, not more
    # similar sizes share grids: far fewer distinct grids than systems
    assert len({g["n_f"] for g in got}) <= len(sizes) // 2


def test_batch_of_one_equals_single_plan_when_on_ladder(lib):
    s = lib.esp_plan_query(3.0, 2700, 1e-4, r_c=1.0)
    b = lib.esp_batch_query([3.0], [2700], 1e-4, r_c=1.0)[0]
    assert b["c1"] == pytest.approx(s["c1"]) and b["P"] == s["P"]
    assert b["n_f"] >= s["n_f"]


@pytest.mark.parametrize("kw,status", [
    (dict(r_c=0.0), 1),                  # a batch needs an explicit r_c
    (dict(r_c=2.0), 2),                  # r_c >= L/2 for the small box
])
def test_batch_query_rejects(lib, kw, status):
    with pytest.raises(lib.EspError) as exc:
        lib.esp_batch_query([3.0, 6.0], [2700, 21600], 1e-4, **kw)
    assert exc.value.status == status
    assert "system 0" in lib.esp_last_error() or status == 1
