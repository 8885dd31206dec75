"""esp_local_part_static: the local part without device allocation.

The entry point serves callers that cannot call cudaMalloc; its working
memory is one static device array shared by every call. It must agree with
the plan-based entry point (esp_plan + esp_compute) on two calls in a row,
so the state a call leaves in the shared array cannot leak into the next.

Two comparisons with the plan-based path on the same inputs:
  * PSWF split, FP64 and FP32: the energy equals the plan-based total minus
    its spectral energy (esp_last_spectral_energy);
  * Gaussian split with alpha = 1e-12: the spectral part vanishes
    identically (exp(-kappa^2/(4 alpha)) underflows to 0 for every k != 0), so
    the plan-based energy, forces and potential are the local part alone.
This file is collected after every other test file, so a run that stops at
the first failure has already run the rest.
"""
import numpy as np
import pytest

from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_PARITY = 5e-6          # the FP32 bound of the GPU parity tests


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp
    _build.build()
    return esp


def plan_based(esp, s, eps, **opts):
    # the static entry point runs the one-thread-per-atom local part; the plan
    # uses the same kernel, so both decide r < r_c with the same FP32 rounding
    # (with alpha = 1e-12 the truncated bare Coulomb force jumps at r_c)
    with esp.Plan(s.L, s.n, eps, near_variant=1, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, u = p.compute()
        e_fourier, _ = esp.esp_last_spectral_energy(p.handle)
    return e, f, u, e_fourier


def static_call(esp, s, eps, **opts):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        x = torch.tensor(s.pos, device=dev)
        q = torch.tensor(s.q, device=dev)
        e = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        f = torch.full((s.n, 3), np.nan, dtype=torch.float64, device=dev)
        u = torch.full((s.n,), np.nan, dtype=torch.float64, device=dev)
    stream.synchronize()
    esp.esp_local_part_static(s.L, s.n, eps, x, q, e, f, u, stream=stream.cuda_stream, **opts)
    stream.synchronize()
    return float(e.cpu()[0]), f.cpu().numpy(), u.cpu().numpy()


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


@pytest.mark.parametrize("precision,bound", [(1, 1e-10), (0, FP32_PARITY)])
def test_energy_matches_plan_minus_spectral_part(lib, precision, bound):
    s = inputs.spce_water(2000, seed=31)
    e_tot, _, _, e_fourier = plan_based(lib, s, 1e-4, r_c=1.0, precision=precision)
    want = e_tot - e_fourier
    for _ in range(2):                                   # two calls in a row
        e, f, u = static_call(lib, s, 1e-4, r_c=1.0, precision=precision)
        assert abs(e - want) <= bound * abs(e_tot), (e, want)
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(u))


@pytest.mark.parametrize("precision,bound", [(1, 1e-10), (0, FP32_PARITY)])
def test_matches_plan_when_spectral_part_vanishes(lib, precision, bound):
    s = inputs.electrolyte(5000, seed=32)
    # the same cell list on both sides (reach and one-cell bricks fixed), so
    # both decide r < r_c from the same FP32 coordinates
    opts = dict(r_c=1.0, kernel=lib.ESP_KERNEL_GAUSS, alpha=1e-12, precision=precision, cell_reach=3,
                brick_cells=1)
    e_ref, f_ref, u_ref, e_fourier = plan_based(lib, s, 1e-4, **opts)
    assert e_fourier == 0.0
    results = [static_call(lib, s, 1e-4, **opts) for _ in range(2)]   # two calls in a row
    for e, f, u in results:
        assert rel_rms(f, f_ref) <= bound
        assert rel_rms(u, u_ref) <= bound
        assert abs(e - e_ref) <= bound * abs(e_ref)


def test_rejects_systems_beyond_the_static_size(lib):
    s = inputs.spce_water(40_000, seed=33)              # 120k atoms > the array's limit
    with pytest.raises(lib.EspError) as exc:
        static_call(lib, s, 1e-4, r_c=1.0)
    assert exc.value.status == 10
    assert "static array" in lib.esp_last_error()


def test_nonfinite_position_is_reported(lib):
    """A NaN position is zeroed by the ingest and flagged; the call waits for
    its kernels and returns ESP_ERR_NONFINITE instead of a wrong result."""
    s = inputs.spce_water(500, seed=34)
    s.pos[17, 1] = np.nan
    with pytest.raises(lib.EspError) as exc:
        static_call(lib, s, 1e-4, r_c=0.7)
    assert exc.value.status == 4          # ESP_ERR_NONFINITE
    # the shared array is usable again on the next call
    s.pos[17, 1] = 0.5
    e, f, u = static_call(lib, s, 1e-4, r_c=0.7)
    assert np.isfinite(e) and np.all(np.isfinite(f)) and np.all(np.isfinite(u))


def test_rejects_buffers_that_are_not_device_float64(lib):
    """Host memory, a wrong dtype or a wrong length is an argument error,
    raised before anything is launched."""
    import torch
    s = inputs.spce_water(200, seed=35)
    dev = torch.device("cuda:0")
    x = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, device=dev)
    with pytest.raises(TypeError):
        lib.esp_local_part_static(s.L, s.n, 1e-4, torch.tensor(s.pos), q, r_c=0.7)
    with pytest.raises(TypeError):
        lib.esp_local_part_static(s.L, s.n, 1e-4, x.float(), q, r_c=0.7)
    with pytest.raises(ValueError):
        lib.esp_local_part_static(s.L, s.n, 1e-4, x[:-1], q, r_c=0.7)
    # a raw host address reaches the C entry, which refuses it
    host = np.ascontiguousarray(s.pos)
    with pytest.raises(lib.EspError) as exc:
        lib.esp_local_part_static(s.L, s.n, 1e-4, host.ctypes.data, q, r_c=0.7)
    assert exc.value.status == 1          # ESP_ERR_INVALID_ARG
