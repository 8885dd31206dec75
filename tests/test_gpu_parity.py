"""CUDA path (through the C-ABI) against the FP64 CPU oracle.

* FP64 plain mode vs the CPU ESP at the same parameters: relative RMS force
  error <= 1e-9, relative energy error <= 1e-10.
* FP32 production mode vs the CPU ESP at the same parameters: the FP32
  arithmetic bound FP32_PARITY, and vs classical Ewald: Delta <= tolerance.
* Edge cases: empty and ragged inputs, a single pair, non-neutral systems,
  non-finite coordinates, unwrapped coordinates, odd stencil widths.
"""
import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald, metrics
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu

# FP32 parity bound against the FP64 oracle at identical parameters: single
# precision weights (2^-24), O(P^3) FP32 grid accumulations and an FP32 FFT
# keep the relative RMS force error near 1e-6; 5e-6 leaves a 5x margin and is
# still 20x below the tightest production tolerance (1e-5) whose error budget
# it must not consume.
FP32_PARITY = 5e-6


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def gpu_solve(esp, s, eps, **opts):
    with esp.Plan(s.L, s.n, eps, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, u = p.compute()
        info = p.info
        ef, eg = esp.esp_last_spectral_energy(p.handle)
    return dict(energy=e, forces=f, potential=u, info=info, e_fourier=ef, e_gather=eg)


def oracle_same(s, eps, info, targets=None, pos=None):
    kind = "pswf" if info["kernel"] == 0 else "gauss"
    window = "bspline" if info["window"] == 1 else "pswf"
    p = oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"],
                       kind=kind, alpha=info["alpha"] if kind == "gauss" else None, window=window,
                       diff="ik" if info["diff"] == 1 else "ad")
    return oesp.esp(s.pos if pos is None else pos, s.q, s.L, p, targets)


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


CASES = {
    "uniform1000_L20": (lambda: inputs.uniform_charges(1000, 20.0, 2505), 1e-4, 5.0),
    "nacl8": (lambda: inputs.nacl_lattice(8), 1e-4, 2.0),
    "ions300_eps1e-5": (lambda: inputs.uniform_charges(300, 5.0, 7), 1e-5, 1.2),
    "ragged258_P7": (lambda: inputs.uniform_charges(258, 4.0, 3), 5e-5, 1.1),
    "water500": (lambda: inputs.spce_water(500, seed=4), 1e-4, 1.0),
    "electrolyte3000_eps1e-3": (lambda: inputs.electrolyte(3000, seed=5), 1e-3, 0.9),
}


def force_error(s, f, f_ref):
    """Relative RMS force error; for lattices whose forces vanish by symmetry
    the denominator is the nearest-neighbour pair force 1/(4 pi d^2) instead."""
    if s.name.startswith("nacl"):
        scale = 1.0 / (4 * np.pi * 0.25)
        return float(np.sqrt(np.mean(np.sum((f - f_ref) ** 2, axis=1)))) / scale
    return metrics.relative_rms_force_error(f, f_ref)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_matches_oracle(esp, name):
    make, eps, r_c = CASES[name]
    s = make()
    g = gpu_solve(esp, s, eps, r_c=r_c, precision=esp.ESP_FP64)
    ref = oracle_same(s, eps, g["info"])
    assert force_error(s, g["forces"], ref["forces"]) <= 1e-9
    assert abs(g["energy"] - ref["energy"]) <= 1e-10 * abs(ref["energy"])
    assert rel_rms(g["potential"], ref["potential"]) <= 1e-9
    # discrete energy identity 1/2 sum q u~ = 1/2 sum p |bh|^2
    assert abs(g["e_fourier"] - g["e_gather"]) <= 1e-11 * abs(g["e_fourier"])
    scale = max(abs(ref["fourier_energy"]), abs(ref["energy"]))
    assert abs(g["e_fourier"] - ref["fourier_energy"]) <= 1e-10 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_oracle(esp, name):
    make, eps, r_c = CASES[name]
    s = make()
    if name == "nacl8":
        # r_c = 2.0 is a lattice shell: pairs at exactly r = r_c, where the
        # truncated local force jumps by O(eps). FP64 decides r < r_c exactly
        # like the oracle; FP32 coordinates cannot, so the FP32 case uses a
        # cutoff between shells.
        r_c = 1.9
    g = gpu_solve(esp, s, eps, r_c=r_c, precision=esp.ESP_FP32)
    ref = oracle_same(s, eps, g["info"])
    assert force_error(s, g["forces"], ref["forces"]) <= FP32_PARITY
    # The FP32 spectral potential at each charge still holds its own smooth
    # self-interaction q_i chi(0)/(4 pi r_c), removed afterwards in FP64; its
    # rounding is relative to that part, which for random +-1 charges is far
    # larger than the (cancelling) total energy.
    e_self = 0.5 * float(np.sum(s.q * ref["self_term"]))
    assert abs(g["energy"] - ref["energy"]) <= FP32_PARITY * max(abs(ref["energy"]), abs(e_self))
    assert rel_rms(g["potential"], ref["potential"]) <= FP32_PARITY


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
@pytest.mark.parametrize("system", ["water", "electrolyte", "ions"])
def test_fp32_within_tolerance_of_ewald(esp, system, eps):
    if system == "water":
        s, r_c = inputs.spce_water(1000, seed=11), 1.0
    elif system == "electrolyte":
        s, r_c = inputs.electrolyte(3000, seed=12), 1.0
    else:
        s, r_c = inputs.uniform_charges(400, 6.0, 13), 1.5
    g = gpu_solve(esp, s, eps, r_c=r_c)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    delta = metrics.relative_rms_force_error(g["forces"], ref["forces"])
    assert delta <= eps, delta
    assert abs(g["energy"] - ref["energy"]) <= eps * abs(ref["energy"])


def test_nacl_madelung_fp32_and_fp64(esp):
    s = inputs.nacl_lattice(8)
    e_closed = -(s.n / 2) * 1.747564594633182 / (4 * np.pi * 0.5)
    g64 = gpu_solve(esp, s, 1e-10, r_c=1.9, precision=esp.ESP_FP64)
    assert abs(g64["energy"] - e_closed) <= 1e-9 * abs(e_closed)
    g32 = gpu_solve(esp, s, 1e-5, r_c=1.9)
    assert abs(g32["energy"] - e_closed) <= 1e-5 * abs(e_closed)
    assert np.max(np.abs(g32["potential"] + s.q * 0.27813354360823)) <= 1e-5 * 0.2781


def test_gaussian_split_variant(esp):
    s = inputs.spce_water(1000, seed=11)
    for prec, bound in ((esp.ESP_FP64, 1e-9), (esp.ESP_FP32, FP32_PARITY)):
        g = gpu_solve(esp, s, 1e-4, r_c=1.0, kernel=esp.ESP_KERNEL_GAUSS, precision=prec)
        ref = oracle_same(s, 1e-4, g["info"])
        assert metrics.relative_rms_force_error(g["forces"], ref["forces"]) <= bound
    ew = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    assert metrics.relative_rms_force_error(g["forces"], ew["forces"]) <= 1e-4


@pytest.mark.parametrize("P", [4, 5])
def test_bspline_window_matches_oracle(esp, P):
    """Gaussian split with the cardinal B-spline window (the comparator's
    spreading kernel): FP64 and FP32 against the oracle at the same
    parameters; odd P puts the stencil's knots on half-integers."""
    s = inputs.spce_water(1000, seed=11)
    for prec, bound in ((esp.ESP_FP64, 1e-9), (esp.ESP_FP32, FP32_PARITY)):
        g = gpu_solve(esp, s, 1e-4, r_c=1.0, kernel=esp.ESP_KERNEL_GAUSS, window=esp.ESP_WINDOW_BSPLINE,
                      P=P, precision=prec)
        assert g["info"]["window"] == esp.ESP_WINDOW_BSPLINE and g["info"]["P"] == P
        assert g["info"]["si_fit_error"] < (1e-6 if prec == esp.ESP_FP32 else 1e-12)
        ref = oracle_same(s, 1e-4, g["info"])
        assert metrics.relative_rms_force_error(g["forces"], ref["forces"]) <= bound
        assert abs(g["energy"] - ref["energy"]) <= 10 * bound * abs(ref["energy"])


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_bspline_window_within_tolerance_of_ewald(esp, eps):
    s = inputs.spce_water(1000, seed=11)
    g = gpu_solve(esp, s, eps, r_c=1.0, kernel=esp.ESP_KERNEL_GAUSS, window=esp.ESP_WINDOW_BSPLINE)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    assert metrics.relative_rms_force_error(g["forces"], ref["forces"]) <= eps
    assert abs(g["energy"] - ref["energy"]) <= eps * abs(ref["energy"])


@pytest.mark.parametrize("name", ["water500", "ions300_eps1e-5", "ragged258_P7"])
def test_ik_matches_oracle(esp, name):
    """ik force differentiation (three gradient grids) against the oracle at
    the same parameters, FP64 and FP32."""
    make, eps, r_c = CASES[name]
    s = make()
    for prec, bound in ((esp.ESP_FP64, 1e-9), (esp.ESP_FP32, FP32_PARITY)):
        g = gpu_solve(esp, s, eps, r_c=r_c, precision=prec, diff=esp.ESP_DIFF_IK)
        assert g["info"]["diff"] == esp.ESP_DIFF_IK
        ref = oracle_same(s, eps, g["info"])
        assert force_error(s, g["forces"], ref["forces"]) <= bound
        assert rel_rms(g["potential"], ref["potential"]) <= bound
        e_self = 0.5 * float(np.sum(s.q * ref["self_term"]))
        assert abs(g["energy"] - ref["energy"]) <= bound * max(abs(ref["energy"]), abs(e_self))


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-5])
def test_ik_within_tolerance_of_ewald(esp, eps):
    s = inputs.spce_water(1000, seed=11)
    g = gpu_solve(esp, s, eps, r_c=1.0, diff=esp.ESP_DIFF_IK)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)
    assert metrics.relative_rms_force_error(g["forces"], ref["forces"]) <= eps
    ad = gpu_solve(esp, s, eps, r_c=1.0)
    assert rel_rms(g["potential"], ad["potential"]) <= FP32_PARITY


def test_empty_system(esp):
    with esp.Plan(5.0, 0, 1e-4, r_c=1.0) as p:
        p.set_charges(np.zeros(0))
        p.set_positions(np.zeros((0, 3)))
        e, f, u = p.compute()
    assert e == 0.0 and f.shape == (0, 3)


def test_single_pair_and_non_neutral(esp):
    s = inputs.System(np.array([[1.0, 1.0, 1.0], [1.3, 1.1, 0.9]]), np.array([1.0, -1.0]), 4.0)
    g = gpu_solve(esp, s, 1e-6, r_c=1.5, precision=esp.ESP_FP64)
    ref = ewald.ewald(s.pos, s.q, s.L)
    assert metrics.relative_rms_force_error(g["forces"], ref["forces"]) <= 1e-6
    # a lone charge: neutralising background, Ewald's background convention
    one = inputs.System(np.array([[0.7, 2.0, 3.1]]), np.array([1.0]), 4.0)
    g1 = gpu_solve(esp, one, 1e-6, r_c=1.5, precision=esp.ESP_FP64)
    r1 = ewald.ewald(one.pos, one.q, one.L)
    assert abs(g1["energy"] - r1["energy"]) <= 1e-6 * abs(r1["energy"])
    assert np.max(np.abs(g1["forces"])) < 1e-6
    with pytest.raises(esp.EspError) as exc:
        gpu_solve(esp, one, 1e-6, r_c=1.5, allow_background=0)
    assert exc.value.status == 3


def test_nonfinite_position_reported(esp):
    s = inputs.uniform_charges(64, 4.0, 1)
    pos = s.pos.copy()
    pos[5, 1] = np.nan
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        with pytest.raises(esp.EspError) as exc:
            p.set_positions(pos)
        assert exc.value.status == 4
        p.set_positions(s.pos)            # recovers on valid input
        e, f, u = p.compute()
    assert np.all(np.isfinite(f))


def test_unwrapped_coordinates_and_translation(esp):
    s = inputs.uniform_charges(500, 6.0, 21)
    g = gpu_solve(esp, s, 1e-4, r_c=1.5)
    shifted = inputs.System(s.pos + s.L * np.array([3.0, -2.0, 7.0]), s.q, s.L)
    g2 = gpu_solve(esp, shifted, 1e-4, r_c=1.5)
    assert metrics.relative_rms_force_error(g2["forces"], g["forces"]) <= 1e-6
    moved = inputs.System(s.pos + np.array([0.37, 1.11, -2.5]), s.q, s.L)
    g3 = gpu_solve(esp, moved, 1e-4, r_c=1.5)
    assert metrics.relative_rms_force_error(g3["forces"], g["forces"]) <= 1e-4


def test_device_pointer_path_matches_host_path(esp):
    import torch
    s = inputs.spce_water(2000, seed=8)
    host = gpu_solve(esp, s, 1e-4, r_c=1.0)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    q = torch.tensor(s.q, device=dev)
    x = torch.tensor(s.pos, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)
    u = torch.zeros(s.n, dtype=torch.float64, device=dev)
    h = esp.esp_plan(s.L, s.n, 1e-4, r_c=1.0, stream=stream.cuda_stream)
    try:
        esp.esp_set_charges(h, q)
        for _ in range(2):
            esp.esp_set_positions(h, x)
            esp.esp_compute(h, e, f, u)
        esp.esp_synchronize(h)
    finally:
        esp.esp_destroy(h)
    torch.cuda.synchronize()
    # same arithmetic; only the order of floating-point atomics differs
    assert metrics.relative_rms_force_error(f.cpu().numpy(), host["forces"]) <= 1e-6
    assert abs(float(e.cpu()[0]) - host["energy"]) <= 1e-6 * abs(host["energy"])
    assert rel_rms(u.cpu().numpy(), host["potential"]) <= 1e-6
    # float32 inputs and outputs
    h = esp.esp_plan(s.L, s.n, 1e-4, r_c=1.0, stream=stream.cuda_stream)
    try:
        f32 = torch.zeros((s.n, 3), dtype=torch.float32, device=dev)
        esp.esp_set_charges(h, q.float())
        esp.esp_set_positions(h, x.float())
        esp.esp_compute(h, e, f32, None)
        esp.esp_synchronize(h)
    finally:
        esp.esp_destroy(h)
    torch.cuda.synchronize()
    torch.cuda.set_stream(torch.cuda.default_stream(dev))
    assert metrics.relative_rms_force_error(f32.double().cpu().numpy(), host["forces"]) <= 1e-5


def test_full_size_water_sampled(esp):
    """3e5-atom water box (1e5 SPC/E molecules, 1e-4, r_c = 1 nm) in the
    benchmark's configuration: sampled atoms vs the oracle ESP and Ewald."""
    s = inputs.spce_water(100_000, seed=2505)
    g = gpu_solve(esp, s, 1e-4, r_c=1.0)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(s.n, size=48, replace=False))
    ref = oracle_same(s, 1e-4, g["info"], targets=idx)
    assert metrics.relative_rms_force_error(g["forces"][idx], ref["forces"]) <= FP32_PARITY
    assert rel_rms(g["potential"][idx], ref["potential"]) <= FP32_PARITY
    ew = ewald.ewald(s.pos, s.q, s.L, acc=1e-10, targets=idx[:24])
    assert metrics.relative_rms_force_error(g["forces"][idx[:24]], ew["forces"]) <= 1e-4
    # properties at any size: the energy identity and finite outputs
    assert abs(g["e_fourier"] - g["e_gather"]) <= 1e-5 * abs(g["e_fourier"])
    assert np.all(np.isfinite(g["forces"]))


@pytest.mark.parametrize("kernel", [0, 1])
def test_forces_are_the_energy_gradient(esp, kernel):
    """FP64: central differences of the computed energy in a few coordinates
    equal -F (the AD forces are the exact gradient of the discrete energy;
    the PSWF local part is continuous at r_c)."""
    s = inputs.uniform_charges(120, 4.0, 61)
    h = 1e-5
    with esp.Plan(s.L, s.n, 1e-6, r_c=1.3, precision=esp.ESP_FP64, kernel=kernel) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        _, f, _ = p.compute()
        for i, a in [(0, 0), (7, 1), (55, 2), (119, 0)]:
            e = []
            for sgn in (1.0, -1.0):
                pos = s.pos.copy()
                pos[i, a] += sgn * h
                p.set_positions(pos)
                e.append(p.compute()[0])
            fd = -(e[0] - e[1]) / (2 * h)
            assert abs(fd - f[i, a]) <= 1e-6 * np.max(np.abs(f)), (i, a, fd, f[i, a])
