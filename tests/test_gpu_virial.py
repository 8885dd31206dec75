"""Virial (opts.virial = 1, esp_last_virial) against the oracle.

FP64 plans equal the oracle's virial at the same parameters to 1e-9 of its
largest component; FP32 plans to 2e-5 (FP32 pair and mode sums); FP32
against the textbook Ewald virial within the tolerance's order; batches per
system; forces and energies do not change when the virial is on; a local
part kernel without the virial is refused.
"""
import numpy as np
import pytest

from oracle import esp as oesp
from oracle import ewald
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def gpu_virial(esp, s, eps, **opts):
    with esp.Plan(s.L, s.n, eps, virial=1, **opts) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e, f, u = p.compute()
        return e, f, esp.esp_last_virial(p.handle), p.info


def oracle_params(eps, info):
    kind = "pswf" if info["kernel"] == 0 else "gauss"
    return oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"], kind=kind,
                          alpha=info["alpha"] if kind == "gauss" else None,
                          diff="ik" if info["diff"] == 1 else "ad")


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


CASES = {
    "water500": (lambda: inputs.spce_water(500, seed=4), 1e-4, 1.0),
    "ions300_eps1e-5": (lambda: inputs.uniform_charges(300, 5.0, 7), 1e-5, 1.2),
    "electrolyte3000": (lambda: inputs.electrolyte(3000, seed=5), 1e-3, 0.9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_virial_fp64_and_fp32_match_oracle(esp, name):
    make, eps, r_c = CASES[name]
    s = make()
    for prec, bound in ((esp.ESP_FP64, 1e-9), (esp.ESP_FP32, 2e-5)):
        _, _, W, info = gpu_virial(esp, s, eps, r_c=r_c, precision=prec)
        ref = oesp.esp(s.pos, s.q, s.L, oracle_params(eps, info))["virial"]
        assert rel_max(W, ref) <= bound, (prec, rel_max(W, ref))


def test_virial_gaussian_split_and_non_neutral(esp):
    s = inputs.uniform_charges(200, 4.5, 9)
    q = s.q.copy()
    q[3] += 0.25                                   # background term on the diagonal
    s2 = inputs.System(s.pos, q, s.L)
    _, _, W, info = gpu_virial(esp, s2, 1e-4, r_c=1.1, precision=esp.ESP_FP64, kernel=esp.ESP_KERNEL_GAUSS,
                               allow_background=1)
    ref = oesp.esp(s2.pos, s2.q, s2.L, oracle_params(1e-4, info))["virial"]
    assert rel_max(W, ref) <= 1e-9


def test_virial_fp32_within_tolerance_of_ewald(esp):
    s = inputs.spce_water(1000, seed=11)
    _, _, W, _ = gpu_virial(esp, s, 1e-4, r_c=1.0)
    ref = ewald.ewald(s.pos, s.q, s.L, acc=1e-14)["virial"]
    assert rel_max(W, ref) <= 1e-3


def test_virial_leaves_forces_and_energy(esp):
    s = inputs.spce_water(800, seed=12)
    e1, f1, W, _ = gpu_virial(esp, s, 1e-4, r_c=1.0)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        e0, f0, _ = p.compute()
    assert np.sqrt(np.sum((f1 - f0) ** 2) / np.sum(f0 ** 2)) <= 5e-6
    assert abs(e1 - e0) <= 5e-6 * abs(e0)
    assert np.allclose(W, W.T)


def test_batch_virials_match_single_plans(esp):
    systems = inputs.electrolyte_batch([3000, 9000, 4000], seed=60)
    eps = 1e-4
    with esp.Batch([s.L for s in systems], [s.n for s in systems], eps, r_c=1.0,
                   precision=esp.ESP_FP64, virial=1) as b:
        pos, q = inputs.concat(systems)
        b.set_charges(q)
        for _ in range(2):                          # direct run, then the captured graph
            b.compute(pos)
        Wb = esp.esp_batch_last_virial(b.handle, len(systems))
        for i, s in enumerate(systems):
            info = b.info(i)
            ref = oesp.esp(s.pos, s.q, s.L, oracle_params(eps, info))["virial"]
            assert rel_max(Wb[i], ref) <= 1e-9


def test_virial_needs_the_default_local_part(esp):
    s = inputs.spce_water(300, seed=13)
    with pytest.raises(esp.EspError):
        esp.esp_plan(s.L, s.n, 1e-4, r_c=0.9, virial=1, near_variant=2)
    with esp.Plan(s.L, s.n, 1e-4, r_c=0.9) as p:
        p.set_charges(s.q)
        p.set_positions(s.pos)
        p.compute()
        with pytest.raises(esp.EspError):
            esp.esp_last_virial(p.handle)
