"""The MD loop (esp_md_*) on the GPU against the oracle's MD workload
(oracle/md.py) at the plan's ESP parameters.

* FP64 plans: positions, velocities and energies after 10 velocity-Verlet
  steps equal the oracle's trajectory (FP64 forces agree to ~1e-10, so the
  trajectories stay within ~1e-12 nm over 10 steps; bounds 1e-8 nm, 1e-7 of
  the potential energy, 1e-9 of the kinetic energy), for a box small enough
  that the Lennard-Jones kernel takes every pair and one that uses its cells.
* FP32 plans: the total energy stays within 2% of the kinetic energy over 40
  steps (the velocity-Verlet error of the flexible model at this step is a
  few tenths of a percent).
* Consecutive runs of growing length fill every energy row.
* Argument checks.
Collected last (test_zz_*): the newest GPU path.
"""
import numpy as np
import pytest

from oracle import esp as oesp
from oracle import md
from oracle import triclinic as tr
from paper_2505_09727_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def esp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_09727_gb300 import _build, esp as binding
    _build.build()
    return binding


def run_gpu(esp, s, v, eps, r_c, r_lj, n_steps, precision, dt=4e-4):
    with esp.Plan(s.L, s.n, eps, r_c=r_c, precision=precision, prefactor=esp.MD_PREFACTOR) as p:
        p.set_charges(s.q)
        info = p.info
        with esp.MD(p.handle, s.pos, v, dt=dt, lj_cutoff=r_lj) as sim:
            e = sim.run(n_steps)
            x, vel = sim.state()
    return e, x, vel, info


@pytest.mark.parametrize("n_mol,density,r_c,r_lj", [(8, 5.0, 0.55, 0.55), (300, 33.4, 0.9, 0.65)],
                         ids=["all_pairs", "cells"])
def test_fp64_trajectory_matches_the_oracle(esp, n_mol, density, r_c, r_lj):
    s = inputs.spce_water(n_mol, density=density, seed=31)
    masses = md.WaterModel().masses(s.n)
    v = md.maxwell_boltzmann(masses, 300.0, 5)
    eps = 1e-8
    e, x, vel, info = run_gpu(esp, s, v, eps, r_c, r_lj, 10, esp.ESP_FP64)
    p = oesp.ESPParams(eps, info["r_c"], info["P"], info["n_f"], c=info["c"], c1=info["c1"])
    ref = md.velocity_verlet(s.pos, v, masses, 4e-4, 10, md.WaterForceField(s.q, s.L, p, r_lj))
    assert np.max(np.abs(x - ref["pos"])) <= 1e-8
    assert np.max(np.abs(vel - ref["vel"])) <= 1e-6 * np.max(np.abs(ref["vel"]))
    e_pot = e[:, 0] + e[:, 1] + e[:, 2]
    assert np.max(np.abs(e_pot - ref["e_pot"])) <= 1e-7 * np.max(np.abs(ref["e_pot"]))
    assert np.max(np.abs(e[:, 3] - ref["e_kin"])) <= 1e-9 * np.max(ref["e_kin"])


def test_fp32_energy_is_conserved(esp):
    s = inputs.spce_water(300, seed=32)
    masses = md.WaterModel().masses(s.n)
    v = md.maxwell_boltzmann(masses, 300.0, 6)
    e, _, _, _ = run_gpu(esp, s, v, 1e-5, 0.9, 0.65, 40, esp.ESP_FP32)
    tot = e.sum(axis=1)
    assert np.all(np.isfinite(e))
    assert np.max(np.abs(tot - tot[0])) <= 0.02 * np.mean(e[:, 3])


def test_consecutive_runs_fill_every_energy_row(esp):
    """Runs of growing length on one MD state (each one reallocates the
    energy rows, possibly at the same address): every row of every run is
    written, and a run's first row carries the previous run's last one. A
    step graph replayed with a smaller row capacity than the run's left the
    last rows at zero."""
    s = inputs.spce_water(300, seed=11)
    v = inputs.water_velocities(300, 300.0, seed=11)
    with esp.Plan(s.L, s.n, 1e-4, r_c=0.9, prefactor=esp.MD_PREFACTOR) as p:
        p.set_charges(s.q)
        with esp.MD(p.handle, s.pos, v, dt=5e-4, lj_cutoff=0.6) as sim:
            prev = None
            for n in (3, 5, 2, 8):
                e = sim.run(n)
                assert e.shape == (n + 1, 4)
                # Coulomb, Lennard-Jones and kinetic energies are never zero here
                assert np.all(e[:, 0] != 0.0) and np.all(e[:, 2] != 0.0) and np.all(e[:, 3] > 0.0), (n, e)
                if prev is not None:
                    assert np.array_equal(e[0, :3], prev[-1, :3])
                prev = e


def test_md_arguments(esp):
    s = inputs.uniform_charges(10, 3.0, 1)
    with esp.Plan(s.L, s.n, 1e-4, r_c=1.0) as p:
        p.set_charges(s.q)
        with pytest.raises(esp.EspError) as exc:             # 10 atoms are no (O, H, H) molecules
            esp.MD(p.handle, s.pos, np.zeros_like(s.pos))
        assert exc.value.status == 1
    w = inputs.spce_water(30, seed=33)                       # L = 0.96 nm
    with esp.Plan(w.L, w.n, 1e-4, r_c=0.45) as p:
        p.set_charges(w.q)
        with pytest.raises(esp.EspError) as exc:             # cutoff beyond L/2
            esp.MD(p.handle, w.pos, np.zeros_like(w.pos), lj_cutoff=w.L)
        assert exc.value.status == 1
    c = inputs.spce_water_cell(30, seed=34)                  # cell heights 0.86 nm
    with esp.Plan(c.H, c.n, 1e-4, r_c=0.4) as p:
        p.set_charges(c.q)
        with pytest.raises(esp.EspError) as exc:
            esp.MD(p.handle, c.pos, np.zeros_like(c.pos), lj_cutoff=0.4)
        assert exc.value.status == 10


def test_destroy_clears_the_plan_exclusions(esp):
    """esp_md_create sets the intramolecular exclusions on the plan; after
    esp_md_destroy a compute on the same plan counts every pair again, as a
    fresh plan does."""
    s = inputs.spce_water(200, seed=35)
    v = np.zeros_like(s.pos)
    with esp.Plan(s.L, s.n, 1e-5, r_c=0.8, precision=esp.ESP_FP64) as p, \
            esp.Plan(s.L, s.n, 1e-5, r_c=0.8, precision=esp.ESP_FP64) as fresh:
        for q in (p, fresh):
            q.set_charges(s.q)
        with esp.MD(p.handle, s.pos, v, lj_cutoff=0.6) as sim:      # L = 1.82 nm
            sim.run(1)
        p.set_positions(s.pos)
        fresh.set_positions(s.pos)
        e, f, u = p.compute()
        e0, f0, u0 = fresh.compute()
    assert abs(e - e0) <= 1e-12 * abs(e0)
    assert np.max(np.abs(f - f0)) <= 1e-12 * np.max(np.abs(f0))
