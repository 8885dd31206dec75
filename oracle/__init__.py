"""CPU oracle for the ESP electrostatics solve -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy code written from the paper (Methods section:
Eqs. task, kernelsplitting, localpart, hS, spectralpart, spread...interp, pk,
pswf, pswfparameters, cem, cemparameters, Deltadef; Table 2). Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and nothing here imports the product.

Modules
  pswf    prolate spheroidal wave function psi_0^c and the splitting functions
  ewald   classical Ewald summation (erfc split, explicit k-space sum)
  images  brute-force spherical image sums for tiny systems
  esp     plain CPU ESP: five-step spectral part, local part, self/background
  params  the paper's parameter rules and Table 2
  metrics relative RMS force error (Eq. Deltadef)
  bspline centred cardinal B-spline window (the "Default" comparator)
  triclinic  Ewald and ESP on a general lattice (triclinic cells), virial
  md      the MD loop workload: flexible water, exclusions, velocity Verlet

Parity status: every function here is pinned by tests under ``tests/`` that
do not use the CUDA path (``-m "not gpu"``). The planner's calibration (how
far n_f is raised above the paper's minimum, which the paper leaves open) is
pinned by numbers the paper prints: its grid meets the force error and stays
within 1.25x of Eq. pswfparameters, and the "Default" comparator's measured
grid reproduces Table 2's R_default row (tests/test_oracle_rdefault.py).
"""
