"""Brute-force periodic image sums for tiny systems (a pin for the Ewald oracle).

Eq. task sums q_j/(4 pi |r_i - r_j - nL|) over all images n. That lattice sum
is only conditionally convergent; summed over growing cubes of whole image
cells (n in [-R,R]^3, an isotropic shape like a sphere) it converges to the
"vacuum" result, which differs from the tinfoil (k = 0 dropped) result of
Ewald by the surface term of the cell dipole D = sum q_i r_i:

    E_vac = E_tin + |D|^2 / (6 V),      F_i,vac = F_i,tin - q_i D / (3 V).

``cube_sum`` returns the partial sums for one R; ``extrapolated`` removes the
leading 1/R^2 and 1/R^3 tails by Richardson extrapolation over R, 2R, 4R.
"""
from __future__ import annotations

import math

import numpy as np


def cube_sum(pos, q, L, R: int):
    """Energy and forces summed over image cells n in [-R,R]^3 (all pairs, j=i only for n != 0)."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    rng = np.arange(-R, R + 1)
    cells = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), axis=-1).reshape(-1, 3) * L
    energy = 0.0
    forces = np.zeros((n, 3))
    for i in range(n):
        d = pos[i][None, None, :] - pos[None, :, :] - cells[:, None, :]   # (cells, N, 3)
        r2 = np.sum(d * d, axis=-1)
        r2[cells.shape[0] // 2, i] = np.inf                               # n = 0, j = i
        r = np.sqrt(r2)
        energy += 0.5 * q[i] * float(np.sum(q[None, :] / (4.0 * math.pi * r)))
        forces[i] = q[i] * np.einsum("cj,cjk->k", q[None, :] / (4.0 * math.pi * r ** 3), d)
    return energy, forces


def extrapolated(pos, q, L, R: int = 16):
    """Richardson-extrapolated cube sums from R, 2R and 4R (tails ~ R^-2, R^-3)."""
    e1, f1 = cube_sum(pos, q, L, R)
    e2, f2 = cube_sum(pos, q, L, 2 * R)
    e4, f4 = cube_sum(pos, q, L, 4 * R)
    # eliminate the R^-2 term, then the R^-3 term
    e12, f12 = (4 * e2 - e1) / 3, (4 * f2 - f1) / 3
    e24, f24 = (4 * e4 - e2) / 3, (4 * f4 - f2) / 3
    return (8 * e24 - e12) / 7, (8 * f24 - f12) / 7


def surface_terms(pos, q, L):
    """(|D|^2/(6V), -q_i D/(3V)): vacuum minus tinfoil for isotropic summation."""
    D = np.sum(np.asarray(q)[:, None] * np.asarray(pos), axis=0)
    V = L ** 3
    return float(D @ D) / (6.0 * V), -np.asarray(q)[:, None] * D[None, :] / (3.0 * V)
