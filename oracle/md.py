"""MD loop workload for the FP64 CPU oracle (test infrastructure: only the
tests, the smoke check and the benchmark's CPU baseline use it).

The paper drives molecular dynamics with ESP inside MD packages and their
force fields (its lysozyme and LiTFSI runs); this workload keeps ESP for the
electrostatics and stands in a small synthetic force field for the rest
(flexible SPC/E-shaped water):

  * charges -0.8476 (O), +0.4238 (H); Coulomb f q_i q_j / r with
    f = 138.935458 kJ mol^-1 nm e^-2, computed by ESP (kernel 1/(4 pi r),
    so the ESP energy is scaled by 4 pi f) over all pairs and images;
  * intramolecular exclusions: the three pairs of a molecule interact only
    through the bonded terms, so their direct Coulomb f q_i q_j / r
    (minimum image) is subtracted from the ESP result, which holds it in
    full (local part plus smooth far part);
  * harmonic O-H bonds k_b (r - r0)^2 / 2 and H-O-H angle
    k_theta (theta - theta0)^2 / 2;
  * O-O Lennard-Jones 4 eps [(sigma/r)^12 - (sigma/r)^6] within r_c,
    shifted to zero at r_c;
  * velocity Verlet with a fixed step.

Units: nm, ps, amu, kJ/mol, e. Molecules are stored as consecutive (O, H, H)
triples. Plain NumPy, sized for small test systems.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import esp as oesp

COULOMB_F = 138.935458          # kJ mol^-1 nm e^-2
BOLTZMANN = 0.0083144626        # kJ mol^-1 K^-1


@dataclass
class WaterModel:
    k_bond: float = 345000.0              # kJ mol^-1 nm^-2
    r0: float = 0.1                       # nm
    k_angle: float = 383.0                # kJ mol^-1 rad^-2
    theta0: float = math.radians(109.47)
    sigma: float = 0.316557               # nm (O-O)
    epsilon: float = 0.650194             # kJ/mol (O-O)
    m_O: float = 15.9994                  # amu
    m_H: float = 1.008

    def masses(self, n_atoms: int) -> np.ndarray:
        return np.tile([self.m_O, self.m_H, self.m_H], n_atoms // 3)


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def bonded(pos: np.ndarray, L: float, model: WaterModel):
    """Bond and angle energy and forces of every (O, H, H) triple."""
    f = np.zeros_like(pos)
    o, h1, h2 = pos[0::3], pos[1::3], pos[2::3]
    energy = 0.0
    vecs = []
    for k, h in ((1, h1), (2, h2)):
        d = min_image(h - o, L)
        r = np.linalg.norm(d, axis=1)
        energy += 0.5 * model.k_bond * float(np.sum((r - model.r0) ** 2))
        fh = -(model.k_bond * (r - model.r0) / r)[:, None] * d       # on H
        f[k::3] += fh
        f[0::3] -= fh
        vecs.append((d, r))
    (u, ru), (v, rv) = vecs
    cos_t = np.clip(np.sum(u * v, axis=1) / (ru * rv), -1.0, 1.0)
    theta = np.arccos(cos_t)
    energy += 0.5 * model.k_angle * float(np.sum((theta - model.theta0) ** 2))
    # d theta / d u = -(v / (|u||v|) - cos u / |u|^2) / sin theta, likewise for v
    sin_t = np.sqrt(np.maximum(1.0 - cos_t * cos_t, 1e-300))
    de = model.k_angle * (theta - model.theta0)
    dtu = -(v / (ru * rv)[:, None] - (cos_t / ru ** 2)[:, None] * u) / sin_t[:, None]
    dtv = -(u / (ru * rv)[:, None] - (cos_t / rv ** 2)[:, None] * v) / sin_t[:, None]
    f1 = -de[:, None] * dtu
    f2 = -de[:, None] * dtv
    f[1::3] += f1
    f[2::3] += f2
    f[0::3] -= f1 + f2
    return energy, f


def lennard_jones_oxygen(pos: np.ndarray, L: float, r_c: float, model: WaterModel):
    """O-O Lennard-Jones within r_c (minimum image, r_c < L/2), energy
    shifted to zero at r_c."""
    o = pos[0::3]
    n = o.shape[0]
    f = np.zeros_like(pos)
    shift = 4.0 * model.epsilon * ((model.sigma / r_c) ** 12 - (model.sigma / r_c) ** 6)
    energy = 0.0
    for i in range(n - 1):
        d = min_image(o[i] - o[i + 1:], L)
        r2 = np.sum(d * d, axis=1)
        sel = r2 < r_c * r_c
        if not np.any(sel):
            continue
        d, r2 = d[sel], r2[sel]
        s6 = (model.sigma * model.sigma / r2) ** 3
        energy += float(np.sum(4.0 * model.epsilon * (s6 * s6 - s6) - shift))
        fm = (24.0 * model.epsilon * (2.0 * s6 * s6 - s6) / r2)[:, None] * d     # on i
        f[3 * i] += np.sum(fm, axis=0)
        j = 3 * (i + 1 + np.nonzero(sel)[0])
        np.add.at(f, j, -fm)
    return energy, f


def exclusion_pairs(n_atoms: int) -> np.ndarray:
    """(i, j) of the three intramolecular pairs of every molecule."""
    base = 3 * np.arange(n_atoms // 3)
    return np.concatenate([np.stack([base, base + 1], 1), np.stack([base, base + 2], 1),
                           np.stack([base + 1, base + 2], 1)])


def exclusion_correction(pos: np.ndarray, q: np.ndarray, L: float, pairs: np.ndarray):
    """Minus the direct Coulomb of the excluded pairs (minimum image), in the
    ESP kernel's units 1/(4 pi r): energy, potentials and forces."""
    i, j = pairs[:, 0], pairs[:, 1]
    d = min_image(pos[i] - pos[j], L)
    r = np.linalg.norm(d, axis=1)
    u = np.zeros(pos.shape[0])
    np.add.at(u, i, -q[j] / (4.0 * math.pi * r))
    np.add.at(u, j, -q[i] / (4.0 * math.pi * r))
    fm = (q[i] * q[j] / (4.0 * math.pi * r ** 3))[:, None] * d     # pair force on i
    f = np.zeros_like(pos)
    np.add.at(f, i, -fm)
    np.add.at(f, j, fm)
    energy = -float(np.sum(q[i] * q[j] / (4.0 * math.pi * r)))
    return energy, u, f


def coulomb(pos: np.ndarray, q: np.ndarray, L: float, p: oesp.ESPParams, pairs: np.ndarray | None):
    """ESP Coulomb with exclusions, in kJ/mol: (energy, forces)."""
    r = oesp.esp(pos, q, L, p)
    e, f = r["energy"], r["forces"]
    if pairs is not None and len(pairs):
        ex, _, fx = exclusion_correction(pos, q, L, pairs)
        e, f = e + ex, f + fx
    scale = 4.0 * math.pi * COULOMB_F
    return scale * e, scale * f


class WaterForceField:
    """Total potential energy and forces of the workload."""

    def __init__(self, q: np.ndarray, L: float, esp_params: oesp.ESPParams, r_c_lj: float,
                 model: WaterModel | None = None):
        self.q = np.asarray(q, dtype=np.float64)
        self.L = float(L)
        self.p = esp_params
        self.r_c_lj = r_c_lj
        self.model = model or WaterModel()
        self.pairs = exclusion_pairs(self.q.shape[0])

    def __call__(self, pos: np.ndarray):
        eb, fb = bonded(pos, self.L, self.model)
        el, fl = lennard_jones_oxygen(pos, self.L, self.r_c_lj, self.model)
        ec, fc = coulomb(pos, self.q, self.L, self.p, self.pairs)
        return eb + el + ec, fb + fl + fc


def maxwell_boltzmann(masses: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Velocities (nm/ps) at the temperature, zero total momentum."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(masses.shape[0], 3)) * np.sqrt(BOLTZMANN * temperature / masses)[:, None]
    v -= np.sum(masses[:, None] * v, axis=0) / np.sum(masses)
    return v


def velocity_verlet(pos: np.ndarray, vel: np.ndarray, masses: np.ndarray, dt: float, n_steps: int, forces):
    """n_steps of velocity Verlet: v += F dt / 2m, r += v dt, F(r), v += F dt / 2m.
    Returns dict(pos, vel, e_pot[n_steps + 1], e_kin[n_steps + 1])."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    inv_m = (1.0 / masses)[:, None]
    e, f = forces(pos)
    e_pot = [e]
    e_kin = [0.5 * float(np.sum(masses[:, None] * vel * vel))]
    for _ in range(n_steps):
        vel += 0.5 * dt * f * inv_m
        pos += dt * vel
        e, f = forces(pos)
        vel += 0.5 * dt * f * inv_m
        e_pot.append(e)
        e_kin.append(0.5 * float(np.sum(masses[:, None] * vel * vel)))
    return dict(pos=pos, vel=vel, e_pot=np.array(e_pot), e_kin=np.array(e_kin))
