"""Seeded synthetic inputs for the ESP electrostatics solve.

This module builds particle configurations only: positions in a cubic periodic
box and point charges. It holds none of the method's arithmetic, imports
nothing from the CUDA binding or from the CPU oracle, and is the one module
that both sides share (tests, benchmark and smoke run feed the same arrays to
the CUDA path and to the oracle).

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64), which
gives the same stream on x86_64 and aarch64.

Workload shapes follow the paper's test systems (Experimental design section;
SPC/E bulk water, aqueous electrolyte) at the paper's densities; the paper's
own input files are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# SPC/E geometry and charges (rigid 3-site water; Experimental design section).
SPCE_Q_O = -0.8476
SPCE_Q_H = +0.4238
SPCE_R_OH = 0.1            # nm
SPCE_ANGLE_DEG = 109.47
WATER_DENSITY = 33.4       # molecules / nm^3 (one molecule per 0.31 nm cube)


@dataclass
class System:
    """A periodic cubic system: ``pos`` (N,3) float64 in [0,L), ``q`` (N,) float64."""
    pos: np.ndarray
    q: np.ndarray
    L: float
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


def _wrap(pos: np.ndarray, L: float) -> np.ndarray:
    out = np.mod(pos, L)
    out[out >= L] -= L          # np.mod can return L for tiny negative inputs
    return out


def uniform_charges(n: int = 1000, L: float = 20.0, seed: int = 2505) -> System:
    """n/2 charges +1 and n/2 charges -1, uniform in [0,L)^3."""
    if n % 2:
        raise ValueError("n must be even for a neutral +-1 system")
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(n, 3))
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    return System(_wrap(pos, L), q, float(L), f"uniform{n}")


def nacl_lattice(cells: int = 8, a: float = 1.0) -> System:
    """Rock-salt lattice: ions at (i,j,k)*a/2, charge (-1)^(i+j+k).

    cells conventional cells per axis (8 ions each), nearest-neighbour
    distance a/2, box L = cells*a.
    """
    m = 2 * cells
    idx = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    pos = idx.astype(np.float64) * (a / 2.0)
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return System(pos, q, float(cells * a), f"nacl{cells}")


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly random rotation matrices from uniform unit quaternions."""
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    w, x, y, z = quat.T
    rot = np.empty((n, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return rot


def _water_sites(rng, oxygen: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Three sites per molecule (O, H, H) around the given O positions."""
    n = oxygen.shape[0]
    half = math.radians(SPCE_ANGLE_DEG) / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [SPCE_R_OH * math.sin(half), 0.0, SPCE_R_OH * math.cos(half)],
                     [-SPCE_R_OH * math.sin(half), 0.0, SPCE_R_OH * math.cos(half)]])
    rot = _random_rotations(rng, n)
    sites = oxygen[:, None, :] + np.einsum("nij,sj->nsi", rot, body)
    q = np.tile(np.array([SPCE_Q_O, SPCE_Q_H, SPCE_Q_H]), n)
    return sites.reshape(-1, 3), q


def spce_water(n_molecules: int = 100_000, density: float = WATER_DENSITY,
               jitter: float = 0.03, seed: int = 2505) -> System:
    """SPC/E-shaped water box.

    O atoms sit on an m^3 cubic lattice (m = ceil(n^(1/3)), spacing L/m; n sites
    chosen without replacement when m^3 > n), jittered uniformly by +-jitter nm
    per axis; each molecule gets a uniformly random orientation. L is set by the
    density: L = (n/density)^(1/3).
    """
    rng = np.random.default_rng(seed)
    L = (n_molecules / density) ** (1.0 / 3.0)
    m = int(math.ceil(round(n_molecules ** (1.0 / 3.0), 9)))
    while m ** 3 < n_molecules:
        m += 1
    sites = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    if m ** 3 > n_molecules:
        keep = np.sort(rng.choice(m ** 3, size=n_molecules, replace=False))
        sites = sites[keep]
    oxygen = (sites + 0.5) * (L / m) + rng.uniform(-jitter, jitter, size=(n_molecules, 3))
    pos, q = _water_sites(rng, oxygen)
    return System(_wrap(pos, L), q, float(L), f"water{n_molecules}")


@dataclass
class CellSystem:
    """A periodic system in a triclinic cell: ``H`` (3,3) has the cell vectors
    a, b, c as columns (a = (ax,0,0), b = (bx,by,0)); ``pos`` (N,3) float64."""
    pos: np.ndarray
    q: np.ndarray
    H: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


def truncated_octahedron(volume: float) -> np.ndarray:
    """Cell vectors (columns) of a truncated octahedron of the given volume:
    nearest-image distance d, a = (d,0,0), b = (d/3, 2 sqrt2 d/3, 0),
    c = (-d/3, sqrt2 d/3, sqrt6 d/3), volume (4 sqrt3 / 9) d^3."""
    d = (volume * 9.0 / (4.0 * math.sqrt(3.0))) ** (1.0 / 3.0)
    return np.array([[d, d / 3.0, -d / 3.0],
                     [0.0, 2.0 * math.sqrt(2.0) * d / 3.0, math.sqrt(2.0) * d / 3.0],
                     [0.0, 0.0, math.sqrt(6.0) * d / 3.0]])


def spce_water_cell(n_molecules: int, H: np.ndarray | None = None, density: float = WATER_DENSITY,
                    jitter: float = 0.03, seed: int = 2505) -> CellSystem:
    """SPC/E-shaped water in a triclinic cell (default: a truncated octahedron
    of volume n / density). O atoms sit on an m^3 lattice of fractional
    coordinates ((i + 1/2)/m per axis, n sites chosen without replacement),
    mapped through H and jittered by +-jitter nm per Cartesian axis; each
    molecule gets a uniformly random orientation."""
    rng = np.random.default_rng(seed)
    if H is None:
        H = truncated_octahedron(n_molecules / density)
    H = np.asarray(H, dtype=np.float64)
    m = int(math.ceil(round(n_molecules ** (1.0 / 3.0), 9)))
    while m ** 3 < n_molecules:
        m += 1
    sites = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    if m ** 3 > n_molecules:
        keep = np.sort(rng.choice(m ** 3, size=n_molecules, replace=False))
        sites = sites[keep]
    oxygen = ((sites + 0.5) / m) @ H.T + rng.uniform(-jitter, jitter, size=(n_molecules, 3))
    pos, q = _water_sites(rng, oxygen)
    return CellSystem(pos, q, H, f"water{n_molecules}_cell")


def water_velocities(n_molecules: int, temperature: float = 300.0, seed: int = 2505,
                     mass_o: float = 15.9994, mass_h: float = 1.008) -> np.ndarray:
    """Maxwell-Boltzmann velocities (nm/ps) of (O, H, H) molecules at the
    temperature (K), total momentum removed."""
    rng = np.random.default_rng(seed)
    m = np.tile([mass_o, mass_h, mass_h], n_molecules)
    v = rng.normal(size=(m.shape[0], 3)) * np.sqrt(0.0083144626 * temperature / m)[:, None]
    return v - np.sum(m[:, None] * v, axis=0) / np.sum(m)


def electrolyte(n_atoms: int, density: float = 100.0, ion_fraction: float = 0.006,
                seed: int = 9727, jitter: float = 0.03) -> System:
    """Neutral +-1 ions plus SPC/E-shaped water at a total atom density.

    round(ion_fraction*n_atoms) ion pairs; the rest are water molecules (the
    water atom count is a multiple of 3). Ions and water oxygens occupy
    distinct sites of a cubic lattice with one site per molecule or ion.
    L = (N/density)^(1/3).
    """
    rng = np.random.default_rng(seed)
    n_pairs = max(1, int(round(ion_fraction * n_atoms)))
    n_water = max(1, (n_atoms - 2 * n_pairs) // 3)
    n_total = 2 * n_pairs + 3 * n_water
    L = (n_total / density) ** (1.0 / 3.0)
    n_sites = 2 * n_pairs + n_water
    m = int(math.ceil(n_sites ** (1.0 / 3.0)))
    while m ** 3 < n_sites:
        m += 1
    grid = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                                indexing="ij"), axis=-1).reshape(-1, 3)
    pick = rng.choice(m ** 3, size=n_sites, replace=False)
    centres = (grid[pick] + 0.5) * (L / m) + rng.uniform(-jitter, jitter, size=(n_sites, 3))
    ions = centres[: 2 * n_pairs]
    ion_q = np.concatenate([np.ones(n_pairs), -np.ones(n_pairs)])
    wpos, wq = _water_sites(rng, centres[2 * n_pairs:])
    pos = np.concatenate([ions, wpos])
    q = np.concatenate([ion_q, wq])
    return System(_wrap(pos, L), q, float(L), f"electrolyte{n_total}")


def batch_sizes(n_systems: int = 64, lo: float = 3e3, hi: float = 2e5,
                seed: int = 9727) -> np.ndarray:
    """Atom counts log-uniform in [lo, hi] (batched-replica workload)."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_systems))).astype(np.int64)


def perturb(system: System, sigma: float, seed: int) -> System:
    """Gaussian step of std sigma per coordinate, wrapped (serving requests)."""
    rng = np.random.default_rng(seed)
    pos = _wrap(system.pos + rng.normal(0.0, sigma, size=system.pos.shape), system.L)
    return System(pos, system.q.copy(), system.L, system.name)


def electrolyte_batch(sizes, seed: int = 9727) -> list[System]:
    """One electrolyte box per atom count; system s uses seed + s."""
    return [electrolyte(int(n), seed=seed + s) for s, n in enumerate(sizes)]


def concat(systems: list[System]) -> tuple[np.ndarray, np.ndarray]:
    """Positions (sum N, 3) and charges (sum N,) of systems in order."""
    return (np.ascontiguousarray(np.concatenate([s.pos for s in systems])),
            np.ascontiguousarray(np.concatenate([s.q for s in systems])))
