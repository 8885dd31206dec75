"""Classical Ewald summation in FP64: the exact-result oracle.

Computes the quantities of Eq. task -- potentials u_i (the k = 0 mode dropped:
"tinfoil" boundary conditions), energy E = 1/2 sum q_i u_i and forces
F_i = -grad_i E -- for the kernel 1/(4 pi r), through the textbook erfc split
(Eq. ewalderf with splitting parameter g = 1/lambda):

  u_i = sum'_{j,n} q_j erfc(g r_ijn)/(4 pi r_ijn)                  (real space)
      + (1/V) sum_{k != 0} exp(-|xi|^2/(4 g^2))/|xi|^2 Re[exp(-i xi.r_i) S(xi)]
      - q_i g / (2 pi^{3/2})                                         (self)
      - Q / (4 V g^2)                              (background, if Q != 0)
  S(xi) = sum_j q_j exp(i xi.r_j),  xi = 2 pi k / L.

The real-space sum runs over the minimum image with cutoff r_cut < L/2 (so
erfc(g r_cut) <= acc); the k-space sum runs over the cube |k_a| <= K with K
chosen so exp(-xi^2/(4g^2)) <= acc at the cube face. erfc comes from SciPy.
Structure factors are assembled with matrix products over per-axis phase
tables (a library matmul used as a step; no reordering of the sum itself).
The virial W_ab = -dE/d eps_ab (homogeneous deformation of atoms and box)
uses the textbook forms: real-space pair terms, reciprocal
E_k [delta_ab - 2 (1 + xi^2/(4 g^2)) xi_a xi_b / xi^2], background E_bg delta_ab.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc, erfcinv


def ewald_parameters(L: float, acc: float = 1e-16) -> tuple[float, float, int]:
    """(g, r_cut, K) with erfc(g r_cut) = acc, r_cut = 0.49 L, Gaussian factor <= acc at K."""
    r_cut = 0.49 * L
    g = float(erfcinv(acc)) / r_cut
    xi_max = 2.0 * g * math.sqrt(-math.log(acc))
    K = int(math.ceil(xi_max * L / (2.0 * math.pi)))
    return g, r_cut, K


def _real_space(pos, q, L, g, r_cut, targets, chunk=256):
    """Minimum-image erfc sum for the target atoms (all j != i); also
    1/2 sum_i sum_j F_ij d_ij^T over the targets' pairs (virial)."""
    n_t = len(targets)
    u = np.zeros(n_t)
    f = np.zeros((n_t, 3))
    W = np.zeros((3, 3))
    for s in range(0, n_t, chunk):
        idx = targets[s:s + chunk]
        d = pos[idx, None, :] - pos[None, :, :]            # r_i - r_j
        d -= L * np.round(d / L)
        r2 = np.sum(d * d, axis=-1)
        self_mask = idx[:, None] == np.arange(pos.shape[0])[None, :]
        keep = (r2 < r_cut * r_cut) & ~self_mask
        r = np.sqrt(np.where(keep, r2, 1.0))
        ec = erfc(g * r)
        pot = np.where(keep, ec / (4.0 * math.pi * r), 0.0)
        u[s:s + chunk] = pot @ q
        # -dL/dr for L = erfc(g r)/(4 pi r), times (r_i - r_j)/r
        dl = (ec / r + 2.0 * g / math.sqrt(math.pi) * np.exp(-(g * r) ** 2)) / (4.0 * math.pi * r * r)
        coef = np.where(keep, dl, 0.0) * q[None, :]
        f[s:s + chunk] = q[idx, None] * np.einsum("ij,ijk->ik", coef, d)
        W += 0.5 * np.einsum("i,ij,ija,ijb->ab", q[idx], coef, d, d)
    return u, f, W


def _k_space(pos, q, L, g, K, targets, want_energy):
    """Explicit Fourier sum over k in the half space kx >= 0 (conjugate pairs folded)."""
    V = L ** 3
    ks = np.arange(-K, K + 1)
    tw = 2.0 * math.pi / L
    # per-axis phase tables exp(i xi_a r_a) for all atoms
    ex = np.exp(1j * tw * np.outer(pos[:, 0], np.arange(0, K + 1)))
    ey = np.exp(1j * tw * np.outer(pos[:, 1], ks))
    ez = np.exp(1j * tw * np.outer(pos[:, 2], ks))
    ky = ks[:, None] * np.ones((1, ks.size))
    kz = np.ones((ks.size, 1)) * ks[None, :]
    n_t = len(targets)
    u = np.zeros(n_t)
    f = np.zeros((n_t, 3))
    energy = 0.0
    W = np.zeros((3, 3))
    for kx in range(0, K + 1):
        k2 = kx * kx + ky * ky + kz * kz
        xi2 = (tw ** 2) * k2
        with np.errstate(divide="ignore"):
            amp = np.where(k2 > 0, np.exp(-xi2 / (4.0 * g * g)) / xi2, 0.0)
        # half-space weights: kx > 0 stands for +-k (factor 2); the kx = 0 plane
        # is summed in full with weight 1.
        wgt = 2.0 if kx > 0 else 1.0
        exy = ex[:, kx, None] * ey                           # (N, 2K+1)
        S = (exy * q[:, None]).T @ ez                        # S[ky, kz]
        if want_energy:
            ek = wgt * 0.5 / V * amp * np.abs(S) ** 2
            energy += float(np.sum(ek))
            # textbook reciprocal virial: E_k [delta - 2 (1 + xi^2/(4 g^2)) xi xi^T / xi^2]
            with np.errstate(divide="ignore", invalid="ignore"):
                fk = np.where(k2 > 0, ek * 2.0 * (1.0 + xi2 / (4.0 * g * g)) / k2, 0.0)
            kv = (kx * np.ones_like(ky), ky, kz)
            W += np.eye(3) * float(np.sum(ek))
            for a in range(3):
                for b in range(3):
                    W[a, b] -= float(np.sum(fk * kv[a] * kv[b]))
        # e^{-i xi.r_i} S summed against amp for the targets
        A = amp * S                                          # (2K+1, 2K+1)
        et = np.conj(exy[targets])                           # (n_t, 2K+1)
        ezt = np.conj(ez[targets])
        M = et @ A                                           # sum over ky
        Mky = et @ (A * ky)
        val = np.sum(M * ezt, axis=1)                        # sum over kz
        valx = kx * val
        valy = np.sum(Mky * ezt, axis=1)
        valz = np.sum(M * (ezt * ks[None, :]), axis=1)
        u += wgt / V * val.real
        # F_i = -q_i/V sum amp xi Im[e^{-i xi r_i} S]
        f[:, 0] += -wgt / V * tw * valx.imag
        f[:, 1] += -wgt / V * tw * valy.imag
        f[:, 2] += -wgt / V * tw * valz.imag
    f *= q[targets, None]
    return u, f, energy, W


def ewald(pos, q, L, acc: float = 1e-16, targets=None, g: float | None = None):
    """Classical Ewald potentials, forces (and energy when all atoms are targets).

    pos (N,3), q (N,), cubic box L. targets: indices to evaluate (default all).
    Returns dict(energy or None, potential, forces, g, r_cut, K, indices).
    """
    pos = np.mod(np.asarray(pos, dtype=np.float64), L)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    g0, r_cut, K = ewald_parameters(L, acc)
    if g is not None:
        # a caller-chosen g: keep r_cut = 0.49 L, so erfc(g r_cut) must stay small
        g0 = float(g)
        if erfc(g0 * r_cut) > acc:
            raise ValueError("g too small for a minimum-image real-space sum")
        K = int(math.ceil(2.0 * g0 * math.sqrt(-math.log(acc)) * L / (2.0 * math.pi)))
    all_atoms = targets is None
    tgt = np.arange(n) if all_atoms else np.asarray(targets, dtype=np.int64)
    u_r, f_r, w_r = _real_space(pos, q, L, g0, r_cut, tgt)
    u_k, f_k, e_k, w_k = _k_space(pos, q, L, g0, K, tgt, all_atoms)
    Q = float(np.sum(q))
    V = L ** 3
    u = u_r + u_k - q[tgt] * g0 / (2.0 * math.pi ** 1.5) - Q / (4.0 * V * g0 * g0)
    f = f_r + f_k
    energy = 0.5 * float(np.dot(q, u)) if all_atoms else None
    # virial W_ab = -dE/d eps_ab: real-space pairs, reciprocal modes, and the
    # background energy -Q^2/(8 V g^2) (proportional to 1/V); self term 0
    virial = w_r + w_k - Q * Q / (8.0 * V * g0 * g0) * np.eye(3) if all_atoms else None
    return dict(energy=energy, potential=u, forces=f, g=g0, r_cut=r_cut, K=K,
                indices=tgt, k_energy=e_k if all_atoms else None, virial=virial)
