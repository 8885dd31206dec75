"""Triclinic periodic boxes for the FP64 CPU oracle (test infrastructure).

The paper's non-orthorhombic benchmarks (truncated-octahedral and
rhombic-dodecahedral boxes, Table 1) need the periodic Coulomb sum of Eq. task
on a general lattice. The box is the matrix H whose columns are the cell
vectors a = (a_x, 0, 0), b = (b_x, b_y, 0), c = (c_x, c_y, c_z); a position r
has fractional coordinates s = H^-1 r, images r + H n (n integer), volume
V = det H, and reciprocal vectors xi(m) = 2 pi H^-T m (m integer).

* `ewald`: classical Ewald on that lattice (erfc split; the real-space sum
  over every image within r_cut, the reciprocal sum over every m with
  |xi| <= xi_max), the exact-result reference.
* `esp`: the ESP steps with the grid laid over the cell (reading for
  triclinic boxes): spread and interpolation on the n_f^3 grid of
  fractional coordinates t = s n_f with the same P-point SI kernel per axis;
  the influence function of Eq. pk with |xi(k)| from the metric,
  p_k = Shat(|xi(k)|) / (V Phi(th_x)^2 Phi(th_y)^2 Phi(th_z)^2); forces from
  the fractional gradient, grad_r = H^-T grad_s; the local part over all
  images within r_c. For H = L I every step is the cubic oracle's.

Plain NumPy; image and mode loops are explicit, sized for small test systems.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def box_matrix(a, b, c) -> np.ndarray:
    """H with columns a, b, c (a along x, b in the xy plane)."""
    H = np.array([a, b, c], dtype=np.float64).T
    if abs(H[1, 0]) > 0 or abs(H[2, 0]) > 0 or abs(H[2, 1]) > 0:
        raise ValueError("cell vectors must be a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)")
    return H


def heights(H) -> np.ndarray:
    """Distances between opposite faces of the cell (V / face area)."""
    V = abs(np.linalg.det(H))
    a, b, c = H[:, 0], H[:, 1], H[:, 2]
    return np.array([V / np.linalg.norm(np.cross(b, c)), V / np.linalg.norm(np.cross(c, a)),
                     V / np.linalg.norm(np.cross(a, b))])


def fractional(pos, H) -> np.ndarray:
    s = np.linalg.solve(H, np.asarray(pos, dtype=np.float64).T).T
    return s - np.floor(s)


def _image_shifts(H, r_max):
    """Integer n that can give |H (ds - n)| < r_max for a fractional
    difference ds in (-1, 1)^3: the a-th fractional component of a vector is
    at most its length over the height h_a, so |ds_a - n_a| < r_max / h_a and
    |n_a| <= floor(r_max / h_a) + 1."""
    h = heights(H)
    K = [int(math.floor(r_max / h[a])) + 1 for a in range(3)]
    return np.array(list(itertools.product(range(-K[0], K[0] + 1), range(-K[1], K[1] + 1),
                                           range(-K[2], K[2] + 1))), dtype=np.float64)


def _pairs_within(pos, H, r_max):
    """(i, j, d) for every ordered pair and image with 0 < |d| < r_max,
    d = r_i - r_j - H n. The positions are first wrapped into the cell (a
    lattice shift of one atom permutes its images and changes no d), so the
    fractional differences lie in (-1, 1)^3 as _image_shifts assumes."""
    pos = fractional(pos, H) @ H.T
    shifts = _image_shifts(H, r_max) @ H.T
    out_i, out_j, out_d = [], [], []
    for i in range(pos.shape[0]):
        d = pos[i][None, None, :] - pos[None, :, :] - shifts[:, None, :]     # (images, N, 3)
        r = np.sqrt(np.sum(d * d, axis=-1))
        sel = (r < r_max) & (r > 0.0)
        k, j = np.nonzero(sel)
        out_i.append(np.full(len(j), i))
        out_j.append(j)
        out_d.append(d[k, j])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_d)


def ewald(pos, q, H, g: float, r_cut: float, xi_max: float):
    """Classical Ewald energy, potentials and forces on the lattice H (kernel
    1/(4 pi r), k = 0 mode dropped, neutralising background for Q != 0).
    Returns dict(energy, potential, forces)."""
    from scipy.special import erfc
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    V = abs(np.linalg.det(H))
    u = np.zeros(n)
    f = np.zeros((n, 3))
    i, j, d = _pairs_within(pos, H, r_cut)
    r = np.sqrt(np.sum(d * d, axis=1))
    np.add.at(u, i, q[j] * erfc(g * r) / (4.0 * math.pi * r))
    mag = (erfc(g * r) / r + 2.0 * g / math.sqrt(math.pi) * np.exp(-(g * r) ** 2)) / (4.0 * math.pi * r * r)
    np.add.at(f, i, (q[i] * q[j] * mag)[:, None] * d)
    # reciprocal space: all m != 0 with |xi(m)| <= xi_max
    Hinv_T = np.linalg.inv(H).T
    h = heights(H)
    M = [int(math.ceil(xi_max * h[a] / (2.0 * math.pi))) + 1 for a in range(3)]
    ms = np.array(list(itertools.product(range(-M[0], M[0] + 1), range(-M[1], M[1] + 1), range(-M[2], M[2] + 1))),
                  dtype=np.float64)
    xi = 2.0 * math.pi * ms @ Hinv_T.T
    x2 = np.sum(xi * xi, axis=1)
    keep = (x2 > 0) & (x2 <= xi_max * xi_max)
    xi, x2 = xi[keep], x2[keep]
    amp = np.exp(-x2 / (4.0 * g * g)) / x2 / V
    phase = pos @ xi.T                                            # (N, modes)
    S = (q[:, None] * np.exp(1j * phase)).sum(axis=0)
    val = np.exp(-1j * phase) * S[None, :]
    u += (val.real * amp[None, :]).sum(axis=1)
    f -= q[:, None] * ((val.imag * amp[None, :]) @ xi)            # grad of Re(e^{-i xi.r} S) is xi Im(...)
    Q = float(np.sum(q))
    u += -q * g / (2.0 * math.pi ** 1.5) - Q / (4.0 * V * g * g)
    return dict(energy=0.5 * float(np.dot(q, u)), potential=u, forces=f)


def ewald_converged(pos, q, H, acc: float = 1e-14):
    """Ewald with g, r_cut, xi_max chosen so both truncations are below acc."""
    from scipy.special import erfcinv
    r_cut = 0.49 * float(np.min(heights(H)))
    g = float(erfcinv(acc)) / r_cut
    xi_max = 2.0 * g * math.sqrt(-math.log(acc))
    return ewald(pos, q, H, g, r_cut, xi_max)


def esp(pos, q, H, split, window, n_f: int, r_c: float, virial: bool = False):
    """ESP on the lattice H (module docstring). split, window: the oracle's
    splitting function and SI kernel (oracle.pswf / oracle.bspline).
    Returns dict(energy, potential, forces, fourier_energy, virial).

    virial: W_ab = -dE/d eps_ab under r -> (1 + eps) r, H -> (1 + eps) H (the
    grid deforms with the cell, so b_l and the grid-unit Phi stay; xi(k)
    becomes (1 + eps)^-T xi and V becomes V (1 + tr eps)): the spectral part
    sum_k 1/2 |bh_k|^2 [p_k delta_ab + p'_k xi_a xi_b / |xi|^2] with
    p'_k = (r_c |xi| chihat'(r_c |xi|) - 2 chihat(r_c |xi|)) / (|xi|^2 V Phi^6),
    averaged over the two aliases of a mode with a component -n_f/2 (the
    real part of the inverse transform applies that average to the energy,
    so its derivative carries it too); the local part 1/2 sum_ij F_ij
    d_ij^T; the background E_bg delta_ab."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    if not r_c < 0.5 * float(np.min(heights(H))):
        raise ValueError("r_c must be below half the smallest cell height")
    V = abs(np.linalg.det(H))
    P = window.P
    # 1. spread on the fractional grid
    t = fractional(pos, H) * n_f
    l0 = np.ceil(t - 0.5 * P).astype(np.int64)
    l = l0[:, :, None] + np.arange(P)[None, None, :]
    w = window.phi(t[:, :, None] - l)
    dw = window.dphi(t[:, :, None] - l) * n_f                      # d/ds
    idx = np.mod(l, n_f)
    b = np.zeros(n_f ** 3)
    for a_, b_, c_ in itertools.product(range(P), repeat=3):
        lin = (idx[:, 0, a_] * n_f + idx[:, 1, b_]) * n_f + idx[:, 2, c_]
        b += np.bincount(lin, weights=q * w[:, 0, a_] * w[:, 1, b_] * w[:, 2, c_], minlength=n_f ** 3)
    b = b.reshape(n_f, n_f, n_f)
    # 2.-4. transform, influence from the metric, back
    bh = np.fft.ifftn(b) * n_f ** 3
    k = np.fft.fftfreq(n_f, d=1.0 / n_f)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), axis=-1)      # (n, n, n, 3)
    xi = 2.0 * math.pi * K @ np.linalg.inv(H)                       # rows: xi = 2 pi H^-T k
    xin = np.sqrt(np.sum(xi * xi, axis=-1))
    Phi = window.Phi(2.0 * math.pi * k / n_f)
    den = V * (Phi[:, None, None] * Phi[None, :, None] * Phi[None, None, :]) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        shat = np.where(xin > 0, split.chihat(r_c * xin) / xin ** 2, 0.0)
    p = shat / den
    fourier_energy = 0.5 * float(np.sum(p * np.abs(bh) ** 2))
    W = np.zeros((3, 3))
    if virial:
        a = 0.5 * np.abs(bh) ** 2
        for alias in (K, np.where(K == -(n_f // 2), n_f // 2, K)):
            xa = 2.0 * math.pi * alias @ np.linalg.inv(H)
            x = np.sqrt(np.sum(xa * xa, axis=-1))
            with np.errstate(divide="ignore", invalid="ignore"):
                pa = np.where(x > 0, split.chihat(r_c * x) / x ** 2, 0.0) / den
                pv = np.where(x > 0, (r_c * x * split.dchihat(r_c * x) - 2.0 * split.chihat(r_c * x)) / x ** 2,
                              0.0) / den
                t = np.where(x > 0, a * pv / x ** 2, 0.0)
            W += 0.5 * np.eye(3) * float(np.sum(a * pa))
            W += 0.5 * np.einsum("xyza,xyzb,xyz->ab", xa, xa, t)
    cgrid = np.fft.fftn(p * bh).real
    # 5. interpolate potential and fractional gradient, grad_r = H^-T grad_s
    u = np.zeros(n)
    gs = np.zeros((n, 3))
    for a_, b_, c_ in itertools.product(range(P), repeat=3):
        val = cgrid[idx[:, 0, a_], idx[:, 1, b_], idx[:, 2, c_]]
        u += w[:, 0, a_] * w[:, 1, b_] * w[:, 2, c_] * val
        gs[:, 0] += dw[:, 0, a_] * w[:, 1, b_] * w[:, 2, c_] * val
        gs[:, 1] += w[:, 0, a_] * dw[:, 1, b_] * w[:, 2, c_] * val
        gs[:, 2] += w[:, 0, a_] * w[:, 1, b_] * dw[:, 2, c_] * val
    grad = gs @ np.linalg.inv(H)                                    # row form of H^-T g
    f = -q[:, None] * grad
    # local part over all images within r_c
    i, j, d = _pairs_within(pos, H, r_c)
    r = np.sqrt(np.sum(d * d, axis=1))
    x = r / r_c
    omg = split.one_minus_g(x)
    np.add.at(u, i, q[j] * omg / (4.0 * math.pi * r))
    mag = (omg / r ** 2 + split.chi(x) / (r_c * r)) / (4.0 * math.pi)
    np.add.at(f, i, (q[i] * q[j] * mag / r)[:, None] * d)
    if virial:
        W += 0.5 * np.einsum("n,na,nb->ab", q[i] * q[j] * mag / r, d, d)
    # self term and neutralising background
    Q = float(np.sum(q))
    bg = -(Q / V) * 0.5 * r_c ** 2 * split.second_moment()
    u += -q * split.chi0 / (4.0 * math.pi * r_c) + bg
    if virial:
        W += 0.5 * Q * bg * np.eye(3)
    return dict(energy=0.5 * float(np.dot(q, u)), potential=u, forces=f, fourier_energy=fourier_energy,
                virial=W if virial else None)
