"""Plain CPU ESP in FP64: the method's steps in the paper's order and notation.

Spectral (far-field) part, the five-step procedure (Eqs. spread ... interp):
  1. spread       b_l  = sum_j phi~(r_j - h l) q_j                  l in I
  2. FFT          bh_k = sum_l exp(+2 pi i k.l / n_f) b_l            k in I
  3. scale        ch_k = p_k bh_k,
                  p_k  = Shat(2 pi k/L) / (L^3 Phi(th_x)^2 Phi(th_y)^2 Phi(th_z)^2)
                  (Eq. pk, first form, Phi the SI-kernel transform in grid units,
                  th = 2 pi k / n_f), p_0 = 0
  4. IFFT         c_l  = sum_k exp(-2 pi i k.l / n_f) ch_k
  5. interpolate  u~_i = sum_l phi~(r_i - h l) c_l, and grad u~_i by exact
                  derivatives of phi (the "AD" force method), or (the "ik"
                  method, Methods) by interpolating with phi~ the three grids
                  IFFT(-2 pi i k_a / L ch_k), a = x, y, z
Local (near-field) part (Eq. localpart): u^l_i = sum' q_j L(|r_i - r_j - nL|) over
pairs closer than r_c, L(r) = (1 - g(r/r_c)) / (4 pi r).
Self term: the spectral sum keeps j = i, n = 0 (spectralpart discussion), whose
value q_i S(0) = q_i chi(0) / (4 pi r_c) is subtracted from u_i.
Totals: u_i = u~_i + u^l_i - self; E = 1/2 sum q_i u_i; F_i = -q_i grad u~_i + F^l_i.
Virial W_ab = -dE/d eps_ab under the homogeneous deformation r -> (1 + eps) r
of atoms and box (the grid deforms with the box, so b_l and the grid-unit
Phi are unchanged): spectral part sum_k 1/2 |bh_k|^2 [p_k delta_ab +
p'_k k_a k_b / |k|^2], p'_k = (r_c xi chihat'(r_c xi) - 2 chihat(r_c xi)) /
(xi^2 L^3 Phi^2 Phi^2 Phi^2); local part 1/2 sum_i sum_j F_ij,a d_ij,b over the
pairs of Eq. localpart; background E_bg delta_ab (E_bg ~ 1/V); self term 0.
Non-neutral systems get the neutralising-background shift
-(Q/V) (r_c^2/2) int_0^1 x^2 chi(x) dx on every u_i.

phi is evaluated by its Legendre series (oracle.pswf), not by piecewise
polynomials. The sums are done with plain NumPy; FFTs by numpy.fft; the
neighbour search of the local part by scipy.spatial.cKDTree.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
from scipy.spatial import cKDTree

from . import params as prm
from . import pswf


@dataclass
class ESPParams:
    """Parameters of one solve: split kind, tolerance, cutoff, grid, stencil."""
    eps: float
    r_c: float
    P: int
    n_f: int
    c: float | None = None        # PSWF split shape (default: psi_0^c(1) = eps)
    c1: float | None = None       # SI kernel shape (default: C1_RATIO * c)
    kind: str = "pswf"            # "pswf" or "gauss"
    alpha: float | None = None    # Gaussian shape (default: ln(1/eps))
    window: str = "pswf"          # SI window: "pswf" (psi_0^{c1}) or "bspline" (order P)
    diff: str = "ad"              # spectral forces: "ad" (derivatives of phi) or "ik"
    virial_nyquist: str = "alias"       # off-diagonal Nyquist products (spectral_virial)

    def resolved(self) -> "ESPParams":
        c = self.c if self.c is not None else pswf.c_from_tolerance(self.eps)
        c1 = self.c1 if self.c1 is not None else prm.C1_RATIO * c
        alpha = self.alpha if self.alpha is not None else math.log(1.0 / self.eps)
        return ESPParams(self.eps, self.r_c, self.P, self.n_f, c, c1, self.kind, alpha, self.window, self.diff,
                         self.virial_nyquist)

    def si_window(self):
        p = self.resolved()
        if p.window == "bspline":
            from . import bspline
            return bspline.BSplineWindow(p.P)
        return pswf.PSWFWindow(p.c1, p.P)

    def split(self):
        p = self.resolved()
        return pswf.PSWFSplit(p.c) if p.kind == "pswf" else pswf.GaussianSplit(p.alpha)


def default_params(eps: float, L: float, r_c: float, kind: str = "pswf",
                   grid_factor: float = 1.0) -> ESPParams:
    if kind == "pswf":
        c, c1, P, n_f = prm.pswf_parameters(eps, L, r_c, grid_factor)
        return ESPParams(eps, r_c, P, n_f, c, c1, "pswf")
    c = pswf.c_from_tolerance(eps)
    n_f = prm.round_grid(grid_factor * prm.gauss_grid_min(eps, L, r_c))
    return ESPParams(eps, r_c, prm.stencil_width(eps), n_f, c, prm.C1_RATIO * c, "gauss",
                     math.log(1.0 / eps))


# ------------------------------------------------------------------ stencils
def stencil(pos, L, n_f, window):
    """Per-axis stencil of every particle: grid indices, weights, d(weight)/dx.

    Grid coordinate t = x/h, evaluated as (x/L) n_f; the P points
    l0 .. l0+P-1 with l0 = ceil(t - P/2) carry weights phi(t - l); derivatives
    are phi'(t - l)/h. (At the measure-zero tie t - P/2 in Z the end point is
    left out; evaluating t as (x/L) n_f fixes how rounding decides that tie.)
    """
    h = L / n_f
    t = (np.mod(np.asarray(pos, dtype=np.float64), L) / L) * n_f
    P = window.P
    l0 = np.ceil(t - 0.5 * P).astype(np.int64)
    l = l0[:, :, None] + np.arange(P)[None, None, :]          # (N,3,P)
    s = t[:, :, None] - l
    return np.mod(l, n_f), window.phi(s), window.dphi(s) / h


def spread(pos, q, L, n_f, window):
    """Step 1 (Eq. spread): b_l on the n_f^3 grid, index order [lx, ly, lz]."""
    idx, w, _ = stencil(pos, L, n_f, window)
    P = window.P
    b = np.zeros(n_f ** 3)
    for a, bb, cc in itertools.product(range(P), repeat=3):
        lin = (idx[:, 0, a] * n_f + idx[:, 1, bb]) * n_f + idx[:, 2, cc]
        b += np.bincount(lin, weights=q * w[:, 0, a] * w[:, 1, bb] * w[:, 2, cc],
                         minlength=n_f ** 3)
    return b.reshape(n_f, n_f, n_f)


def influence(L, n_f, r_c, split, window):
    """Step 3 coefficients p_k on the FFT-ordered grid (Eq. pk), p_0 = 0."""
    k = np.fft.fftfreq(n_f, d=1.0 / n_f)                      # integers in I
    Phi = window.Phi(2.0 * math.pi * k / n_f)
    k2 = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2).astype(np.int64)
    uniq, inv = np.unique(k2, return_inverse=True)
    xi = 2.0 * math.pi * np.sqrt(uniq.astype(np.float64)) / L
    with np.errstate(divide="ignore", invalid="ignore"):
        shat = np.where(uniq > 0, split.chihat(r_c * xi) / xi ** 2, 0.0)
    shat = shat[inv.reshape(k2.shape)]
    den = L ** 3 * (Phi[:, None, None] * Phi[None, :, None] * Phi[None, None, :]) ** 2
    return shat / den


def ik_gradient(ch, L):
    """The three grids of the ik method: c^a_l = sum_k exp(-2 pi i k.l/n_f)
    (-2 pi i k_a / L) ch_k, the exact derivatives along a of the
    trigonometric interpolant of c_l (ch in numpy's FFT order). The Nyquist
    component k_a = -n_f/2 of the differentiated axis is set to zero: its
    derivative is not a real grid function (reading of the ik method for
    even n_f)."""
    n_f = ch.shape[0]
    k = np.fft.fftfreq(n_f, d=1.0 / n_f)
    k = np.where(k == -(n_f // 2), 0.0, k) if n_f % 2 == 0 else k
    out = []
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = n_f
        mult = (-2j * math.pi / L) * k.reshape(shape)
        out.append(np.fft.fftn(ch * mult).real)
    return out


def influence_virial(L, n_f, r_c, split, window):
    """p'_k of the spectral virial (FFT order, p'_0 = 0): the derivative of
    Shat(xi) = chihat(r_c xi)/xi^2 with respect to ln xi, over L^3 Phi^2 Phi^2
    Phi^2, i.e. (r_c xi chihat'(r_c xi) - 2 chihat(r_c xi)) / xi^2 / den."""
    k = np.fft.fftfreq(n_f, d=1.0 / n_f)
    Phi = window.Phi(2.0 * math.pi * k / n_f)
    k2 = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2).astype(np.int64)
    uniq, inv = np.unique(k2, return_inverse=True)
    xi = 2.0 * math.pi * np.sqrt(uniq.astype(np.float64)) / L
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(uniq > 0, (r_c * xi * split.dchihat(r_c * xi) - 2.0 * split.chihat(r_c * xi)) / xi ** 2, 0.0)
    d = d[inv.reshape(k2.shape)]
    den = L ** 3 * (Phi[:, None, None] * Phi[None, :, None] * Phi[None, None, :]) ** 2
    return d / den


def spectral_virial(bh, p, pv, n_f, nyquist="alias"):
    """sum_k 1/2 |bh_k|^2 [p_k delta + p'_k k k^T / |k|^2] (3 x 3).

    A Nyquist index k_a = -n_f/2 stands for both aliases +-n_f/2 (the
    diagonal k_a^2 is the same for both). Off-diagonal products k_a k_b:
    "alias" (default): the mode and the representative of -k, whose Nyquist
    components flip together (the pairing the real part of the inverse
    transform applies to the energy of a deformed cell): zero when exactly
    one of k_a, k_b is Nyquist, k_a k_b when both are. This is the exact
    -dE/d eps_ab (pinned by shearing the cube through the triclinic oracle).
    "component": each Nyquist component averaged on its own, so a product
    with any Nyquist component is zero; kept for comparison, it differs from
    the derivative only through the modes with two Nyquist components."""
    k = np.fft.fftfreq(n_f, d=1.0 / n_f)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"))         # (3, n, n, n)
    if nyquist == "alias" and n_f % 2 == 0:
        nyq = K == -(n_f // 2)
        Kp = {(i, j): np.where(nyq[i] ^ nyq[j], 0.0, K[i] * K[j]) for i in range(3) for j in range(3)}
    else:
        ks = np.where(k == -(n_f // 2), 0.0, k) if n_f % 2 == 0 else k
        Ks = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"))
        Kp = {(i, j): Ks[i] * Ks[j] for i in range(3) for j in range(3)}
    k2 = np.sum(K * K, axis=0)
    a = 0.5 * np.abs(bh) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(k2 > 0, a * pv / k2, 0.0)
    W = np.eye(3) * float(np.sum(a * p))
    for i in range(3):
        for j in range(3):
            W[i, j] += float(np.sum(t * K[i] * K[j])) if i == j else float(np.sum(t * Kp[(i, j)]))
    return W


def far_field(pos, q, L, n_f, r_c, split, window, targets, diff="ad", virial=None, virial_nyquist="alias"):
    """Steps 1-5: (u~ at targets, grad u~ at targets, 1/2 sum_k p_k |bh_k|^2).
    With a dict `virial`, its key "spectral" receives the spectral virial."""
    b = spread(pos, q, L, n_f, window)
    bh = np.fft.ifftn(b) * n_f ** 3                           # exp(+2 pi i k.l/n_f)
    p = influence(L, n_f, r_c, split, window)
    fourier_energy = 0.5 * float(np.sum(p * np.abs(bh) ** 2))
    if virial is not None:
        virial["spectral"] = spectral_virial(bh, p, influence_virial(L, n_f, r_c, split, window), n_f,
                                             virial_nyquist)
    ch = p * bh
    cgrid = np.fft.fftn(ch).real                              # exp(-2 pi i k.l/n_f)
    idx, w, dw = stencil(pos[targets], L, n_f, window)
    P = window.P
    u = np.zeros(len(targets))
    grad = np.zeros((len(targets), 3))
    if diff == "ik":
        gx, gy, gz = ik_gradient(ch, L)
        for a, bb, cc in itertools.product(range(P), repeat=3):
            ii = (idx[:, 0, a], idx[:, 1, bb], idx[:, 2, cc])
            www = w[:, 0, a] * w[:, 1, bb] * w[:, 2, cc]
            u += www * cgrid[ii]
            grad[:, 0] += www * gx[ii]
            grad[:, 1] += www * gy[ii]
            grad[:, 2] += www * gz[ii]
        return u, grad, fourier_energy
    if diff != "ad":
        raise ValueError("diff must be 'ad' or 'ik'")
    for a, bb, cc in itertools.product(range(P), repeat=3):
        val = cgrid[idx[:, 0, a], idx[:, 1, bb], idx[:, 2, cc]]
        u += w[:, 0, a] * w[:, 1, bb] * w[:, 2, cc] * val
        grad[:, 0] += dw[:, 0, a] * w[:, 1, bb] * w[:, 2, cc] * val
        grad[:, 1] += w[:, 0, a] * dw[:, 1, bb] * w[:, 2, cc] * val
        grad[:, 2] += w[:, 0, a] * w[:, 1, bb] * dw[:, 2, cc] * val
    return u, grad, fourier_energy


def near_field(pos, q, L, r_c, split, targets, virial=None):
    """Local part (Eq. localpart) and its forces at the targets.

    Pairs closer than r_c (strictly) under the minimum image, r_c < L/2.
    u^l_i += q_j (1 - g(x)) / (4 pi r),  x = r / r_c
    F^l_i += q_i q_j [(1 - g(x))/r^2 + chi(x)/(r_c r)] / (4 pi) * (r_i - r_j)/r
    With a dict `virial`, its key "local" receives 1/2 sum over the targets'
    pairs of F_ij d_ij^T (the local virial when every atom is a target).
    """
    if not r_c < 0.5 * L:
        raise ValueError("r_c must be smaller than L/2")
    pos = np.mod(np.asarray(pos, dtype=np.float64), L)
    pos[pos >= L] = 0.0
    tree = cKDTree(pos, boxsize=L)
    u = np.zeros(len(targets))
    f = np.zeros((len(targets), 3))
    W = np.zeros((3, 3))
    for t_i, i in enumerate(targets):
        js = np.asarray(tree.query_ball_point(pos[i], r_c), dtype=np.int64)
        js = js[js != i]
        d = pos[i] - pos[js]
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        keep = r < r_c
        d, r, js = d[keep], r[keep], js[keep]
        x = r / r_c
        omg = split.one_minus_g(x)
        u[t_i] = np.sum(q[js] * omg / (4.0 * math.pi * r))
        mag = (omg / r ** 2 + split.chi(x) / (r_c * r)) / (4.0 * math.pi)
        f[t_i] = q[i] * np.sum((q[js] * mag / r)[:, None] * d, axis=0)
        if virial is not None:
            W += 0.5 * q[i] * (d.T * (q[js] * mag / r)) @ d
    if virial is not None:
        virial["local"] = W
    return u, f


def esp(pos, q, L, p: ESPParams, targets=None):
    """ESP potentials, forces and (for all-atom runs) energy.

    Returns dict(energy, potential, forces, fourier_energy, spectral_potential,
    spectral_forces, local_potential, local_forces, self_term, indices, params).
    """
    p = p.resolved()
    pos = np.mod(np.asarray(pos, dtype=np.float64), L)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    all_atoms = targets is None
    tgt = np.arange(n) if all_atoms else np.asarray(targets, dtype=np.int64)
    split = p.split()
    window = p.si_window()
    parts = {} if all_atoms else None
    u_s, grad_s, e_fourier = far_field(pos, q, L, p.n_f, p.r_c, split, window, tgt, p.diff, parts,
                                       p.virial_nyquist)
    u_l, f_l = near_field(pos, q, L, p.r_c, split, tgt, parts)
    self_term = q[tgt] * split.chi0 / (4.0 * math.pi * p.r_c)
    Q = float(np.sum(q))
    background = -(Q / L ** 3) * 0.5 * p.r_c ** 2 * split.second_moment()
    u = u_s + u_l - self_term + background
    f = -q[tgt, None] * grad_s + f_l
    energy = 0.5 * float(np.dot(q, u)) if all_atoms else None
    virial = None
    if all_atoms:
        e_bg = 0.5 * Q * background
        virial = parts["spectral"] + parts["local"] + e_bg * np.eye(3)
    return dict(energy=energy, potential=u, forces=f, fourier_energy=e_fourier, virial=virial,
                spectral_potential=u_s, spectral_forces=-q[tgt, None] * grad_s,
                local_potential=u_l, local_forces=f_l, self_term=self_term,
                indices=tgt, params=p)
