"""Prolate spheroidal wave function psi_0^c and the ESP splitting functions.

Definitions (Methods, "Optimizing the evaluation of the spectral part using
PSWFs"): psi_0^c is the eigenfunction with the largest eigenvalue of
F_c[f](x) = int_{-1}^{1} f(t) exp(i c x t) dt on L^2[-1,1]. ESP takes
chi(x) = psi_0^c(x)/C0 as the splitting kernel (Eq. pswf) and
phi(x) = psi_0^{c1}(2x/(P h)) as the spreading/interpolation (SI) kernel.

Construction used here (the classical route cited by the paper for PSWFs):
psi_0^c commutes with the prolate differential operator
    -d/dx (1-x^2) d/dx + c^2 x^2,
whose matrix in the L^2-normalised Legendre basis Pbar_k = sqrt(k+1/2) P_k is
symmetric tridiagonal in the even degrees; psi_0^c is its eigenvector of
smallest eigenvalue. A second, independent construction (Nystrom
discretisation of F_c on Gauss-Legendre nodes) is provided for cross-checks.

Readings of the paper (each listed in the design notes):
  * psi_0^c is L^2-normalised on [-1,1], sign psi(0) > 0; c solves psi(1) = eps.
    This reproduces Table 2's c_pswf.
  * C0 = int_0^1 psi_0^c, so that g(1) = int_0^1 chi = 1 and the local part
    L(r) vanishes for r >= r_c; chi is truncated to [0,1].
  * chihat(kappa) = int_0^inf chi(x) cos(kappa x) dx, so chihat(0) = 1 and
    Shat(k) = chihat(r_c |k|) / |k|^2 (Eq. hS) tends to the Coulomb 1/|k|^2.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.linalg import eigh_tridiagonal
from scipy.optimize import brentq
from scipy.special import roots_legendre


def _n_terms(c: float) -> int:
    """Number of even Legendre terms; coefficients decay super-exponentially past k ~ c."""
    return int(40 + 1.5 * c)


@lru_cache(maxsize=256)
def _legendre_coefficients(c: float) -> tuple:
    """Coefficients of psi_0^c in the plain Legendre basis P_k (tuple, even and odd slots)."""
    m = _n_terms(c)
    k = 2.0 * np.arange(m)                      # even degrees 0, 2, 4, ...
    diag = k * (k + 1) + c * c * (2 * k * (k + 1) - 1) / ((2 * k + 3) * (2 * k - 1))
    kk = k[:-1]
    off = c * c * (kk + 2) * (kk + 1) / ((2 * kk + 3) * np.sqrt((2 * kk + 1) * (2 * kk + 5)))
    _, vec = eigh_tridiagonal(diag, off, select="i", select_range=(0, 0))
    beta = vec[:, 0]                            # coefficients on Pbar_{2j}
    coef = np.zeros(2 * m)
    coef[0::2] = beta * np.sqrt(k + 0.5)        # Pbar_k = sqrt(k+1/2) P_k
    if npleg.legval(0.0, coef) < 0:
        coef = -coef
    # drop the tail below 1e-17 of the largest coefficient (below FP64 resolution)
    last = int(np.nonzero(np.abs(coef) > 1e-17 * np.max(np.abs(coef)))[0].max())
    return tuple(coef[: last + 1])


def psi_coefficients(c: float) -> np.ndarray:
    """Legendre-series coefficients (P_k basis) of L^2-normalised psi_0^c."""
    return np.array(_legendre_coefficients(float(c)))


def psi(c: float, x) -> np.ndarray:
    """psi_0^c(x) for |x| <= 1 (the Legendre series; analytic beyond)."""
    return npleg.legval(np.asarray(x, dtype=np.float64), psi_coefficients(c))


def dpsi(c: float, x) -> np.ndarray:
    """d/dx psi_0^c(x)."""
    return npleg.legval(np.asarray(x, dtype=np.float64), npleg.legder(psi_coefficients(c)))


def psi_integral_from_zero(c: float, x) -> np.ndarray:
    """int_0^x psi_0^c(t) dt (exact antiderivative of the Legendre series)."""
    return npleg.legval(np.asarray(x, dtype=np.float64),
                        npleg.legint(psi_coefficients(c), lbnd=0.0))


def eigenvalue(c: float) -> float:
    """lambda_0 with F_c[psi] = lambda psi; at x=0: lambda = int_{-1}^1 psi / psi(0)."""
    coef = psi_coefficients(c)
    total = 2.0 * coef[0]                       # int_{-1}^1 P_k = 2 delta_{k0}
    return float(total / psi(c, 0.0))


def psi_nystrom(c: float, n: int = 200) -> tuple[np.ndarray, np.ndarray, float]:
    """Independent construction: top eigenpair of the discretised F_c.

    Returns (nodes, psi at nodes (L^2-normalised, psi(0)-side positive), lambda).
    For even eigenfunctions F_c reduces to the cosine kernel cos(c x t).
    """
    x, w = roots_legendre(n)
    sw = np.sqrt(w)
    a = sw[:, None] * np.cos(c * np.outer(x, x)) * sw[None, :]
    vals, vecs = np.linalg.eigh(a)
    u = vecs[:, -1]
    f = u / sw
    f /= np.sqrt(np.sum(w * f * f))
    if f[n // 2] < 0:
        f = -f
    return x, f, float(vals[-1])


def c_from_tolerance(eps: float) -> float:
    """Shape parameter c with psi_0^c(1) = eps (psi L^2-normalised)."""
    return float(brentq(lambda c: float(psi(c, 1.0)) - eps, 0.5, 80.0, xtol=1e-14, rtol=1e-15))


# ---------------------------------------------------------------- splitting
_GL_X, _GL_W = roots_legendre(400)
_GL01_X = 0.5 * (_GL_X + 1.0)                   # nodes on [0,1]
_GL01_W = 0.5 * _GL_W


class PSWFSplit:
    """PSWF split chi = psi_0^c / C0 on [0,1] (Eq. kernelsplitting with Eq. pswf)."""

    kind = "pswf"

    def __init__(self, c: float):
        self.c = float(c)
        self.C0 = float(psi_integral_from_zero(self.c, 1.0))   # int_0^1 psi

    def chi(self, x):
        x = np.abs(np.asarray(x, dtype=np.float64))
        return np.where(x <= 1.0, psi(self.c, np.minimum(x, 1.0)) / self.C0, 0.0)

    def g(self, x):
        """g(x) = int_0^x chi, equal to 1 for x >= 1."""
        x = np.asarray(x, dtype=np.float64)
        return np.where(x < 1.0, psi_integral_from_zero(self.c, np.minimum(x, 1.0)) / self.C0, 1.0)

    def one_minus_g(self, x):
        """1 - g(x) = int_x^1 chi for x < 1, 0 beyond."""
        x = np.asarray(x, dtype=np.float64)
        xm = np.minimum(x, 1.0)
        tail = (psi_integral_from_zero(self.c, 1.0) - psi_integral_from_zero(self.c, xm)) / self.C0
        return np.where(x < 1.0, tail, 0.0)

    def chihat(self, kappa):
        """int_0^1 chi(x) cos(kappa x) dx by 400-point Gauss-Legendre."""
        kappa = np.asarray(kappa, dtype=np.float64)
        vals = self.chi(_GL01_X)
        flat = kappa.reshape(-1)
        out = np.cos(np.outer(flat, _GL01_X)) @ (_GL01_W * vals)
        return out.reshape(kappa.shape)

    def dchihat(self, kappa):
        """d chihat / d kappa = -int_0^1 x chi(x) sin(kappa x) dx (same rule)."""
        kappa = np.asarray(kappa, dtype=np.float64)
        vals = self.chi(_GL01_X)
        flat = kappa.reshape(-1)
        out = -np.sin(np.outer(flat, _GL01_X)) @ (_GL01_W * _GL01_X * vals)
        return out.reshape(kappa.shape)

    def second_moment(self) -> float:
        """int_0^1 x^2 chi(x) dx (enters the neutralising-background energy)."""
        return float(np.sum(_GL01_W * _GL01_X ** 2 * self.chi(_GL01_X)))

    @property
    def chi0(self) -> float:
        return float(self.chi(0.0))


class GaussianSplit:
    """Classical split (Eq. cem), read as chi(x) = 2 sqrt(alpha/pi) exp(-alpha x^2).

    With this normalisation int_0^inf chi = 1, g(x) = erf(sqrt(alpha) x),
    chihat(kappa) = exp(-kappa^2/(4 alpha)): classical Ewald with splitting
    parameter sqrt(alpha)/r_c. chi is not truncated; the local part is cut at r_c.
    """

    kind = "gauss"

    def __init__(self, alpha: float):
        from scipy.special import erf, erfc
        self.alpha = float(alpha)
        self._erf, self._erfc = erf, erfc

    def chi(self, x):
        x = np.asarray(x, dtype=np.float64)
        return 2.0 * np.sqrt(self.alpha / np.pi) * np.exp(-self.alpha * x * x)

    def g(self, x):
        return self._erf(np.sqrt(self.alpha) * np.asarray(x, dtype=np.float64))

    def one_minus_g(self, x):
        return self._erfc(np.sqrt(self.alpha) * np.asarray(x, dtype=np.float64))

    def chihat(self, kappa):
        kappa = np.asarray(kappa, dtype=np.float64)
        return np.exp(-kappa * kappa / (4.0 * self.alpha))

    def dchihat(self, kappa):
        kappa = np.asarray(kappa, dtype=np.float64)
        return -kappa / (2.0 * self.alpha) * np.exp(-kappa * kappa / (4.0 * self.alpha))

    def second_moment(self) -> float:
        return 1.0 / (2.0 * self.alpha)          # int_0^inf x^2 chi

    @property
    def chi0(self) -> float:
        return float(2.0 * np.sqrt(self.alpha / np.pi))


class PSWFWindow:
    """SI kernel phi(t) = psi_0^{c1}(2t/P) in grid units t = x/h (Eq. pswf).

    Support (-P/2, P/2]: the stencil of a particle at grid coordinate t is the P
    points l = ceil(t - P/2) ... ceil(t - P/2) + P - 1 (a reading: at the
    measure-zero tie t - l = -P/2 the end point is left out).
    """

    def __init__(self, c1: float, P: int):
        self.c1 = float(c1)
        self.P = int(P)

    def phi(self, t):
        t = np.asarray(t, dtype=np.float64)
        half = 0.5 * self.P
        inside = (t > -half) & (t <= half)
        return np.where(inside, psi(self.c1, np.clip(t / half, -1.0, 1.0)), 0.0)

    def dphi(self, t):
        """d phi / dt (grid units)."""
        t = np.asarray(t, dtype=np.float64)
        half = 0.5 * self.P
        inside = (t > -half) & (t <= half)
        return np.where(inside, dpsi(self.c1, np.clip(t / half, -1.0, 1.0)) / half, 0.0)

    def Phi(self, theta):
        """Fourier transform in grid units: int phi(t) cos(theta t) dt, theta = xi h."""
        theta = np.asarray(theta, dtype=np.float64)
        half = 0.5 * self.P
        vals = psi(self.c1, _GL01_X)
        flat = theta.reshape(-1)
        out = 2.0 * half * (np.cos(np.outer(flat, half * _GL01_X)) @ (_GL01_W * vals))
        return out.reshape(theta.shape)
