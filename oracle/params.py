"""The paper's parameter rules for ESP and the classical Gaussian split.

* Table 2 (optimal values): eps -> alpha_G, c_pswf, P_esp, R_default.
* Eq. pswfparameters: c from psi_0^c(1) = eps, n_f = ceil(c L / (pi r_c)).
* Eq. cemparameters: alpha_G = ln(1/eps), n_f = 2 ceil(ln(1/eps) L / (pi r_c)).
* The spectral part uses an even number of modes per axis: n_f is even.

Readings (the paper does not fix these):
  * n_f is rounded up to an even FFT-friendly size 2^a 3^b 5^c 7^d (a larger n_f
    only lowers the truncation error).
  * P between Table 2's tolerances takes the entry of the next tighter one;
    below 1e-5 it is extrapolated as ceil(log10(1/eps)) + 3.
  * The SI-kernel shape c1 (the paper only says it exceeds c a little) minimises the relative
    aliasing estimate over c1/c in [1.1, 1.4]; n_f is raised until that estimate
    is at most eps/2 (``plan``). C1_RATIO = 1.2 is the fixed default of
    ``pswf_parameters``.
"""
from __future__ import annotations

import math

import numpy as np

from . import pswf

# Table 2: eps -> (alpha_G, c_pswf, P_esp, R_default)
TABLE2 = {
    1e-3: (6.9078, 9.5392, 5, 5.78),
    5e-4: (7.6009, 10.290, 5, 7.71),
    1e-4: (9.2103, 12.024, 6, 14.32),
    5e-5: (9.9035, 12.762, 7, 22.42),
    1e-5: (11.5129, 14.471, 8, 54.57),
}

C1_RATIO = 1.2


def stencil_width(eps: float) -> int:
    """P_esp(eps) from Table 2 (next tighter entry), extrapolated below 1e-5."""
    for tol in sorted(TABLE2, reverse=True):
        if eps >= tol * (1 - 1e-12):
            return TABLE2[tol][2]
    if eps >= 1e-5 * (1 - 1e-12):
        return TABLE2[1e-5][2]
    return int(math.ceil(math.log10(1.0 / eps))) + 3


def is_smooth(n: int) -> bool:
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def round_grid(n: float) -> int:
    """Smallest even 2^a 3^b 5^c 7^d integer >= n."""
    m = max(2, int(math.ceil(n - 1e-9)))
    if m % 2:
        m += 1
    while not is_smooth(m):
        m += 2
    return m


def pswf_grid_min(c: float, L: float, r_c: float) -> float:
    """Eq. pswfparameters before rounding: c L / (pi r_c)."""
    return c * L / (math.pi * r_c)


def gauss_grid_min(eps: float, L: float, r_c: float) -> int:
    """Eq. cemparameters: 2 ceil(ln(1/eps) L / (pi r_c))."""
    return 2 * int(math.ceil(math.log(1.0 / eps) * L / (math.pi * r_c)))


def pswf_parameters(eps: float, L: float, r_c: float, grid_factor: float = 1.0):
    """(c, c1, P, n_f) for the PSWF split at tolerance eps.

    grid_factor >= 1 raises n_f above the paper's minimum (aliasing margin).
    """
    c = pswf.c_from_tolerance(eps)
    P = stencil_width(eps)
    n_f = round_grid(grid_factor * pswf_grid_min(c, L, r_c))
    return c, C1_RATIO * c, P, n_f


# ------------------------------------------------------------ aliasing rule
C1_RATIOS = tuple(1.1 + 0.05 * i for i in range(7))     # 1.10 ... 1.40
ALIAS_TARGET = 0.5                                       # accept E_A,rel <= 0.5 eps


def aliasing_error(split, c1: float, P: int, n_f: int, L: float, r_c: float, window=None) -> float:
    """Relative form of Eq. errorformula.

    E_A = 6 sum_{k in I, k != 0} |chihat(2 pi r_c |k|/L)| / |k|^2 * |Phi(th_x + 2 pi) / Phi(th_x)|,
    divided by sum_{k in I, k != 0} |chihat(2 pi r_c |k|/L)| / |k|^2 (the same sum
    without the alias ratio). The normalisation is a reading; the paper leaves it open.
    """
    k = np.arange(-n_f // 2, n_f // 2)
    k2 = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    uniq, inv = np.unique(k2, return_inverse=True)
    ch = np.abs(split.chihat(2.0 * math.pi * r_c * np.sqrt(uniq.astype(np.float64)) / L))
    with np.errstate(divide="ignore"):
        base_u = np.where(uniq > 0, ch / uniq, 0.0)
    base = base_u[inv.reshape(k2.shape)]
    per_kx = base.sum(axis=(1, 2))                         # sum over ky, kz for each kx
    if window is None:
        window = pswf.PSWFWindow(c1, P)
    th = 2.0 * math.pi * k / n_f
    ratio = np.abs(window.Phi(th + 2.0 * math.pi) / window.Phi(th))
    return float(6.0 * np.sum(per_kx * ratio) / np.sum(per_kx))


def next_grid(n: int) -> int:
    return round_grid(n + 1)


BSPLINE_ORDER = 5          # the default of both MD packages (Table 2's caption)


def default_grid_ratio(eps: float) -> float:
    """R_default(eps)^(1/3): the per-axis grid ratio of the default PME (Gaussian
    split, B-spline order 5, n_f raised until the error is met) to ESP, from
    Table 2's last row, interpolated linearly in (log eps, log R) between the
    tabulated tolerances and extrapolated along the nearest segment."""
    tols = sorted(TABLE2)                                   # 1e-5 ... 1e-3
    x = [math.log(t) for t in tols]
    y = [math.log(TABLE2[t][3]) for t in tols]
    lx = math.log(eps)
    k = 0
    while k < len(x) - 2 and lx > x[k + 1]:
        k += 1
    logR = y[k] + (y[k + 1] - y[k]) * (lx - x[k]) / (x[k + 1] - x[k])
    return math.exp(logR / 3.0)


def plan_bspline(eps: float, L: float, r_c: float, P: int = BSPLINE_ORDER):
    """The "Default" comparator (Methods, classical fast Ewald methods): the
    Gaussian split (Eq. cem, alpha = ln(1/eps), Table 2's alpha_G) with the
    cardinal B-spline window of order P, on the grid Table 2 says the default
    PME needs for the same error: n_f = R_default^(1/3) times ESP's
    Eq. pswfparameters value c L / (pi r_c), at least Eq. cemparameters' value,
    rounded up to an even FFT-friendly size. The relative aliasing estimate
    (Eq. errorformula) at that grid is reported with it.
    Returns dict(kind, window, alpha, P, n_f, alias)."""
    from . import bspline
    if not r_c < 0.5 * L:
        raise ValueError("r_c must be smaller than L/2")
    alpha = math.log(1.0 / eps)
    c = pswf.c_from_tolerance(eps)
    n_min = max(gauss_grid_min(eps, L, r_c), default_grid_ratio(eps) * pswf_grid_min(c, L, r_c))
    n_f = round_grid(n_min)
    err = aliasing_error(pswf.GaussianSplit(alpha), 0.0, P, n_f, L, r_c, window=bspline.BSplineWindow(P))
    return dict(kind="gauss", window="bspline", alpha=alpha, P=P, n_f=n_f, alias=err)


def plan(eps: float, L: float, r_c: float, kind: str = "pswf", max_steps: int = 8):
    """Paper's selection rules (Methods, parameter selection), as read here.

    c (or alpha) from the tolerance; P from Table 2; n_f from Eq. pswfparameters
    (Eq. cemparameters for the Gaussian split); then the SI-kernel shape c1 is
    the ratio in C1_RATIOS minimising the relative E_A, and n_f is raised to
    the next FFT-friendly size until that minimum is <= ALIAS_TARGET * eps.
    Returns dict(kind, c, alpha, c1, P, n_f, alias).
    """
    if not r_c < 0.5 * L:
        raise ValueError("r_c must be smaller than L/2")
    c = pswf.c_from_tolerance(eps)
    P = stencil_width(eps)
    if kind == "pswf":
        split = pswf.PSWFSplit(c)
        n_f = round_grid(pswf_grid_min(c, L, r_c))
        alpha = None
    else:
        alpha = math.log(1.0 / eps)
        split = pswf.GaussianSplit(alpha)
        n_f = round_grid(gauss_grid_min(eps, L, r_c))
    for _ in range(max_steps):
        errs = [aliasing_error(split, r * c, P, n_f, L, r_c) for r in C1_RATIOS]
        best = int(np.argmin(errs))
        if errs[best] <= ALIAS_TARGET * eps:
            break
        n_f = next_grid(n_f)
    return dict(kind=kind, c=c, alpha=alpha, c1=C1_RATIOS[best] * c, P=P, n_f=n_f,
                alias=errs[best])
