"""Cardinal B-spline spreading/interpolation window (oracle; test
infrastructure only).

The paper compares ESP with the classical Gaussian split run on the standard
smooth-PME machinery, whose SI kernel is the cardinal B-spline (Methods,
comparison with the "Default" parameters; Table 2's R_default). The
centred B-spline of order P, in grid units t,

    phi(t) = M_P(t + P/2),   M_P(x) = 1/(P-1)! sum_{k=0}^{P} (-1)^k C(P,k) (x-k)_+^{P-1},

is a piecewise polynomial of degree P-1 on the P unit pieces of (-P/2, P/2]
(the same stencil convention as the PSWF window), and its transform is

    Phi(theta) = int phi(t) exp(i theta t) dt = (sin(theta/2) / (theta/2))^P.

The derivative is M_P'(x) = M_{P-1}(x) - M_{P-1}(x-1).
"""
from __future__ import annotations

import math

import numpy as np


def cardinal(P: int, x):
    """M_P(x) by the truncated-power formula (support [0, P])."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for k in range(P + 1):
        out += (-1) ** k * math.comb(P, k) * np.maximum(x - k, 0.0) ** (P - 1)
    out /= math.factorial(P - 1)
    return np.where((x > 0.0) & (x < P), out, 0.0)


def cardinal_recursive(P: int, x):
    """M_P(x) by the two-term recursion from the unit box (an independent
    construction used to pin `cardinal`)."""
    x = np.asarray(x, dtype=np.float64)
    if P == 1:
        return np.where((x >= 0.0) & (x < 1.0), 1.0, 0.0)
    return (x * cardinal_recursive(P - 1, x) + (P - x) * cardinal_recursive(P - 1, x - 1.0)) / (P - 1)


class BSplineWindow:
    """Centred cardinal B-spline of order P as an SI window in grid units."""

    kind = "bspline"

    def __init__(self, P: int):
        if P < 2:
            raise ValueError("B-spline order must be >= 2")
        self.P = int(P)

    def phi(self, t):
        t = np.asarray(t, dtype=np.float64)
        half = 0.5 * self.P
        inside = (t > -half) & (t <= half)
        return np.where(inside, cardinal(self.P, t + half), 0.0)

    def dphi(self, t):
        """d phi / dt (grid units)."""
        t = np.asarray(t, dtype=np.float64)
        half = 0.5 * self.P
        x = t + half
        inside = (t > -half) & (t <= half)
        return np.where(inside, cardinal(self.P - 1, x) - cardinal(self.P - 1, x - 1.0), 0.0)

    def Phi(self, theta):
        """Fourier transform in grid units: (sin(theta/2)/(theta/2))^P."""
        theta = np.asarray(theta, dtype=np.float64)
        half = 0.5 * theta
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(np.abs(half) > 1e-12, np.sin(half) / half, 1.0)
        return s ** self.P
