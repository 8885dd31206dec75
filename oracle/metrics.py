"""Error metric of the paper (Eq. Deltadef)."""
from __future__ import annotations

import numpy as np


def relative_rms_force_error(f_approx, f_ref) -> float:
    """Delta = sqrt( sum |F~_i - F_i|^2 / sum |F_i|^2 )."""
    f_approx = np.asarray(f_approx, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    return float(np.sqrt(np.sum((f_approx - f_ref) ** 2) / np.sum(f_ref ** 2)))
