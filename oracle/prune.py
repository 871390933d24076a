"""Selection by accumulated blending weight (test infrastructure).

MSv2-D (Sec. 6.1) replaces simplification by importance-based pruning: the
importance of Gaussian i is its accumulated blending weight I_i (Sec. 3.2),
and the least important Gaussians are removed.  The reading adopted here for
"keep the top fraction f": keep the ceil(f N) Gaussians with the largest I_i,
ties broken towards the lower index, and list the kept indices ascending.
"""
from __future__ import annotations

import math

import numpy as np


def keep_top_k(weight_sum, k: int) -> np.ndarray:
    """The k largest weights, ties towards the lower index, ascending indices.
    Importance-based pruning of MSv2-D (Sec. 6.1)."""
    w = np.asarray(weight_sum, np.float64)
    n = len(w)
    order = np.lexsort((np.arange(n), -w))      # descending weight, then index
    return np.sort(order[:min(k, n)])


def keep_top(weight_sum, frac: float) -> np.ndarray:
    """Importance-based pruning of MSv2-D (Sec. 6.1): the top fraction f."""
    n = len(weight_sum)
    return keep_top_k(weight_sum, min(n, math.ceil(frac * n)))
