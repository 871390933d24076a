"""Identification of Gaussians from one rendered view (test infrastructure).

Written from the definitions of Sec. 4 and 5; only the tests, the smoke
check and the benchmark's CPU-baseline leg use it.

  blur_split(S, H, W, theta)  G^blur = {i : S_i > theta H W}, theta = 2e-4
                              (the blur-split criterion of Sec. 4.1); S_i is
                              the number of pixels whose i_max is i.
  intersected(S)              G^int = {i : i is the i_max of some pixel}
                              (intersection preserving, Sec. 4.3), S_i > 0.
  keep_quantile(values, q)    Sec. 5.1 and 5.2 derive their thresholds
                              from a quantile of the values with a keep
                              quantile of 0.99, and define it no further.
                              Reading: of the M positive values, keep the
                              ceil(q M) largest, ties towards the lower index
                              (the rule of the importance pruning); q is the
                              single-precision value of the configuration and
                              q M is formed in double.
  visible(I, q)               V_i = 1 for the kept I_i of the view (Sec. 5.2).
  critical(imax, wmax, q, n)  G^crit: the i_max of the pixels whose w_max is
                              kept (Sec. 5.1: the Gaussians that provide the
                              maximum blending weight of a pixel, minus the
                              least significant by a 0.99 keep quantile).
"""
from __future__ import annotations

import math

import numpy as np


def blur_split(S, H: int, W: int, theta: float = 2e-4) -> np.ndarray:
    S = np.asarray(S, np.int64)
    return S > float(np.float32(theta)) * H * W


def intersected(S) -> np.ndarray:
    return np.asarray(S, np.int64) > 0


def keep_count(M: int, q: float) -> int:
    """Number of values a keep quantile q of M values keeps (the reading of Sec. 5.1, 5.2)."""
    return min(M, math.ceil(float(np.float32(q)) * M))


def keep_quantile(values, q: float) -> np.ndarray:
    v = np.asarray(values, np.float64)
    n = len(v)
    pos = np.nonzero(v > 0)[0]
    k = keep_count(len(pos), q)
    order = pos[np.lexsort((pos, -v[pos]))]      # descending value, then index
    keep = np.zeros(n, bool)
    keep[order[:k]] = True
    return keep


def visible(I, q: float = 0.99) -> np.ndarray:
    return keep_quantile(I, q)


def critical(imax, wmax, q: float, n: int) -> np.ndarray:
    imax = np.asarray(imax, np.int64)
    kept = keep_quantile(np.where(imax >= 0, np.asarray(wmax, np.float64), 0.0), q)
    out = np.zeros(n, bool)
    out[imax[kept & (imax >= 0)]] = True
    return out
