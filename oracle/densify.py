"""Aggressive clone of Sec. 5.1 (test infrastructure; used only by the tests,
the smoke check and the benchmark's CPU-baseline leg).

Every selected (critical) Gaussian is cloned into two (the number of clones
is fixed to 2 in the paper, which simplifies the state transition it adopts):
both keep the centre, rotation and SH; the opacity becomes
o' = 1 - sqrt(1 - o) and the covariance o^2 (2 o' - o'^2 / sqrt 2)^-2 Sigma,
so the scales are multiplied by o / (2 o' - o'^2 / sqrt 2).  Layout reading:
the first member replaces the Gaussian's row, the second is appended (row
n + r for the r-th selected Gaussian).
"""
from __future__ import annotations

import numpy as np


def clone_opacity(o):
    """Opacity of each clone, o' = 1 - sqrt(1 - o) (aggressive clone, Sec. 5.1)."""
    return 1.0 - np.sqrt(1.0 - np.asarray(o, np.float64))


def clone_scale_factor(o):
    """Scale factor of each clone, o / (2 o' - o'^2 / sqrt 2) (aggressive clone, Sec. 5.1)."""
    o = np.asarray(o, np.float64)
    on = clone_opacity(o)
    return o / (2.0 * on - on * on / np.sqrt(2.0))


def clone(means, scales, rotations, opacities, sh, idx) -> dict:
    idx = np.asarray(idx, np.int64)
    n = len(opacities)
    out = {}
    for name, a in (("means", means), ("scales", scales), ("rotations", rotations), ("opacities", opacities),
                    ("sh", sh)):
        a = np.asarray(a, np.float64)
        out[name] = np.concatenate([a, a[idx]], 0)
    o = np.asarray(opacities, np.float64)[idx]
    on, f = clone_opacity(o), clone_scale_factor(o)
    for rows in (idx, n + np.arange(len(idx))):
        out["opacities"][rows] = on
        out["scales"][rows] = np.asarray(scales, np.float64)[idx] * f[:, None]
    return out
