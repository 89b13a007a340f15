"""Band-structure post-processing: the band-gap ratio of Section 6.2 from the eigenvalues of a k-point path.

The solver returns omega^2 per band and k-point; the frequencies are their square roots. For the gap above band n
(1-based), omega_low is the largest frequency of band n over the path and omega_up the smallest of band n + 1; the
ratio is (omega_up - omega_low) / ((omega_up + omega_low) / 2) when omega_up > omega_low (a complete gap), else 0.
"""
from __future__ import annotations

import numpy as np


def gap_ratios(evals) -> np.ndarray:
    """Ratio of the gap above each band n = 1 .. nbands - 1 (index n - 1), 0 where bands overlap.

    evals: array [nk][nbands] of omega^2 (ascending per k-point)."""
    w = np.sqrt(np.maximum(np.asarray(evals, dtype=np.float64), 0.0))
    low = w[:, :-1].max(axis=0)
    up = w[:, 1:].min(axis=0)
    r = (up - low) / (0.5 * (up + low))
    return np.where(up > low, r, 0.0)


def largest_gap(evals):
    """(n, ratio) of the widest complete gap, n the band below it (1-based); (0, 0.0) when there is none."""
    r = gap_ratios(evals)
    if r.size == 0 or r.max() <= 0.0:
        return 0, 0.0
    n = int(np.argmax(r))
    return n + 1, float(r[n])
