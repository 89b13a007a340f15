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


def solve_path_two_pass(solver, kpts, nbands: int, tol: float):
    """All k-points of a path in two batched solves: the even-indexed k-points from random blocks, then the odd ones
    from the eigenvectors of their preceding (even) neighbour (pc_solve_init). Along a path the neighbour's
    eigenvectors are a close start: the oracle's LOBPCG needs about 30% fewer iterations from them.

    Returns the dict of Solver.solve (evals, iters, resid, status) in path order."""
    kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
    nk = kpts.shape[0]
    even = np.arange(0, nk, 2)
    odd = np.arange(1, nk, 2)
    first = solver.solve(kpts[even], nbands, tol, want_vectors=odd.size > 0)
    evals = np.zeros((nk, nbands))
    resid = np.zeros((nk, nbands))
    iters = np.zeros(nk, dtype=np.int32)
    evals[even], resid[even], iters[even] = first["evals"], first["resid"], first["iters"]
    status = first["status"]
    if odd.size:
        import torch
        x0 = first["evecs"][(odd - 1) // 2].to(torch.complex64).contiguous()  # odd i starts from i - 1 = 2 ((i-1)/2)
        del first["evecs"]
        second = solver.solve(kpts[odd], nbands, tol, x0=x0)
        evals[odd], resid[odd], iters[odd] = second["evals"], second["resid"], second["iters"]
        status = max(status, second["status"])
    return {"evals": evals, "iters": iters, "resid": resid, "status": status}
