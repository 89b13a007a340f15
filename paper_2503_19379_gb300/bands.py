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


def structure_eps(workload) -> np.ndarray:
    """Edge permittivity of a workload of the paper's own cells (workloads.workload_bcc_gyroid / _fcc_diamond, whose
    `extra` names the geometry), or of a sphere workload on the cube."""
    from . import pc
    ex = getattr(workload, "extra", {}) or {}
    geom = ex.get("geometry")
    if geom == "gyroid":
        return pc.eps_gyroid(workload.N, ex["lattice"], 1.0, ex["threshold"], ex["eps_in"], 1.0)
    if geom == "diamond":
        return pc.eps_diamond(workload.N, ex["lattice"], 1.0, ex["r"], ex["b"], ex["eps_in"], 1.0)
    s = workload.structure
    return pc.eps_spheres(workload.N, s.as_array(), s.eps_bg)


def timed_solve(workload, precision: int, repeats: int = 1):
    """Seconds per solve of the workload's k-points (CUDA events around pc_solve, after one untimed solve), with the
    eigenvalues and iteration counts: the paper's timing setting (first 10 eigenvalues at k = (pi, pi, pi) / l)."""
    from . import pc
    torch = pc._torch()
    ex = getattr(workload, "extra", {}) or {}
    solver = pc.Solver(workload.N, structure_eps(workload), lattice=ex.get("lattice"), precision=precision)
    try:
        solver.solve(workload.kpts, workload.nbands, workload.tol)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(repeats):
            out = solver.solve(workload.kpts, workload.nbands, workload.tol)
        b.record()
        torch.cuda.synchronize()
    finally:
        solver.close()
    return {"seconds": a.elapsed_time(b) / 1e3 / repeats, "evals": out["evals"], "iters": out["iters"],
            "status": out["status"]}
