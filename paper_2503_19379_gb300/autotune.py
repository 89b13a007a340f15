"""Autotuner for the batched solve: picks the k-point group count and the block width (guard columns) that give the
most k-points per second on this GPU for a given grid, band count and precision.

Each candidate is timed on a sample of the k-points (a real solve to the requested tolerance through pc_solve, CUDA
events around it) and must reproduce the eigenvalues of the default configuration to that tolerance; the fastest
valid candidate is kept in a JSON cache keyed by the GPU name, N, the band count, the precision and the size class
of the k-point batch. Only configurations that the library's tests cover are candidates: groups 1, 2 and 4 and
guard widths around the default (half the bands plus one), with nbands + guard <= 21.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import pc


def default_guard(nbands: int) -> int:
    return max(0, min(nbands // 2 + 1, 21 - nbands))


def candidates(nbands: int, nk: int, precision: int):
    """Configurations to try: dicts with 'groups' and 'guard'."""
    g0 = default_guard(nbands)
    guards = sorted({g for g in (g0 - 2, g0, g0 + 2) if g >= 0 and nbands + g <= 21})
    groups = [1]
    if precision == pc.PC_PREC_MIXED:
        groups += [g for g in (2, 4) if nk >= 2 * g]
    return [{"groups": gr, "guard": gd} for gr in groups for gd in guards]


def cache_key(device: str, N: int, nbands: int, precision: int, nk: int) -> str:
    size_class = 1 << max(0, int(np.ceil(np.log2(max(nk, 1)))))  # batches of similar size share a choice
    return f"{device}|N={N}|nb={nbands}|prec={precision}|nk<={size_class}"


def _timed_solve(N, eps, kpts, nbands, tol, precision, cfg):
    """k-points/s and eigenvalues of one solve with configuration cfg (CUDA events on the solver's stream)."""
    torch = pc._torch()
    solver = pc.Solver(N, eps, precision=precision, groups=cfg["groups"], guard=cfg["guard"])
    try:
        solver.solve(kpts[:1], nbands, tol)  # warm-up: first-call allocations and kernel attributes
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record()
        out = solver.solve(kpts, nbands, tol)
        end.record()
        torch.cuda.synchronize()
        secs = start.elapsed_time(end) / 1e3
    finally:
        solver.close()
    return kpts.shape[0] / secs, out["evals"], out["status"]


def tune(N: int, eps, kpts, nbands: int, tol: float, precision: int = pc.PC_PREC_MIXED, sample: int = 8,
         cache_path: str | None = None, device: str | None = None, solve=None):
    """Best configuration for this workload: a dict with 'groups', 'guard', 'kpts_per_s' and 'trials'.

    sample: k-points timed per candidate (evenly spaced over the batch; at least 8, or the whole batch).
    solve: a replacement for the timed solve with the signature of _timed_solve (tests pass a fake). A cached choice
    for the same key is returned without timing anything."""
    kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
    nk = kpts.shape[0]
    if device is None:
        device = pc._torch().cuda.get_device_name(0)
    key = cache_key(device, N, nbands, precision, nk)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key], cached=True)
    solve = solve or _timed_solve
    # at least two k-points per group of the largest group count, so that every candidate is timed as it would run
    pick = np.unique(np.linspace(0, nk - 1, min(nk, max(sample, 8))).round().astype(int))
    ks = kpts[pick]
    trials = []
    ref = None
    for cfg in [{"groups": 1 if precision != pc.PC_PREC_MIXED else 0, "guard": -1}] + candidates(nbands, len(ks),
                                                                                                   precision):
        rate, evals, status = solve(N, eps, ks, nbands, tol, precision, cfg)
        if ref is None:  # the default configuration: the reference eigenvalues
            ref = np.asarray(evals)
            continue
        ok = status == 0 and np.max(np.abs(np.asarray(evals) - ref) / np.abs(ref)) <= 10 * tol
        trials.append({"groups": cfg["groups"], "guard": cfg["guard"], "kpts_per_s": float(rate), "valid": bool(ok)})
    valid = [t for t in trials if t["valid"]]
    if not valid:
        raise pc.PCError("autotune: no candidate reproduced the default configuration's eigenvalues")
    best = max(valid, key=lambda t: t["kpts_per_s"])
    result = {"groups": best["groups"], "guard": best["guard"], "kpts_per_s": best["kpts_per_s"], "trials": trials}
    if cache_path:
        cache[key] = result
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(result, cached=False)
