"""Writes the oracle's eigenvalues at sampled k-points of the benchmark paths into tests/golden/.

Only the FP64 oracle (``oracle/``) and the shared input generators (``workloads``) run here: the permittivity from
``oracle.geometry``, Algorithm 4.1 with the oracle's own LOBPCG and FFT preconditioner (``oracle.eigs``), to a
relative residual of 1e-8 (eigenvalues accurate to about 1e-14 relative). The GPU parity tests read the file and
compare the CUDA solves with it; no value in it comes from the CUDA path. Each row also records the oracle's own
LOBPCG iteration count to the workload's tolerance (a separate solve from the same random start, with the block size
of the CUDA solve), which the benchmark's reference arm uses to turn its timed oracle iterations into k-points/s.

Usage: python tests/golden/make_oracle_evals.py WORKLOAD [k-index ...]   (one process per k-index, in parallel)
       python tests/golden/make_oracle_evals.py --iters-at-tol WORKLOAD  (adds the iteration counts to a file)
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# the k-indices of each workload's path whose oracle eigenvalues are stored
SAMPLES = {
    "fcc-spheres-N32": [0, 3, 10, 17, 20, 26, 39],
    "diamond-air-N64": [0, 21, 59],
}
ORACLE_TOL = 1e-8


def workload(name):
    import workloads as wl
    return {"fcc-spheres-N32": wl.workload_fcc_32, "diamond-air-N64": wl.workload_diamond_64}[name]()


def solve_one(args):
    name, kidx = args
    import numpy as np

    from oracle import eigs, geometry
    w = workload(name)
    m0 = 1.0 / geometry.eps_edges(w.N, w.structure.as_array(), w.structure.eps_bg)
    t = time.perf_counter()
    out = eigs.solve_kpoint(w.N, w.kpts[kidx], m0, w.nbands, ORACLE_TOL, guard=w.nbands // 2 + 1, maxiter=600)
    secs = time.perf_counter() - t
    return {"kidx": int(kidx), "k": [float(x) for x in w.kpts[kidx]], "evals": [float(x) for x in out["evals"]],
            "max_resid": float(np.max(out["resid"])), "iters": int(out["iters"]), "doublings": int(out["doublings"]),
            "seconds": secs}


def iters_at_tol(args):
    """The oracle's LOBPCG iterations to the workload's tolerance at one k-point (block size of the CUDA solve)."""
    name, kidx = args
    from oracle import eigs, geometry
    w = workload(name)
    m0 = 1.0 / geometry.eps_edges(w.N, w.structure.as_array(), w.structure.eps_bg)
    guard = min(w.nbands // 2 + 1, 21 - w.nbands)
    t = time.perf_counter()
    out = eigs.solve_kpoint(w.N, w.kpts[kidx], m0, w.nbands, w.tol, guard=guard, maxiter=600)
    return int(out["iters"]), time.perf_counter() - t


def add_iters(name):
    path = os.path.join(HERE, f"oracle_evals_{name}.json")
    with open(path) as f:
        doc = json.load(f)
    kidx = [r["kidx"] for r in doc["kpoints"]]
    with mp.get_context("spawn").Pool(len(kidx)) as pool:
        res = pool.map(iters_at_tol, [(name, k) for k in kidx])
    for r, (its, secs) in zip(doc["kpoints"], res):
        r["iters_at_workload_tol"] = its
        r["seconds_at_workload_tol"] = secs
    doc["workload_tol"] = workload(name).tol
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    print(path)


def main():
    if sys.argv[1] == "--iters-at-tol":
        os.environ.setdefault("OMP_NUM_THREADS", "2")
        add_iters(sys.argv[2])
        return
    name = sys.argv[1]
    kidx = [int(x) for x in sys.argv[2:]] or SAMPLES[name]
    os.environ.setdefault("OMP_NUM_THREADS", "2")
    w = workload(name)
    with mp.get_context("spawn").Pool(len(kidx)) as pool:
        rows = pool.map(solve_one, [(name, k) for k in kidx])
    path = os.path.join(HERE, f"oracle_evals_{name}.json")
    doc = {"workload": name, "N": w.N, "nbands": w.nbands, "oracle_tol": ORACLE_TOL,
           "source": "tests/golden/make_oracle_evals.py (oracle.eigs.solve_kpoint, FP64)", "kpoints": rows}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
