"""The autotuner (paper_2503_19379_gb300/autotune.py) on the device: it times real solves of a sample of the
fcc-spheres-N32 batch for each candidate configuration (k-point groups, guard columns), keeps the fastest one that
reproduces the default configuration's eigenvalues, and caches it; the cached configuration solves the whole batch
to the default's eigenvalues, and a second call returns the cached choice without timing anything.
"""
import os

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2503_19379_gb300 as p
    return p


def test_autotune_picks_a_valid_configuration(pcmod, tmp_path):
    from paper_2503_19379_gb300 import autotune
    w = wl.workload_fcc_32()
    eps = pcmod.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    prec = pcmod.pc.PC_PREC_MIXED
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(w.N, eps, w.kpts, w.nbands, w.tol, precision=prec, sample=8, cache_path=cache)
    assert not res["cached"]
    assert any(t["valid"] for t in res["trials"])
    assert res["kpts_per_s"] == max(t["kpts_per_s"] for t in res["trials"] if t["valid"])
    again = autotune.tune(w.N, eps, w.kpts, w.nbands, w.tol, precision=prec, sample=8, cache_path=cache)
    assert again["cached"] and again["groups"] == res["groups"] and again["guard"] == res["guard"]
    # the chosen configuration on the whole batch: the default configuration's eigenvalues
    base = pcmod.Solver(w.N, eps, precision=prec).solve(w.kpts, w.nbands, w.tol)
    tuned = pcmod.Solver(w.N, eps, precision=prec, groups=res["groups"], guard=res["guard"]).solve(
        w.kpts, w.nbands, w.tol)
    assert base["status"] == 0 and tuned["status"] == 0
    assert np.max(np.abs(tuned["evals"] - base["evals"]) / base["evals"]) <= 10 * w.tol
    assert np.all(tuned["resid"] <= w.tol)
