"""Host logic of the batched-solve autotuner (no GPU: the timed solve is replaced by a fake): the candidate set, the
choice of the fastest candidate that reproduces the default eigenvalues, and the cache."""
import numpy as np
import pytest

from paper_2503_19379_gb300 import autotune as at
from paper_2503_19379_gb300 import pc

REF = np.array([[1.0, 2.0, 3.0]] * 64)


def fake_solve_factory(rates, bad=()):
    calls = []

    def solve(N, eps, ks, nbands, tol, precision, cfg):
        calls.append(dict(cfg))
        key = (cfg["groups"], cfg["guard"])
        ev = REF[: ks.shape[0]] * (1.0 + (1e-3 if key in bad else 0.0))
        return rates.get(key, 1.0), ev, 0
    return solve, calls


def test_candidates_cover_groups_and_guards():
    c = at.candidates(10, 40, pc.PC_PREC_MIXED)
    assert {x["groups"] for x in c} == {1, 2, 4}
    assert {x["guard"] for x in c} == {4, 6, 8}
    assert all(10 + x["guard"] <= 21 for x in c)
    assert {x["groups"] for x in at.candidates(10, 40, pc.PC_PREC_FP64)} == {1}
    assert {x["groups"] for x in at.candidates(10, 5, pc.PC_PREC_MIXED)} == {1, 2}
    assert {x["guard"] for x in at.candidates(19, 40, pc.PC_PREC_FP64)} == {0, 2}


def test_picks_fastest_valid_and_caches(tmp_path):
    rates = {(4, 6): 50.0, (2, 8): 80.0, (1, 6): 20.0}
    solve, calls = fake_solve_factory(rates, bad={(2, 8)})
    cache = str(tmp_path / "tune.json")
    kp = np.zeros((40, 3))
    r = at.tune(32, None, kp, 10, 1e-6, pc.PC_PREC_MIXED, sample=4, cache_path=cache, device="gpu", solve=solve)
    assert (r["groups"], r["guard"]) == (4, 6) and not r["cached"]  # (2, 8) is faster but wrong
    assert calls[0] == {"groups": 0, "guard": -1}  # the default runs first as the reference
    assert len(calls) == 1 + len(at.candidates(10, 8, pc.PC_PREC_MIXED))  # the sample grows to 8 k-points
    solve2, calls2 = fake_solve_factory({})
    r2 = at.tune(32, None, kp, 10, 1e-6, pc.PC_PREC_MIXED, cache_path=cache, device="gpu", solve=solve2)
    assert r2["cached"] and (r2["groups"], r2["guard"]) == (4, 6) and calls2 == []
    r3 = at.tune(64, None, kp, 10, 1e-6, pc.PC_PREC_MIXED, sample=4, cache_path=cache, device="gpu", solve=solve2)
    assert not r3["cached"]  # another grid size is another key


def test_rejects_when_nothing_matches():
    solve, _ = fake_solve_factory({}, bad={(g, d) for g in (1, 2, 4) for d in (4, 6, 8)})
    with pytest.raises(pc.PCError):
        at.tune(32, None, np.zeros((40, 3)), 10, 1e-6, pc.PC_PREC_MIXED, sample=4, device="gpu", solve=solve)


def test_cache_key_size_classes():
    assert at.cache_key("g", 32, 10, 1, 40) == at.cache_key("g", 32, 10, 1, 64)
    assert at.cache_key("g", 32, 10, 1, 40) != at.cache_key("g", 32, 10, 1, 65)
