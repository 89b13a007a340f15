"""Device geometry of Section 6.3's structures (pc_eps_gyroid, pc_eps_diamond) against the oracle's sampling
(oracle/geometry.py), on the BCC and FCC primitive cells (and the gyroid on the cube).

Both sides decide "inside" in FP64, but from their own sin/cos and dot products, which may differ in the last bit.
A point therefore may differ only where the oracle's own decision value lies within 1e-12 of the boundary (the
gyroid's g at its threshold, a distance at a radius, a focal-distance sum at its major axis); every other point
must agree exactly.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import geometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    import os
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2503_19379_gb300 as p
    return p


def edge_points(N, A):
    return [geometry.edge_positions(N, axis) @ np.asarray(A).T for axis in range(3)]


@pytest.mark.parametrize("N", [16, 32, 64])
@pytest.mark.parametrize("cell", ["bcc", "sc"])
def test_gyroid_matches_oracle(pcmod, N, cell):
    A = wl.BCC_CELL if cell == "bcc" else wl.SC_CELL
    got = pcmod.eps_gyroid(N, A, 1.0, 1.1, 16.0, 1.0)
    ref = geometry.eps_edges_gyroid(N, A, 1.0, 1.1, 16.0, 1.0)
    diff = got != ref
    if diff.any():
        pts = edge_points(N, A)
        g = np.stack([geometry.gyroid_value(p, 1.0) for p in pts])
        assert np.all(np.abs(g[diff] - 1.1) <= 1e-12)
    assert 0.0 < np.mean(ref == 16.0) < 0.5


def diamond_margin(N, A):
    """Per edge point, the distance of the oracle's decision values to their thresholds (smallest over objects)."""
    A = np.asarray(A, dtype=np.float64)
    Ainv = np.linalg.inv(A)
    spheres, spheroids = geometry.diamond_objects(1.0, 0.12, 0.11)
    out = []
    for p in edge_points(N, A):
        x = p.reshape(-1, 3)
        m = np.full(x.shape[0], np.inf)
        for c, rad in spheres:
            d = np.sqrt(np.sum(geometry._nearest_offset(x, c, A, Ainv) ** 2, axis=-1))
            m = np.minimum(m, np.abs(d - rad))
        for f1, f2, a in spheroids:
            v = geometry._nearest_offset(x, 0.5 * (f1 + f2), A, Ainv)
            h = 0.5 * (f2 - f1)
            s = np.sqrt(np.sum((v + h) ** 2, axis=-1)) + np.sqrt(np.sum((v - h) ** 2, axis=-1))
            m = np.minimum(m, np.abs(s - 2.0 * a))
        out.append(m.reshape(N, N, N))
    return np.stack(out)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_diamond_matches_oracle(pcmod, N):
    A = wl.FCC_CELL
    got = pcmod.eps_diamond(N, A, 1.0, 0.12, 0.11, 13.0, 1.0)
    ref = geometry.eps_edges_diamond(N, A, 1.0, 0.12, 0.11, 13.0, 1.0)
    diff = got != ref
    if diff.any():
        assert np.all(diamond_margin(N, A)[diff] <= 1e-12)
    assert 0.03 < np.mean(ref == 13.0) < 0.2
