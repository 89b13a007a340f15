"""pc_solve_init (a caller-provided initial block), the chunked pc_solve (opts.kchunk) and the two-pass path solve
through the C ABI.

- From the oracle's own eigenvectors (LAPACK on the oracle's operator at N = 8), rounded to complex64, the solve
  converges within a few LOBPCG iterations (the complex64 rounding of the start leaves a relative residual of about
  1e-4 here: |Op| ~ 1e4 times 6e-8, over lambda ~ 5); from a random complex64 block it reaches the same eigenvalues
  as pc_solve.
- A batch solved in chunks of two k-points (with eigenvectors and an initial block) gives the unchunked solve's
  eigenvalues and eigenvector subspaces, with each k-point's iterations and residuals in its own place.
- The two-pass path solve (even k-points from random blocks, odd ones from their neighbours' eigenvectors) gives the
  one-pass eigenvalues.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import eigs, geometry, mfd

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


def sphere_setup(N):
    s = wl.sc_single_sphere()
    eps = geometry.eps_edges(N, s.as_array(), s.eps_bg)
    return eps, 1.0 / eps


def oracle_vectors(N, m0, k, nb):
    kr = eigs.reduce_to_first_zone(k)
    Op = mfd.compensated_operator(N, kr, 1.0 / N, m0, mfd.penalty_gamma(1.0 / N, kr))
    w, V = eigs.lowest_dense(Op, nb)
    return w, V


def subspace_gap(U, V):
    """Largest sine of the principal angles between span(U) and span(V) (columns)."""
    qu, _ = np.linalg.qr(U)
    qv, _ = np.linalg.qr(V)
    s = np.linalg.svd(qu.conj().T @ qv, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - np.min(s) ** 2)))


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_init_from_oracle_eigenvectors(pcmod, precision):
    N, nb, tol = 8, 6, 1e-6
    eps, m0 = sphere_setup(N)
    # |k| large enough that the lowest compensation eigenvalue gamma |k|^2 (Proposition 3.1 at mode 0) lies above
    # the requested bands: the oracle's lowest eigenpairs are then the physical ones
    kpts = np.array([[1.9, 0.2, -0.4], [0.0, 1.7, 0.3]])
    x0 = np.empty((2, nb, 3, N, N, N), dtype=np.complex64)
    refs = []
    for b, k in enumerate(kpts):
        w, V = oracle_vectors(N, m0, k, nb)
        assert w[-1] < mfd.penalty_gamma(1.0 / N, k) * float(np.dot(k, k))
        refs.append(w)
        x0[b] = V.T.reshape(nb, 3, N, N, N).astype(np.complex64)
    S = pcmod.Solver(N, eps, precision=precision)
    base = S.solve(kpts, nb, tol)
    warm = S.solve(kpts, nb, tol, x0=torch.from_numpy(x0).cuda())
    assert base["status"] == 0 and warm["status"] == 0
    # the FP64 solve keeps the start's accuracy and needs a few iterations; the mixed solve starts in complex64 (the
    # start rounded again by its first Rayleigh-Ritz in complex64) and switches to its FP64-accurate phase first
    assert np.all(warm["iters"] <= (4 if precision == 0 else 15)), warm["iters"]
    assert np.all(base["iters"] >= (3 if precision == 0 else 2) * np.maximum(warm["iters"], 1)), (base["iters"],
                                                                                                   warm["iters"])
    for b in range(2):
        assert np.max(np.abs(warm["evals"][b] - refs[b]) / refs[b]) <= 1e-8
        assert np.max(np.abs(base["evals"][b] - refs[b]) / refs[b]) <= 1e-8
    assert np.max(warm["resid"]) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_init_random_block_gives_same_eigenvalues(pcmod, precision):
    N, nb, tol = 16, 8, 1e-8 if precision == 0 else 1e-6
    eps, _ = sphere_setup(N)
    kpts = np.array([[np.pi / 2, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 2.0, 0.5]])
    g = np.random.default_rng(3)
    x0 = (g.standard_normal((3, 5, 3, N, N, N)) + 1j * g.standard_normal((3, 5, 3, N, N, N))).astype(np.complex64)
    S = pcmod.Solver(N, eps, precision=precision)
    base = S.solve(kpts, nb, tol)
    warm = S.solve(kpts, nb, tol, x0=torch.from_numpy(x0).cuda())
    assert base["status"] == 0 and warm["status"] == 0
    assert np.max(np.abs(warm["evals"] - base["evals"]) / base["evals"]) <= 10 * tol
    assert np.max(warm["resid"]) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_chunked_solve_matches_unchunked(pcmod, precision):
    """Five k-points with kchunk = 2 (chunks of 2, 2, 1): eigenvalues within 10 tol of the unchunked solve, the same
    eigenvector subspaces (the first nbands columns; clusters are not cut at nbands here), iteration counts and
    residuals at the right k-point, and an initial block (pc_solve_init) taken at the right offset."""
    N, nb, tol = 8, 5, 1e-8 if precision == 0 else 1e-6
    eps, m0 = sphere_setup(N)
    kpts = np.array([[1.6, 0.0, 0.0], [2.9, 0.4, 0.0], [1.1, 1.1, 0.2], [0.0, 0.0, 0.0], [0.7, -2.0, 1.5]])
    full = pcmod.Solver(N, eps, precision=precision)
    chunked = pcmod.Solver(N, eps, precision=precision, kchunk=2)
    a = full.solve(kpts, nb, tol, want_vectors=True)
    b = chunked.solve(kpts, nb, tol, want_vectors=True)
    assert a["status"] == 0 and b["status"] == 0
    assert np.max(np.abs(a["evals"] - b["evals"]) / a["evals"]) <= 10 * tol
    assert np.max(b["resid"]) <= tol
    # each k-point's iteration count is its own: the initial block of a k-point does not depend on the chunking, so
    # the counts differ only through the reductions' rounding
    assert np.all(np.abs(a["iters"] - b["iters"]) <= 5), (a["iters"], b["iters"])
    Va = a["evecs"].cpu().numpy().reshape(5, nb, -1)
    Vb = b["evecs"].cpu().numpy().reshape(5, nb, -1)
    for k in range(5):
        # the subspace of the first nbands columns is unique only where band nbands + 1 is separated from band
        # nbands (at Gamma the cubic symmetry makes the second cluster threefold, and nbands = 5 cuts it)
        kr0 = eigs.reduce_to_first_zone(kpts[k])
        wk, _ = eigs.lowest_dense(mfd.compensated_operator(N, kr0, 1.0 / N, m0, mfd.penalty_gamma(1.0 / N, kr0)),
                                  nb + 1, skip=0 if np.any(kr0) else 3)
        if wk[nb] - wk[nb - 1] > 1e-3 * wk[nb]:
            assert subspace_gap(Va[k].T, Vb[k].T) <= 1e-4
        # and each is an eigenbasis of its own k-point's operator (oracle), so no chunk wrote another's slot
        kr = eigs.reduce_to_first_zone(kpts[k])
        Op = mfd.compensated_operator(N, kr, 1.0 / N, m0, mfd.penalty_gamma(1.0 / N, kr))
        X = Vb[k].T
        r = np.linalg.norm(Op @ X - X * b["evals"][k][None, :], axis=0) / (b["evals"][k] * np.linalg.norm(X, axis=0))
        assert np.max(r) <= 2 * tol
    # the initial block of k-point j is x0[j] in the chunked solve too: start from each k-point's own eigenvectors
    x0 = torch.from_numpy(Va.reshape(5, nb, 3, N, N, N).astype(np.complex64)).cuda()
    c = chunked.solve(kpts, nb, tol, x0=x0)
    assert c["status"] == 0
    assert np.all(c["iters"] <= (8 if precision == 0 else 15)), c["iters"]  # from complex64-rounded vectors, to tol
    assert np.max(np.abs(c["evals"] - a["evals"]) / a["evals"]) <= 10 * tol


def test_two_pass_path_matches_one_pass(pcmod):
    from paper_2503_19379_gb300 import bands
    w = wl.workload_fcc_32(npts=12)
    N = 16
    eps = geometry.eps_edges(N, w.structure.as_array(), w.structure.eps_bg)
    S = pcmod.Solver(N, eps, precision=1)
    one = S.solve(w.kpts, 8, 1e-6)
    two = bands.solve_path_two_pass(S, w.kpts, 8, 1e-6)
    assert one["status"] == 0 and two["status"] == 0
    assert np.max(np.abs(one["evals"] - two["evals"]) / one["evals"]) <= 1e-5
    assert np.max(two["resid"]) <= 1e-6
