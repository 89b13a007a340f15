"""Parity of every CUDA step (through the C ABI) with the FP64 oracle, on seeded inputs.

Tolerances (FP64 path): each stencil output is a signed sum of ~25 terms bounded by |Op| |x|, so rounding leaves
errors of a few ulp of |Op| |x|; comparisons use 1e-13 relative to the largest output. The FFT solve divides modes
by sigma(m) after O(log n) rounding steps: 1e-12 relative to the largest output. FP32 stencil: 1e-5.
Eigenvalues: 1e-10 relative (the requirement for the FP64 solve).
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import eigs, geometry, mfd, precond, rng, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    b.build()
    import paper_2503_19379_gb300 as p
    return p


def make_solver(pcmod, N, structure=None, **opts):
    s = structure or wl.sc_single_sphere()
    eps = geometry.eps_edges(N, s.as_array(), s.eps_bg)
    return pcmod.Solver(N, eps, **opts), 1.0 / eps


def rand_block(seed, shape):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


# ------------------------------------------------------------------------------------------- a0 geometry
@pytest.mark.parametrize("N,struct", [(6, wl.sc_single_sphere()), (16, wl.diamond_air_spheres()),
                                      (32, wl.fcc_spheres()), (16, wl.random_structure(11)),
                                      (12, wl.random_structure(5))])
def test_eps_spheres_bit_exact(pcmod, N, struct):
    got = pcmod.eps_spheres(N, struct.as_array(), struct.eps_bg)
    ref = geometry.eps_edges(N, struct.as_array(), struct.eps_bg)
    assert np.array_equal(got, ref)


# ------------------------------------------------------------------------------------------- a1 stencil
@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_apply_op_fp64(pcmod, N):
    S, m0 = make_solver(pcmod, N)
    g = np.random.default_rng(N)
    nb, m = 2, 2
    kpts = g.uniform(-3.5, 3.5, (nb, 3))
    gammas = g.uniform(1.0, 2.0 * N, nb)
    X = rand_block(N, (nb, m, 3 * N ** 3))
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(nb, m, 3, N, N, N))).cpu().numpy().reshape(nb, m, -1)
    for b in range(nb):
        Op = mfd.compensated_operator(N, kpts[b], 1.0 / N, m0, gammas[b])
        ref = (Op @ X[b].T).T
        assert np.max(np.abs(Y[b] - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_apply_op_double_float(pcmod, N):
    """complex128 block evaluated in double-float arithmetic (the phase-2 stencil of the mixed solve): rounding of
    ~2^-44 per operation, so 1e-11 relative to the largest output."""
    S, m0 = make_solver(pcmod, N)
    g = np.random.default_rng(N + 5)
    nb, m = 2, 3
    kpts = g.uniform(-3.5, 3.5, (nb, 3))
    gammas = np.array([2.0 * N, 7.25])
    X = rand_block(N + 3, (nb, m, 3 * N ** 3))
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(nb, m, 3, N, N, N)), double_float=True).cpu().numpy()
    Y = Y.reshape(nb, m, -1)
    for b in range(nb):
        ref = (mfd.compensated_operator(N, kpts[b], 1.0 / N, m0, gammas[b]) @ X[b].T).T
        assert np.max(np.abs(Y[b] - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_apply_op_fp32(pcmod, N):
    S, m0 = make_solver(pcmod, N)
    kpts = np.array([[0.4, -1.3, 2.2]])
    gammas = np.array([2.0 * N])
    X = rand_block(7, (1, 3, 3 * N ** 3)).astype(np.complex64)
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(1, 3, 3, N, N, N), torch.complex64)).cpu().numpy().reshape(1, 3, -1)
    Op = mfd.compensated_operator(N, kpts[0], 1.0 / N, m0, gammas[0])
    ref = (Op @ X[0].astype(np.complex128).T).T
    assert np.max(np.abs(Y[0] - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_apply_op_gamma_point_annihilates_constants(pcmod):
    N = 16
    S, _ = make_solver(pcmod, N)
    X = np.zeros((1, 3, 3, N, N, N), dtype=np.complex128)
    for c in range(3):
        X[0, c, c] = 1.0 + 0.5j
    Y = S.apply_op(np.zeros((1, 3)), np.array([32.0]), to_dev(X)).cpu().numpy()
    assert np.max(np.abs(Y)) == 0.0


@pytest.mark.parametrize("N", [8, 16])
def test_apply_half_and_recompute_norms(pcmod, N):
    S, m0 = make_solver(pcmod, N)
    kpts = np.array([[0.3, 0.9, -1.7], [2.0, 0.0, 0.5]])
    X = rand_block(3, (2, 2, 3 * N ** 3))
    E, Cc = S.apply_half(kpts, to_dev(X.reshape(2, 2, 3, N, N, N)))
    E = E.cpu().numpy().reshape(2, 2, -1)
    Cc = Cc.cpu().numpy().reshape(2, 2, -1)
    nrm = S.recompute_norms(kpts, to_dev(X.reshape(2, 2, 3, N, N, N))).cpu().numpy()
    for b in range(2):
        Ah, B = mfd.half_operators(N, kpts[b], 1.0 / N)
        Eref = (Ah @ X[b].T).T
        Cref = (B @ X[b].T).T
        assert np.max(np.abs(E[b] - Eref)) <= 1e-13 * np.max(np.abs(Eref))
        assert np.max(np.abs(Cc[b] - Cref)) <= 1e-13 * np.max(np.abs(Cref))
        ref = np.stack([np.sum(m0.ravel()[None, :] * np.abs(Eref) ** 2, 1), np.sum(np.abs(Cref) ** 2, 1),
                        np.sum(np.abs(X[b]) ** 2, 1)], 1)
        assert np.allclose(nrm[b], ref, rtol=1e-12)


# ------------------------------------------------------------------------------------------- a2 preconditioner
@pytest.mark.parametrize("N,variant", [(8, 0), (16, 0), (32, 0), (64, 0), (16, 1)])
def test_apply_precond_fp64(pcmod, N, variant):
    S, _ = make_solver(pcmod, N, precond=variant)
    g = np.random.default_rng(100 + N)
    kpts = np.vstack([g.uniform(-3, 3, (2, 3)), np.zeros((1, 3))])
    gammas = np.array([2.0 * N, 7.0, 2.0 * N])
    R = rand_block(N + 1, (3, 2, 3 * N ** 3))
    W = S.apply_precond(kpts, gammas, to_dev(R.reshape(3, 2, 3, N, N, N))).cpu().numpy().reshape(3, 2, -1)
    name = "laplacian" if variant else "gamma"
    for b in range(3):
        for j in range(2):
            ref = precond.apply_preconditioner(R[b, j], N, 1.0 / N, kpts[b], gammas[b], 1, name).ravel()
            assert np.max(np.abs(W[b, j] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,variant", [(8, 0), (16, 0), (32, 0), (64, 0), (32, 1), (128, 0)])
def test_apply_precond_fp32(pcmod, N, variant):
    """complex64 solve (two-level register/shared-memory line FFTs in natural order for N <= 128, the shared-memory
    radix-2 FFTs above) against the FP64 oracle, including a k = 0 point whose zero mode is singular and maps to
    zero."""
    S, _ = make_solver(pcmod, N, precond=variant)
    kpts = np.array([[1.1, -0.2, 0.7], [0.0, 0.0, 0.0]])
    gammas = [64.0, 2.0 * N]
    nf = 1 if N > 64 else 2
    R = rand_block(5 + N, (2, nf, 3 * N ** 3)).astype(np.complex64)
    W = S.apply_precond(kpts, gammas, to_dev(R.reshape(2, nf, 3, N, N, N), torch.complex64)).cpu().numpy()
    W = W.reshape(2, nf, -1)
    name = "laplacian" if variant else "gamma"
    for b in range(2):
        for j in range(nf):
            ref = precond.apply_preconditioner(R[b, j].astype(np.complex128), N, 1.0 / N, kpts[b], gammas[b], 1,
                                               name).ravel()
            assert np.max(np.abs(W[b, j] - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_precond_inverts_operator_at_unit_eps(pcmod):
    """P^{-1} Op = I when M0 = I (the preconditioner is the operator), applied through both kernels."""
    N = 16
    S, _ = make_solver(pcmod, N, structure=wl.homogeneous(1.0))
    kpts = np.array([[0.5, 1.5, -2.5]])
    X = rand_block(9, (1, 2, 3, N, N, N))
    Y = S.apply_op(kpts, [32.0], to_dev(X))
    Z = S.apply_precond(kpts, [32.0], Y).cpu().numpy()
    assert np.max(np.abs(Z - X)) <= 1e-11 * np.max(np.abs(X))


# ------------------------------------------------------------------------------------------- a3 / a5 dense blocks
@pytest.mark.parametrize("p,q,L", [(36, 36, 98304), (20, 12, 3 * 8 ** 3), (64, 64, 5000), (1, 7, 37)])
def test_gram(pcmod, p, q, L):
    A = rand_block(p, (3, p, L))
    B = rand_block(q + 1, (3, q, L))
    G = pcmod.gram(to_dev(A), to_dev(B)).cpu().numpy()
    ref = np.einsum("bil,bjl->bij", A.conj(), B)
    assert np.max(np.abs(G - ref)) <= 1e-13 * np.max(np.abs(ref)) * np.sqrt(L)


@pytest.mark.parametrize("p,L", [(36, 98304), (48, 5000), (54, 4000), (64, 3000), (13, 777), (1, 37)])
def test_gram_pair(pcmod, p, L):
    """Upper triangles of S^H S and S^H AS, lower triangles their conjugate mirrors; AS = d * S with d > 0 is the
    image of S under a Hermitian operator, so both products are Hermitian."""
    Sb = rand_block(p, (2, p, L))
    ASb = Sb * np.random.default_rng(p + 100).uniform(0.5, 2.0, L)[None, None, :]
    G, H = pcmod.gram_pair(to_dev(Sb), to_dev(ASb))
    G, H = G.cpu().numpy(), H.cpu().numpy()
    Gr = np.einsum("bil,bjl->bij", Sb.conj(), Sb)
    Hr = np.einsum("bil,bjl->bij", Sb.conj(), ASb)
    iu = np.triu_indices(p)
    tol = 1e-13 * np.sqrt(L) * np.max(np.abs(Gr))
    for b in range(2):
        assert np.max(np.abs(G[b][iu] - Gr[b][iu])) <= tol
        assert np.max(np.abs(H[b][iu] - Hr[b][iu])) <= tol
        assert np.array_equal(G[b], G[b].conj().T) and np.array_equal(H[b], H[b].conj().T)


@pytest.mark.parametrize("p,q,L", [(36, 12, 98304), (24, 12, 1000), (64, 33, 777)])
def test_block_update(pcmod, p, q, L):
    Sb = rand_block(1, (2, p, L))
    Cm = rand_block(2, (2, p, q))
    Y = pcmod.block_update(to_dev(Sb), to_dev(Cm)).cpu().numpy()
    ref = np.einsum("bil,biq->bql", Sb, Cm)
    assert np.max(np.abs(Y - ref)) <= 1e-14 * np.max(np.abs(ref)) * p


@pytest.mark.parametrize("q", [5, 10, 12, 16, 19, 21, 24, 33])
def test_block_update_complex64(pcmod, q):
    # every column-group width of the complex64 kernel (8, 10, 12, 16, 20, 24; 33 = two groups) and a ragged tail
    p, L = 38, 70001
    Sb = rand_block(3, (2, p, L))
    Cm = rand_block(4, (2, p, q))
    S32 = to_dev(Sb, torch.complex64)
    Y = pcmod.block_update(S32, to_dev(Cm)).cpu().numpy()
    # reference from the complex64-rounded inputs in FP64; FP32 products and sums: error ~eps32 sqrt(p) |S| |C|
    ref = np.einsum("bil,biq->bql", S32.cpu().numpy().astype(np.complex128), Cm)
    bound = 8 * np.finfo(np.float32).eps * np.sqrt(p) * np.max(np.abs(Sb)) * np.max(np.abs(Cm)) * 2
    assert Y.dtype == np.complex64 and Y.shape == (2, q, L)
    assert np.max(np.abs(Y - ref)) <= bound


# ------------------------------------------------------------------------------------------- a4 small dense
@pytest.mark.parametrize("n", [1, 2, 13, 36, 64])
def test_eigh_batched(pcmod, n):
    A = rand_block(n, (4, n, n))
    A = A + A.conj().transpose(0, 2, 1)
    A[1] = np.diag(np.arange(n, dtype=float))  # already diagonal
    w, V = pcmod.eigh_batched(to_dev(A))
    w = w.cpu().numpy()
    V = V.cpu().numpy()
    for b in range(4):
        ref = np.linalg.eigvalsh(A[b])
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.max(np.abs(w[b] - ref)) <= 1e-13 * scale * n
        assert np.max(np.abs(A[b] @ V[b] - V[b] * w[b][None, :])) <= 1e-12 * scale
        assert np.max(np.abs(V[b].conj().T @ V[b] - np.eye(n))) <= 1e-12


@pytest.mark.parametrize("L,n,m", [(300, 30, 8), (400, 48, 16), (400, 64, 40), (400, 64, 64), (300, 40, 33)])
def test_rayleigh_ritz(pcmod, L, n, m):
    """Pencils up to the 64-column maximum: Householder steps with more than 32 trailing rows (two row warps), more
    than 32 wanted pairs, and both back-transformation forms (block-parallel when its work space fits)."""
    import scipy.linalg as sla
    g = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rand_block(5, (L, L)))
    lam = np.sort(g.uniform(0.5, 1e4, L))
    A = (Q * lam) @ Q.conj().T
    Sb = rand_block(6, (L, n)) * np.logspace(0, -6, n)[None, :]  # badly scaled columns
    G = Sb.conj().T @ Sb
    H = Sb.conj().T @ A @ Sb
    theta, coef, rank = pcmod.rayleigh_ritz(to_dev(G[None]), to_dev(H[None]), m)
    theta = theta.cpu().numpy()[0]
    coef = coef.cpu().numpy()[0]
    ref = sla.eigh(H, G, eigvals_only=True)[:m]
    assert int(rank.cpu()[0]) == n
    assert np.max(np.abs(theta - ref) / ref) <= 1e-10
    Xr = Sb @ coef
    assert np.max(np.abs(Xr.conj().T @ Xr - np.eye(m))) <= 1e-8
    assert np.max(np.abs(Xr.conj().T @ A @ Xr - np.diag(theta))) <= 1e-8 * lam.max()


def test_rayleigh_ritz_degenerate_clusters(pcmod):
    """A search space that contains a 3-fold and a 2-fold eigenspace of the operator: the pencil has exactly repeated
    eigenvalues, whose Ritz vectors come out of inverse iteration with Gram-Schmidt inside each cluster."""
    g = np.random.default_rng(11)
    L, n, m = 300, 48, 16
    Q, _ = np.linalg.qr(rand_block(12, (L, L)))
    lam = np.sort(g.uniform(3.0, 50.0, L))
    lam[:3] = 1.0
    lam[3:5] = 2.0
    A = (Q * lam) @ Q.conj().T
    Sb = np.concatenate([Q[:, :5] @ rand_block(13, (5, 5)), rand_block(14, (L, n - 5))], axis=1)
    G = Sb.conj().T @ Sb
    H = Sb.conj().T @ A @ Sb
    theta, coef, rank = pcmod.rayleigh_ritz(to_dev(G[None]), to_dev(H[None]), m)
    theta = theta.cpu().numpy()[0]
    coef = coef.cpu().numpy()[0]
    assert int(rank.cpu()[0]) == n
    assert np.allclose(theta[:5], [1, 1, 1, 2, 2], rtol=0, atol=1e-11)
    ref = np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(G), np.linalg.solve(np.linalg.cholesky(G), H).conj().T))
    assert np.max(np.abs(theta - np.sort(ref)[:m]) / np.sort(ref)[:m]) <= 1e-10
    Xr = Sb @ coef
    assert np.max(np.abs(Xr.conj().T @ Xr - np.eye(m))) <= 1e-9
    assert np.max(np.abs(Xr.conj().T @ A @ Xr - np.diag(theta))) <= 1e-9 * lam.max()
    # the first five are exact eigenvectors of the operator
    assert np.max(np.abs(A @ Xr[:, :5] - Xr[:, :5] * theta[None, :5])) <= 1e-9 * lam.max()


def test_rayleigh_ritz_drops_dependent_directions(pcmod):
    L, n, m = 200, 12, 4
    Sb = rand_block(8, (L, n))
    Sb[:, 11] = Sb[:, 3] + Sb[:, 5]  # exactly dependent column
    A = np.diag(np.linspace(1, 10, L)).astype(np.complex128)
    G = Sb.conj().T @ Sb
    H = Sb.conj().T @ A @ Sb
    theta, coef, rank = pcmod.rayleigh_ritz(to_dev(G[None]), to_dev(H[None]), m, 1e-12)
    assert int(rank.cpu()[0]) == n - 1
    Q, _ = np.linalg.qr(Sb[:, :11])
    ref = np.linalg.eigvalsh(Q.conj().T @ A @ Q)[:m]
    assert np.allclose(theta.cpu().numpy()[0], ref, rtol=1e-10)


def test_residual(pcmod):
    X = rand_block(1, (3, 5, 1000))
    AX = rand_block(2, (3, 5, 1000))
    th = np.random.default_rng(3).uniform(1, 5, (3, 5))
    R, nr = pcmod.residual(to_dev(X), to_dev(AX), torch.from_numpy(th).cuda())
    ref = AX - X * th[:, :, None]
    assert np.max(np.abs(R.cpu().numpy() - ref)) <= 1e-14 * np.max(np.abs(ref))
    nr = nr.cpu().numpy()
    assert np.allclose(nr[..., 0], np.linalg.norm(ref, axis=2), rtol=1e-13)
    assert np.allclose(nr[..., 1], np.linalg.norm(X, axis=2), rtol=1e-13)


def test_init_block_matches_oracle_generator(pcmod):
    L, m = 3 * 8 ** 3, 4
    X = pcmod.init_block(2, L, m, 1234, 5).cpu().numpy()
    for b in range(2):
        ref = rng.initial_block(1234, 5 + b, L, m).T
        assert np.max(np.abs(X[b] - ref)) <= 1e-13


# ------------------------------------------------------------------------------------------- full solves
def test_solve_homogeneous_closed_form(pcmod):
    """eps = 1 at N = 8: the lowest eigenvalues equal the closed-form spectrum (fixed gamma = 100, large enough to keep
    the compensation values gamma sigma above the 8th band; the FP64 residual floor eps |Op| / lambda stays ~1e-11)."""
    N = 8
    S, _ = make_solver(pcmod, N, structure=wl.homogeneous(1.0), gamma_override=100.0)
    k = np.array([0.3, -0.7, 1.1])
    out = S.solve(k[None], 8, 1e-10)
    ref = spectrum.homogeneous_spectrum(N, 1.0 / N, k, 1.0, 100.0)[:8]
    assert out["status"] == 0
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-10


def test_solve_sc_sphere_N16_matches_oracle(pcmod):
    """SC lattice, eps=13 sphere r=0.25, N=16, k=(pi/2,0,0), 8 bands, tol 1e-10 vs the oracle (ARPACK)."""
    w = wl.workload_sc_sphere_16()
    S, m0 = make_solver(pcmod, w.N, structure=w.structure)
    out = S.solve(w.kpts, w.nbands, w.tol, want_vectors=True)
    assert out["status"] == 0
    h = 1.0 / w.N
    k = w.kpts[0]
    Op = mfd.compensated_operator(w.N, k, h, m0, mfd.penalty_gamma(h, k))
    ref, _ = eigs.lowest_sparse(Op, w.nbands)
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-10
    assert np.all(out["resid"][0] <= w.tol)
    V = out["evecs"][0].reshape(w.nbands, -1).cpu().numpy()
    assert np.max(np.abs(V.conj() @ V.T - np.eye(w.nbands))) <= 1e-9
    Y = (Op @ V.T).T
    r = np.linalg.norm(Y - out["evals"][0][:, None] * V, axis=1) / out["evals"][0]
    assert np.all(r <= 2 * w.tol)


def test_solve_gamma_point_deflation(pcmod):
    N = 8
    S, m0 = make_solver(pcmod, N)
    out = S.solve(np.zeros((1, 3)), 6, 1e-10)
    Op = mfd.compensated_operator(N, np.zeros(3), 1.0 / N, m0, 2.0 * N)
    ref, _ = eigs.lowest_dense(Op, 6, skip=3)
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-10


def test_solve_reduces_k_into_first_zone(pcmod):
    """k = (0, 2 pi, 0) is equivalent to Gamma and is solved as k = 0."""
    N = 8
    S, _ = make_solver(pcmod, N)
    a = S.solve(np.array([[0.0, 2 * np.pi, 0.0]]), 6, 1e-10)["evals"]
    b = S.solve(np.zeros((1, 3)), 6, 1e-10)["evals"]
    assert np.max(np.abs(a - b) / b) <= 1e-10


def test_algorithm_4_1_gamma_doubling(pcmod):
    """With a deliberately small gamma the compensation eigenvalue gamma |k|^2 enters the lowest bands; Algorithm 4.1
    detects it and doubles gamma until the result is the physical spectrum of A M0 A'."""
    N = 8
    S, m0 = make_solver(pcmod, N, gamma_override=8.0, maxiter=1500)
    k = np.array([0.3, 0.1, 0.2])
    out = S.solve(k[None], 6, 1e-9)
    wa = np.linalg.eigvalsh(mfd.curl_part(N, k, 1.0 / N, m0).toarray())
    phys = np.sort(wa[wa > 1e-10 * wa.max()])[:6]
    # gamma |k|^2 = 1.12 starts below the 3rd band; 8 * 2^5 = 256 puts it (35.8) above the 6th (18.45); each round
    # re-finds the compensation vector while it is among the lowest eigenvalues, as Algorithm 4.1 intends
    assert out["status"] == 0
    assert np.max(np.abs(out["evals"][0] - phys) / phys) <= 1e-9


def oracle_golden(name):
    """The oracle's eigenvalues at sampled k-points of a benchmark path (tests/golden/make_oracle_evals.py: the FP64
    oracle's Algorithm 4.1 + LOBPCG to a relative residual of 1e-8)."""
    path = os.path.join(os.path.dirname(__file__), "golden", f"oracle_evals_{name}.json")
    with open(path) as f:
        doc = json.load(f)
    idx = [r["kidx"] for r in doc["kpoints"]]
    return idx, np.array([r["evals"] for r in doc["kpoints"]]), np.array([r["k"] for r in doc["kpoints"]])


def test_solve_fcc_batch_matches_oracle(pcmod):
    """FCC spheres at N = 32: the sampled k-points of the path (Gamma, X folded onto Gamma, interior points, L) solved
    together by the FP64 solve; every eigenvalue matches the oracle's to 1e-10 relative."""
    w = wl.workload_fcc_32()
    S, m0 = make_solver(pcmod, w.N, structure=w.structure)
    idx, ref, kref = oracle_golden(w.name)
    assert np.array_equal(kref, w.kpts[idx])
    out = S.solve(w.kpts[idx], w.nbands, 1e-8)
    assert out["status"] == 0
    assert np.max(np.abs(out["evals"] - ref) / ref) <= 1e-10


# ------------------------------------------------------------------------------------------- mixed precision
def test_mixed_solve_sc_sphere_matches_oracle(pcmod):
    """Mixed precision (complex64 search space, FP64 block/residual/RR): eigenvalues within 1e-6 relative of the
    FP64 oracle and every returned eigenvector has an FP64 relative residual <= tol against the oracle operator."""
    w = wl.workload_sc_sphere_16()
    tol = 1e-6
    S, m0 = make_solver(pcmod, w.N, structure=w.structure, precision=1)
    out = S.solve(w.kpts, w.nbands, tol, want_vectors=True)
    assert out["status"] == 0
    h = 1.0 / w.N
    k = w.kpts[0]
    Op = mfd.compensated_operator(w.N, k, h, m0, mfd.penalty_gamma(h, k))
    ref, _ = eigs.lowest_sparse(Op, w.nbands)
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-6
    V = out["evecs"][0].reshape(w.nbands, -1).cpu().numpy()
    lam = out["evals"][0]
    r = np.linalg.norm((Op @ V.T).T - lam[:, None] * V, axis=1) / (lam * np.linalg.norm(V, axis=1))
    assert np.all(r <= tol * 1.01), r


def test_mixed_fcc_batch_matches_fp64(pcmod):
    """FCC spheres at N = 32 including Gamma, X (folded onto Gamma) and L: the mixed solve agrees with the FP64
    solve to 1e-6 relative on every eigenvalue."""
    w = wl.workload_fcc_32()
    idx = [0, 3, 10, 20, 39]
    kp = w.kpts[idx]
    S64, _ = make_solver(pcmod, w.N, structure=w.structure)
    S32, _ = make_solver(pcmod, w.N, structure=w.structure, precision=1)
    a = S64.solve(kp, w.nbands, w.tol)
    b = S32.solve(kp, w.nbands, w.tol)
    assert a["status"] == 0 and b["status"] == 0
    assert np.max(np.abs(a["evals"] - b["evals"]) / a["evals"]) <= 1e-6
    assert np.all(b["resid"] <= w.tol)


@pytest.mark.parametrize("groups", [2, 4])
def test_mixed_groups_match_one(pcmod, groups):
    """The multi-stream schedule (k-points in 2 or 4 groups, served in turn) computes the same thing as one group:
    the same eigenvalues to far below the tolerance, every residual within tol, on 10 FCC k-points (Gamma, X and L
    among them, so the groups hold a k = 0 point or a folded one). Chunked reductions depend on the batch size, so
    the runs differ in rounding, not in the converged eigenpairs."""
    w = wl.workload_fcc_32()
    idx = [0, 3, 6, 10, 14, 20, 24, 28, 33, 39]
    kp = w.kpts[idx]
    S1, _ = make_solver(pcmod, w.N, structure=w.structure, precision=1, groups=1)
    S2, _ = make_solver(pcmod, w.N, structure=w.structure, precision=1, groups=groups)
    a = S1.solve(kp, w.nbands, w.tol)
    b = S2.solve(kp, w.nbands, w.tol)
    assert a["status"] == 0 and b["status"] == 0
    assert np.max(np.abs(a["evals"] - b["evals"]) / a["evals"]) <= 1e-8
    assert np.all(b["resid"] <= w.tol)


def test_mixed_fp64_finish_of_capped_kpoints(pcmod):
    # a phase-2 cap of 30 iterations hands most k-points of an fcc-spheres-N32 slice to the FP64 solve, which starts
    # from their double-float blocks; the result is the plain FP64 solve's, with eigenvectors and residuals to tol
    w = wl.workload_fcc_32()
    eps = pcmod.eps_spheres(w.N, w.structure.as_array(), w.structure.eps_bg)
    ks = w.kpts[[3, 11, 20, 29]]
    mixed = pcmod.Solver(w.N, eps, precision=pcmod.pc.PC_PREC_MIXED, maxiter=30)
    out = mixed.solve(ks, w.nbands, w.tol, want_vectors=True)
    ref = pcmod.Solver(w.N, eps).solve(ks, w.nbands, w.tol)
    assert out["status"] == 0 and ref["status"] == 0
    assert out["fp64_finish"].sum() >= 1
    assert np.all(out["resid"] <= w.tol)
    assert np.max(np.abs(out["evals"] - ref["evals"]) / ref["evals"]) <= 10 * w.tol
    # the handed-over k-points' eigenvectors: unit norm, Rayleigh quotients equal to their eigenvalues
    for b in np.nonzero(out["fp64_finish"])[0]:
        V = out["evecs"][b:b + 1]
        kr = ks[b:b + 1] - 2 * np.pi * np.round(ks[b:b + 1] / (2 * np.pi))  # the solver's reduced k
        gam = np.full(1, 2.0 * max(w.N, 1.0 / float(np.sum(kr * kr))))
        AV = mixed.apply_op(kr, gam, V)
        num = torch.sum(V.conj() * AV, dim=(2, 3, 4, 5)).real.cpu().numpy()[0]
        nrm = torch.sum(V.conj() * V, dim=(2, 3, 4, 5)).real.cpu().numpy()[0]
        assert np.allclose(nrm, 1.0, atol=1e-10)
        assert np.max(np.abs(num / nrm - out["evals"][b]) / out["evals"][b]) <= 10 * w.tol
    mixed.close()


def test_mixed_full_benchmark_batch(pcmod):
    """The fcc-spheres-N32 configuration as a benchmark runs it: all 40 FCC k-points in one mixed solve with the
    default four k-point groups on four streams. Every residual reported within tol; at the oracle's sampled k-points
    (Gamma, X, interior points, L) the eigenvalues equal the oracle's to 1e-6 relative, and the residual of every
    returned eigenvector, recomputed with the oracle's operator (eq. Ker_comp at the penalty of eq. pnt_number),
    is within 1.01 tol."""
    w = wl.workload_fcc_32()
    S32, m0 = make_solver(pcmod, w.N, structure=w.structure, precision=1)
    b = S32.solve(w.kpts, w.nbands, w.tol, want_vectors=True)
    assert b["status"] == 0
    assert np.all(b["resid"] <= w.tol)
    assert np.max(b["iters"]) <= 150
    idx, ref, _ = oracle_golden(w.name)
    assert np.max(np.abs(b["evals"][idx] - ref) / ref) <= 1e-6
    h = 1.0 / w.N
    for i in idx:
        k = eigs.reduce_to_first_zone(w.kpts[i])
        Op = mfd.compensated_operator(w.N, k, h, m0, mfd.penalty_gamma(h, k))
        V = b["evecs"][i].reshape(w.nbands, -1).cpu().numpy()
        lam = b["evals"][i]
        r = np.linalg.norm((Op @ V.T).T - lam[:, None] * V, axis=1) / (lam * np.linalg.norm(V, axis=1))
        assert np.all(r <= 1.01 * w.tol), (i, r)


def test_mixed_diamond_benchmark_batch(pcmod):
    """The diamond-air-N64 configuration as the benchmark runs it (60 k-points of the FCC path, 12 bands, N = 64, the
    mixed solve with its default four k-point groups): every reported residual within tol; at the oracle's sampled
    k-points (Gamma with its 6-fold clusters, an interior point of Gamma-X, and L with its 8-fold cluster) the
    eigenvalues equal the oracle's to 1e-6 relative, and the residual of every returned eigenvector, recomputed with
    the oracle's operator, is within 1.01 tol."""
    w = wl.workload_diamond_64()
    S32, m0 = make_solver(pcmod, w.N, structure=w.structure, precision=1)
    b = S32.solve(w.kpts, w.nbands, w.tol, want_vectors=True)
    assert b["status"] == 0
    assert np.all(b["resid"] <= w.tol)
    idx, ref, kref = oracle_golden(w.name)
    assert np.array_equal(kref, w.kpts[idx])
    assert np.max(np.abs(b["evals"][idx] - ref) / ref) <= 1e-6
    h = 1.0 / w.N
    for i in idx:
        k = eigs.reduce_to_first_zone(w.kpts[i])
        Op = mfd.compensated_operator(w.N, k, h, m0, mfd.penalty_gamma(h, k))
        V = b["evecs"][i].reshape(w.nbands, -1).cpu().numpy()
        lam = b["evals"][i]
        r = np.linalg.norm((Op @ V.T).T - lam[:, None] * V, axis=1) / (lam * np.linalg.norm(V, axis=1))
        assert np.all(r <= 1.01 * w.tol), (i, r)
