"""General lattices (Section 2's coordinate change x = A y, Section 4.2.2: D_hat_i = sum_j b_ji K_j + i L_i) through
the C ABI against the oracle's lattice operators: the edge permittivity of a primitive cell, the operator (complex128
and complex64), the half-apply and Algorithm 4.1 norms, the preconditioner with the lattice symbols, and FP64 solves
against the closed form and a dense LAPACK solve, on triclinic, FCC and BCC cells."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import eigs, geometry, mfd, precond, spectrum  # noqa: E402

TRICLINIC = np.array([[1.0, 0.3, 0.1], [0.2, 1.1, -0.4], [0.05, 0.25, 0.9]])
FCC = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
BCC = 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])
LATTICES = {"triclinic": TRICLINIC, "fcc": FCC, "bcc": BCC}
SPHERES = np.array([[0.05, 0.1, -0.02, 0.21, 13.0], [0.31, 0.12, 0.27, 0.08, 5.0]])


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    b.build()
    import paper_2503_19379_gb300 as p
    return p


def rand_block(seed, shape):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def lattice_m0(N, A):
    return 1.0 / geometry.eps_edges(N, SPHERES, 1.0, A)


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_eps_spheres_lattice_matches_oracle(pcmod, name):
    """pc_eps_spheres_lattice equals the oracle's lattice geometry; an edge may differ only where its distance to a
    sphere surface is within rounding of the radius (the two sides form A y and A^{-1}(x - c) in different orders)."""
    N = 16
    A = LATTICES[name]
    got = pcmod.eps_spheres_lattice(N, A, SPHERES, 1.0)
    ref = geometry.eps_edges(N, SPHERES, 1.0, A)
    bad = np.argwhere(got != ref)
    for axis, z, y, x in bad:
        pos = geometry.edge_positions(N, axis)[z, y, x] @ A.T
        d = [abs(geometry._lattice_distance(pos[None, :], s[:3], A, np.linalg.inv(A))[0] - s[3]) for s in SPHERES]
        assert min(d) < 1e-9
    assert len(bad) <= 3
    assert np.any(ref == 13.0) and np.any(ref == 5.0) and np.any(ref == 1.0)


@pytest.mark.parametrize("name,korder", [("triclinic", 1), ("fcc", 1), ("bcc", 2), ("triclinic", 3)])
def test_apply_op_lattice_fp64(pcmod, name, korder):
    N = 8
    A = LATTICES[name]
    m0 = lattice_m0(N, A)
    S = pcmod.Solver(N, 1.0 / m0, lattice=A, order=korder)
    g = np.random.default_rng(7 * korder + len(name))
    kpts = g.uniform(-3.5, 3.5, (2, 3))
    gammas = g.uniform(1.0, 2.0 * N, 2)
    X = rand_block(N + korder, (2, 2, 3 * N ** 3))
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(2, 2, 3, N, N, N))).cpu().numpy().reshape(2, 2, -1)
    for b in range(2):
        Op = mfd.compensated_operator(N, kpts[b], 1.0 / N, m0, gammas[b], korder, A)
        ref = (Op @ X[b].T).T
        assert np.max(np.abs(Y[b] - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_apply_op_lattice_fp32(pcmod):
    N = 16
    A = TRICLINIC
    m0 = lattice_m0(N, A)
    S = pcmod.Solver(N, 1.0 / m0, lattice=A)
    kpts = np.array([[0.4, -1.3, 2.2], [0.0, 0.0, 0.0]])
    gammas = np.array([2.0 * N, 5.0])
    X = rand_block(11, (2, 2, 3 * N ** 3)).astype(np.complex64)
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(2, 2, 3, N, N, N), torch.complex64)).cpu().numpy()
    Y = Y.reshape(2, 2, -1)
    for b in range(2):
        Op = mfd.compensated_operator(N, kpts[b], 1.0 / N, m0, gammas[b], 1, A)
        ref = (Op @ X[b].astype(np.complex128).T).T
        assert np.max(np.abs(Y[b] - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("korder", [1, 3])
def test_apply_half_and_recompute_norms_lattice(pcmod, korder):
    N = 8
    A = FCC
    m0 = lattice_m0(N, A)
    S = pcmod.Solver(N, 1.0 / m0, lattice=A, order=korder)
    kpts = np.array([[0.3, 0.9, -1.7], [2.0, 0.0, 0.5]])
    X = rand_block(3 + korder, (2, 2, 3 * N ** 3))
    E, Cc = S.apply_half(kpts, to_dev(X.reshape(2, 2, 3, N, N, N)))
    E = E.cpu().numpy().reshape(2, 2, -1)
    Cc = Cc.cpu().numpy().reshape(2, 2, -1)
    nrm = S.recompute_norms(kpts, to_dev(X.reshape(2, 2, 3, N, N, N))).cpu().numpy()
    for b in range(2):
        Ah, B = mfd.half_operators(N, kpts[b], 1.0 / N, korder, A)
        Eref = (Ah @ X[b].T).T
        Cref = (B @ X[b].T).T
        assert np.max(np.abs(E[b] - Eref)) <= 1e-13 * np.max(np.abs(Eref))
        assert np.max(np.abs(Cc[b] - Cref)) <= 1e-13 * np.max(np.abs(Cref))
        ref = np.stack([np.sum(m0.ravel()[None, :] * np.abs(Eref) ** 2, 1), np.sum(np.abs(Cref) ** 2, 1),
                        np.sum(np.abs(X[b]) ** 2, 1)], 1)
        assert np.allclose(nrm[b], ref, rtol=1e-12)


@pytest.mark.parametrize("name,korder,variant", [("triclinic", 1, 0), ("bcc", 2, 0), ("fcc", 1, 1)])
def test_apply_precond_lattice(pcmod, name, korder, variant):
    """complex128 to 1e-12 and complex64 to 2e-5 against the oracle's FFT solve with the lattice symbols; the
    k = 0 mode-0 pseudo-inverse included."""
    N = 16
    A = LATTICES[name]
    S = pcmod.Solver(N, np.ones((3, N, N, N)), lattice=A, precond=variant, order=korder)
    g = np.random.default_rng(300 + korder)
    kpts = np.vstack([g.uniform(-3, 3, (2, 3)), np.zeros((1, 3))])
    gammas = np.array([2.0 * N, 7.0, 2.0 * N])
    R = rand_block(N + korder, (3, 2, 3 * N ** 3))
    W = S.apply_precond(kpts, gammas, to_dev(R.reshape(3, 2, 3, N, N, N))).cpu().numpy().reshape(3, 2, -1)
    W32 = S.apply_precond(kpts, gammas, to_dev(R.reshape(3, 2, 3, N, N, N), torch.complex64)).cpu().numpy()
    W32 = W32.reshape(3, 2, -1)
    vname = "laplacian" if variant else "gamma"
    for b in range(3):
        for j in range(2):
            ref = precond.apply_preconditioner(R[b, j], N, 1.0 / N, kpts[b], gammas[b], korder, vname, A).ravel()
            assert np.max(np.abs(W[b, j] - ref)) <= 1e-12 * np.max(np.abs(ref))
            assert np.max(np.abs(W32[b, j] - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_precond_inverts_operator_lattice(pcmod):
    """At eps = 1 the preconditioner with the lattice symbols inverts the lattice stencil, both on the GPU: pins the
    symbol tables against the stencil independently of the oracle."""
    N = 16
    S = pcmod.Solver(N, np.ones((3, N, N, N)), lattice=TRICLINIC)
    kpts = np.array([[0.5, 1.5, -2.5]])
    X = rand_block(21, (1, 2, 3, N, N, N))
    Z = S.apply_precond(kpts, [32.0], S.apply_op(kpts, [32.0], to_dev(X))).cpu().numpy()
    assert np.max(np.abs(Z - X)) <= 1e-11 * np.max(np.abs(X))


# The residual target tol |lambda| |x| must stay above the rounding floor of Op x, about 1e-16 gamma sigma_max |x|
# (sigma_max = 1025 on the FCC cell at N = 8): gamma is kept just large enough to hold the compensation values above
# the requested bands, and tol = 1e-9.
@pytest.mark.parametrize("name", ["fcc", "triclinic"])
def test_solve_homogeneous_lattice_closed_form(pcmod, name):
    """eps = 1 on a primitive cell at N = 8: the lowest 8 eigenvalues equal the lattice closed form (gamma = 100:
    the lowest compensation value gamma |k|^2 = 179 lies above the 8th band)."""
    N = 8
    A = LATTICES[name]
    S = pcmod.Solver(N, np.ones((3, N, N, N)), lattice=A, gamma_override=100.0)
    k = np.array([0.3, -0.7, 1.1])
    out = S.solve(k[None], 8, 1e-9)
    ref = spectrum.homogeneous_physical_spectrum(N, 1.0 / N, k, 1.0, 1, A)[:8]
    assert ref[-1] < 100.0 * float(np.dot(k, k))
    assert out["status"] == 0
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-9


def test_solve_reciprocal_vector_is_gamma_point(pcmod):
    """k = G = 2 pi A^{-T} (1, 0, 0) on the FCC cell reduces to k = 0: the 3 constant fields are projected out and
    the lowest nonzero eigenvalues of the closed form at k = 0 come back (the default gamma = 2/h)."""
    N = 8
    S = pcmod.Solver(N, np.ones((3, N, N, N)), lattice=FCC)
    G = 2.0 * np.pi * np.linalg.inv(FCC).T @ np.array([1.0, 0.0, 0.0])
    out = S.solve(G[None], 6, 1e-9)
    sig = np.sort(spectrum.homogeneous_physical_spectrum(N, 1.0 / N, np.zeros(3), 1.0, 1, FCC))
    ref = sig[sig > 1e-9][:6]
    assert out["status"] == 0
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-9


def test_solve_sphere_fcc_matches_dense(pcmod):
    """Two dielectric spheres in the FCC primitive cell at N = 8: 6 bands against LAPACK on the oracle's lattice
    operator, with eps from the library's own lattice geometry (gamma = 64: the lowest compensation value
    gamma |k|^2 = 54 lies above the 6th band)."""
    N = 8
    eps = pcmod.eps_spheres_lattice(N, FCC, SPHERES, 1.0)
    S = pcmod.Solver(N, eps, lattice=FCC, gamma_override=64.0)
    k = np.array([0.4, 0.8, -0.2])
    out = S.solve(k[None], 6, 1e-9)
    assert out["status"] == 0
    Op = mfd.compensated_operator(N, k, 1.0 / N, 1.0 / eps, 64.0, 1, FCC)
    ref, _ = eigs.lowest_dense(Op, 6)
    assert ref[-1] < 64.0 * float(np.dot(k, k))
    assert np.max(np.abs(out["evals"][0] - ref) / ref) <= 1e-9


@pytest.mark.parametrize("name,N", [("triclinic", 8), ("fcc", 16), ("bcc", 16)])
def test_apply_op_lattice_double_float(pcmod, name, N):
    """The mixed solve's phase-2 stencil on a general cell: a complex128 block evaluated in double-float arithmetic
    (PC_C128_DF, ~2^-44 relative rounding per operation) against the oracle's lattice operator, 1e-11 relative to
    the largest output."""
    A = LATTICES[name]
    m0 = lattice_m0(N, A)
    S = pcmod.Solver(N, 1.0 / m0, lattice=A)
    g = np.random.default_rng(41 + N)
    kpts = np.vstack([g.uniform(-3.5, 3.5, (2, 3)), np.zeros((1, 3))])
    gammas = np.array([2.0 * N, 9.5, 2.0 * N])
    X = rand_block(N + 13, (3, 2, 3 * N ** 3))
    Y = S.apply_op(kpts, gammas, to_dev(X.reshape(3, 2, 3, N, N, N)), double_float=True).cpu().numpy()
    Y = Y.reshape(3, 2, -1)
    for b in range(3):
        ref = (mfd.compensated_operator(N, kpts[b], 1.0 / N, m0, gammas[b], 1, A) @ X[b].T).T
        assert np.max(np.abs(Y[b] - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["fcc", "triclinic"])
def test_mixed_solve_lattice_matches_fp64(pcmod, name):
    """The mixed-precision solve on a general cell (two k-point groups on their own streams, each with its own
    two-pass stencil scratch) against the FP64 solve of the same cell: eigenvalues within 1e-6 relative, and every
    returned eigenvector's residual, recomputed with the oracle's lattice operator, at most twice the tolerance
    (the oracle's operator takes the penalty of eq. pnt_number; the physical eigenvectors do not depend on it up to
    their divergence, which is of the order of the tolerance). One k-point is a reciprocal-lattice vector (k = 0)."""
    N, nb, tol = 16, 6, 1e-6
    A = LATTICES[name]
    eps = geometry.eps_edges(N, SPHERES, 1.0, A)
    m0 = 1.0 / eps
    G = 2.0 * np.pi * np.linalg.inv(A).T @ np.array([0.0, 1.0, 0.0])
    kpts = np.array([[0.4, 0.8, -0.2], [1.0, -0.3, 0.6], [2.0, 1.0, 0.5], G])
    o64 = pcmod.Solver(N, eps, lattice=A).solve(kpts, nb, tol)
    sm = pcmod.Solver(N, eps, lattice=A, precision=pcmod.pc.PC_PREC_MIXED, groups=2)
    om = sm.solve(kpts, nb, tol, want_vectors=True)
    assert o64["status"] == 0 and om["status"] == 0
    assert np.max(np.abs(om["evals"] - o64["evals"]) / o64["evals"]) <= 1e-6
    assert np.max(om["resid"]) <= tol
    V = om["evecs"].cpu().numpy().reshape(len(kpts), nb, -1)
    for b, k in enumerate(kpts):
        kr = eigs.reduce_by_reciprocal_lattice(k, A)
        Op = mfd.compensated_operator(N, kr, 1.0 / N, m0, mfd.penalty_gamma(1.0 / N, kr), 1, A)
        X = V[b].T
        R = Op @ X - X * om["evals"][b][None, :]
        rel = np.linalg.norm(R, axis=0) / (om["evals"][b] * np.linalg.norm(X, axis=0))
        assert np.max(rel) <= 2.0 * tol, (b, rel)
