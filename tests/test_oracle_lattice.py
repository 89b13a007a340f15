"""Pins of the oracle's general-lattice operators (Section 2's coordinate change x = A y and Section 4.2.2:
K_hat_i = sum_j b_ji K_j, b = A^{-1}) against what mathematics fixes independently of the oracle's own formulas:

* A = I gives back the cube's operators exactly; A = l I is the cube of side l;
* the discrete de Rham identities and the vector-Laplacian corollary, which the paper states for general lattices;
* the closed-form spectrum against a dense LAPACK solve of the sparse operator;
* the continuum limit: the lowest bands of a homogeneous medium converge to |k + G|^2 over the reciprocal lattice
  G = 2 pi A^{-T} n, which a transposed b or a dropped term cannot reach;
* the FFT preconditioner against the sparse operator it inverts at eps = 1;
* the geometry of a primitive cell against the same crystal built on the cubic cell.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as wl
from oracle import geometry, mfd, precond, spectrum

TRICLINIC = np.array([[1.0, 0.3, 0.1], [0.2, 1.1, -0.4], [0.05, 0.25, 0.9]])
FCC = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])   # columns a_1, a_2, a_3 (Section 6)
BCC = 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])
LATTICES = {"triclinic": TRICLINIC, "fcc": FCC, "bcc": BCC}
K_GENERIC = np.array([0.4, -0.9, 1.3])


def sparse_maxabs(M):
    M = sp.csr_matrix(M)
    return 0.0 if M.nnz == 0 else float(np.max(np.abs(M.data)))


def test_identity_lattice_is_the_cube():
    N, h = 5, 1.0 / 5
    for korder in (1, 2):
        D = mfd.D_blocks(N, K_GENERIC, h, korder)
        Dl = mfd.D_blocks(N, K_GENERIC, h, korder, lattice=np.eye(3))
        for a, b in zip(D, Dl):
            assert sparse_maxabs(a - b) == 0.0
    m0 = np.random.default_rng(3).uniform(0.1, 1.0, 3 * N ** 3)
    Op = mfd.compensated_operator(N, K_GENERIC, h, m0, 7.0, 1)
    Opl = mfd.compensated_operator(N, K_GENERIC, h, m0, 7.0, 1, np.eye(3))
    assert sparse_maxabs(Op - Opl) == 0.0


def test_scaled_identity_lattice_is_a_cube_of_side_l():
    """A = l I on the unit y-cube with h = 1/N is the cube [0, l)^3 with spacing l/N (Tables 2-5 use l = 2 pi)."""
    N, l = 6, 2.0 * np.pi
    Op = mfd.compensated_operator(N, K_GENERIC, l / N, np.ones(3 * N ** 3), 5.0, 2)
    Opl = mfd.compensated_operator(N, K_GENERIC, 1.0 / N, np.ones(3 * N ** 3), 5.0, 2, l * np.eye(3))
    assert sparse_maxabs(Op - Opl) <= 1e-14 * sparse_maxabs(Op)


@pytest.mark.parametrize("name", sorted(LATTICES))
@pytest.mark.parametrize("korder", [1, 3])
def test_de_rham_general_lattice(name, korder):
    """curl grad = 0 and div curl = 0 on a general lattice (Section 4.2.2, eq. discrete_de_Rham)."""
    N = 7
    grad, curl, div = mfd.grad_curl_div(N, K_GENERIC, 1.0 / N, korder, LATTICES[name])
    scale = sparse_maxabs(curl) * sparse_maxabs(grad)
    assert sparse_maxabs(curl @ grad) <= 1e-13 * scale
    assert sparse_maxabs(div @ curl) <= 1e-13 * scale


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_vector_laplacian_corollary_general_lattice(name):
    """curl curl' + div' div = diag(L, L, L) with L = div div' (corollary discrete_vec_lap_mat, stated for general
    lattices): the off-diagonal blocks cancel and the three diagonal blocks are equal."""
    N = 4
    n = N ** 3
    _, curl, div = mfd.grad_curl_div(N, K_GENERIC, 1.0 / N, 2, LATTICES[name])
    Lvec = (curl @ curl.conj().T + div.conj().T @ div).tocsr()
    L = (div @ div.conj().T).tocsr()
    ref = sp.block_diag([L, L, L]).tocsr()
    assert sparse_maxabs(Lvec - ref) <= 1e-12 * sparse_maxabs(ref)
    assert sparse_maxabs(Lvec[:n, n:]) <= 1e-12 * sparse_maxabs(ref)


@pytest.mark.parametrize("name", sorted(LATTICES))
@pytest.mark.parametrize("korder", [1, 2])
def test_closed_form_matches_dense_general_lattice(name, korder):
    """The symbols d_i = i (sum_j b_ji e^{i theta_j/2} S_j + k_i e^{i theta_i/2} Z_i) give every eigenvalue of the
    sparse operator at eps = eps0 (LAPACK on the dense matrix)."""
    N = 4
    A = LATTICES[name]
    Op = mfd.compensated_operator(N, K_GENERIC, 1.0 / N, np.full(3 * N ** 3, 1.0 / 2.5), 9.0, korder, A)
    w = sla.eigh(Op.toarray(), eigvals_only=True)
    ref = spectrum.homogeneous_spectrum(N, 1.0 / N, K_GENERIC, 2.5, 9.0, korder, A)
    assert np.max(np.abs(w - ref)) <= 1e-12 * np.max(ref)


def continuum_error(A, N, korder, count=12):
    """Largest relative error of the lowest ``count`` eigenvalues against |k + G|^2."""
    w = spectrum.homogeneous_physical_spectrum(N, 1.0 / N, K_GENERIC, 1.0, korder, A)[:count]
    ex = spectrum.exact_continuum_eigs_lattice(K_GENERIC, A, count)
    return np.max(np.abs(w - ex) / ex)


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_continuum_limit_general_lattice(name):
    """The lowest 12 eigenvalues (6 bands, two polarisations) of the homogeneous medium converge to the free-photon
    bands |k + G|^2, G = 2 pi A^{-T} n, at second order: halving h divides the error by about 4."""
    A = LATTICES[name]
    e32 = continuum_error(A, 32, 1)
    e64 = continuum_error(A, 64, 1)
    assert e64 < 0.01
    assert 3.5 < e32 / e64 < 4.5


def test_non_orthogonal_lattice_is_second_order_at_every_stencil_order():
    """Each K_j is centred half a cell along its own axis, so on a non-orthogonal cell the terms of K_hat_i sit at
    different points and the symbol error is O(h^2) whatever the stencil order: the 4th-order stencils of Table 1 also
    converge at second order on the FCC cell."""
    e32 = continuum_error(FCC, 32, 2)
    e64 = continuum_error(FCC, 64, 2)
    assert 3.5 < e32 / e64 < 4.5


def test_orthorhombic_lattice_keeps_the_stencil_order():
    """On a diagonal A (orthorhombic cell) each K_hat_i is a multiple of K_i alone and the 2k-th order survives: the
    4th-order stencils divide the error by about 16 when h halves."""
    A = np.diag([1.0, 1.3, 0.8])
    e16 = continuum_error(A, 16, 2)
    e32 = continuum_error(A, 32, 2)
    assert 13.0 < e16 / e32 < 17.0


@pytest.mark.parametrize("name", sorted(LATTICES))
@pytest.mark.parametrize("korder", [1, 3])
def test_precond_inverts_operator_general_lattice(name, korder):
    """At eps = 1 the FFT solve with the lattice symbols inverts the sparse operator (Algorithm 5.1 with the 3x3
    symbol); the Laplacian variant inverts curl curl' + div' div."""
    N = 6
    A = LATTICES[name]
    g = np.random.default_rng(40 + korder)
    x = g.standard_normal(3 * N ** 3) + 1j * g.standard_normal(3 * N ** 3)
    Op = mfd.compensated_operator(N, K_GENERIC, 1.0 / N, np.ones(3 * N ** 3), 9.0, korder, A)
    z = precond.apply_preconditioner(Op @ x, N, 1.0 / N, K_GENERIC, 9.0, korder, "gamma", A).ravel()
    assert np.max(np.abs(z - x)) <= 1e-11 * np.max(np.abs(x))
    P1 = mfd.preconditioner_matrix(N, K_GENERIC, 1.0 / N, 1.0, korder, A)
    z = precond.apply_preconditioner(P1 @ x, N, 1.0 / N, K_GENERIC, 1.0, korder, "laplacian", A).ravel()
    assert np.max(np.abs(z - x)) <= 1e-11 * np.max(np.abs(x))


def test_penalised_blocks_general_lattice():
    """The blockwise form of eq. penalised_marix equals A A' + gamma B'B on a general lattice."""
    N = 4
    P = mfd.preconditioner_matrix(N, K_GENERIC, 1.0 / N, 9.0, 2, TRICLINIC)
    Pb = mfd.preconditioner_matrix_blocks(N, K_GENERIC, 1.0 / N, 9.0, 2, TRICLINIC)
    assert sparse_maxabs(P - Pb) <= 1e-13 * sparse_maxabs(P)


def test_compensation_fills_kernel_general_lattice():
    """Proposition 3.1 on an FCC primitive cell holding a dielectric sphere: the spectrum of the compensated operator
    is the nonzero spectrum of A M0 A' together with gamma times the nonzero spectrum of B'B."""
    N = 4
    A = FCC
    spheres = np.array([[0.05, 0.1, 0.0, 0.2, 13.0]])
    m0 = geometry.m0_from_structure(N, spheres, 1.0, A).ravel()
    assert np.any(m0 < 1.0) and np.any(m0 == 1.0)
    gamma = 3.0
    h = 1.0 / N
    w = sla.eigh(mfd.compensated_operator(N, K_GENERIC, h, m0, gamma, 1, A).toarray(), eigvals_only=True)
    wa = sla.eigh(mfd.curl_part(N, K_GENERIC, h, m0, 1, A).toarray(), eigvals_only=True)
    wb = sla.eigh(mfd.compensation_part(N, K_GENERIC, h, 1, A).toarray(), eigvals_only=True)
    tol = 1e-9 * np.max(w)
    union = np.sort(np.concatenate([wa[wa > tol], gamma * wb[wb > tol]]))
    assert union.size == w.size
    assert np.max(np.abs(union - w)) <= 1e-10 * np.max(w)


def test_geometry_identity_lattice_is_the_cube():
    s = wl.fcc_spheres()
    N = 10
    assert np.array_equal(geometry.eps_edges(N, s.as_array(), s.eps_bg),
                          geometry.eps_edges(N, s.as_array(), s.eps_bg, np.eye(3)))


def test_geometry_fcc_primitive_cell_equals_cubic_cell():
    """One sphere per FCC primitive cell is the same crystal as four spheres per cubic cell (Section 6's FCC
    vectors): at random Cartesian points both give the same permittivity, which pins the nearest-image search of a
    non-orthogonal cell against the cube's rounding."""
    r, e = 0.3, 13.0
    cubic = np.array([[0.0, 0.0, 0.0, r, e], [0.0, 0.5, 0.5, r, e], [0.5, 0.0, 0.5, r, e], [0.5, 0.5, 0.0, r, e]])
    prim = np.array([[0.0, 0.0, 0.0, r, e]])
    x = np.random.default_rng(5).uniform(-1.0, 2.0, (4000, 3))
    ec, _ = geometry.eps_at_points(x - np.floor(x), cubic, 1.0)
    y = x @ np.linalg.inv(FCC).T
    ep, _ = geometry.eps_at_points(y, prim, 1.0, FCC)
    assert np.array_equal(ec, ep)
    assert 0.2 < np.mean(ec == e) < 0.6


def test_geometry_fill_fraction_general_lattice():
    """The share of edge DoFs inside a sphere tends to its volume over the cell volume |det A|."""
    spheres = np.array([[0.1, 0.2, 0.15, 0.25, 13.0]])
    eps = geometry.eps_edges(24, spheres, 1.0, BCC)
    frac = 4.0 / 3.0 * np.pi * 0.25 ** 3 / abs(np.linalg.det(BCC))
    assert abs(np.mean(eps == 13.0) - frac) < 0.01


def test_lattice_inverse_rejects_bad_matrices():
    with pytest.raises(ValueError):
        mfd.lattice_inverse(np.ones((3, 3)))
    with pytest.raises(ValueError):
        mfd.lattice_inverse(np.eye(2))
    with pytest.raises(ValueError):
        mfd.lattice_inverse(np.diag([1.0, np.nan, 1.0]))


def test_planted_transposed_b_fails_the_dense_pin(monkeypatch):
    """b_ij in place of b_ji (A^{-T} for A^{-1}) is a plausible slip; on the triclinic cell the closed form, which
    keeps b_ji, no longer matches the sparse operator."""
    orig = mfd.lattice_inverse
    monkeypatch.setattr(mfd, "lattice_inverse", lambda A: orig(A).T)
    N = 4
    Op = mfd.compensated_operator(N, K_GENERIC, 1.0 / N, np.ones(3 * N ** 3), 9.0, 1, TRICLINIC)
    w = sla.eigh(Op.toarray(), eigvals_only=True)
    ref = spectrum.homogeneous_spectrum(N, 1.0 / N, K_GENERIC, 1.0, 9.0, 1, TRICLINIC)
    assert np.max(np.abs(w - ref)) > 1e-3 * np.max(ref)


def test_planted_transposed_lattice_fails_the_continuum_pin():
    """The same slip made consistently in the operator and its closed form (the symbols built from A^T) moves the
    bands of the triclinic cell away from its |k + G|^2 by a relative error that no refinement removes."""
    ex = spectrum.exact_continuum_eigs_lattice(K_GENERIC, TRICLINIC, 12)
    for A, bad in ((TRICLINIC.T, True), (TRICLINIC, False)):
        w = spectrum.homogeneous_physical_spectrum(64, 1.0 / 64, K_GENERIC, 1.0, 1, A)[:12]
        err = np.max(np.abs(w - ex) / ex)
        assert (err > 0.05) if bad else (err < 0.002)


def test_oracle_lobpcg_on_a_lattice_matches_dense():
    """The oracle's Algorithm 4.1 + LOBPCG with the lattice operators and preconditioner reproduces LAPACK on the FCC
    cell holding a sphere (N = 8, gamma = 64 keeps the compensation values above the 6 bands)."""
    from oracle import eigs
    N = 8
    m0 = geometry.m0_from_structure(N, np.array([[0.05, 0.1, 0.0, 0.2, 13.0]]), 1.0, FCC).ravel()
    k = np.array([0.4, 0.8, -0.2])
    out = eigs.solve_kpoint(N, k, m0, 6, 1e-9, guard=4, gamma=64.0, lattice=FCC)
    Op = mfd.compensated_operator(N, k, 1.0 / N, m0, 64.0, 1, FCC)
    ref, _ = eigs.lowest_dense(Op, 6)
    assert out["doublings"] == 0
    assert np.max(np.abs(out["evals"] - ref) / ref) <= 1e-9


def test_reciprocal_lattice_reduction():
    """A reciprocal-lattice vector reduces to exactly 0; a general k moves by one, keeping every eigenvalue of the
    continuum (|k + G|^2 over all G is unchanged); the cube's rule is the special case A = I."""
    from oracle import eigs
    G = 2 * np.pi * np.linalg.inv(FCC).T @ np.array([1.0, -2.0, 1.0])
    assert np.array_equal(eigs.reduce_by_reciprocal_lattice(G, FCC), np.zeros(3))
    k = np.array([7.0, -1.0, 3.5])
    kr = eigs.reduce_by_reciprocal_lattice(k, FCC)
    frac = FCC.T @ (k - kr) / (2 * np.pi)
    assert np.allclose(frac, np.round(frac), atol=1e-12)
    assert np.all(np.abs(FCC.T @ kr / (2 * np.pi)) <= 0.5 + 1e-12)
    assert np.allclose(eigs.reduce_by_reciprocal_lattice(k, np.eye(3)), eigs.reduce_to_first_zone(k))
