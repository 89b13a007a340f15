"""Pins of the oracle's operators against the structural facts the paper proves (Sections 3-5)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import geometry, mfd, spectrum

K_GENERIC = np.array([0.41, 0.23, -0.37])


def sphere_m0(N):
    s = wl.sc_single_sphere()
    return geometry.m0_from_structure(N, s.as_array(), s.eps_bg)


@pytest.mark.parametrize("korder", [1, 2])
def test_discrete_de_rham(korder):
    """CURL_k GRAD_k = 0 and DIV_k CURL_k = 0 (eq. discrete_de_Rham), i.e. assumption B A = 0 (eq. assumpt1)."""
    N = 8
    grad, curl, div = mfd.grad_curl_div(N, K_GENERIC, 1.0 / N, korder)
    assert abs(curl @ grad).max() < 1e-12 * N ** 2
    assert abs(div @ curl).max() < 1e-12 * N ** 2


def test_operator_hermitian():
    N = 6
    h = 1.0 / N
    Op = mfd.compensated_operator(N, K_GENERIC, h, sphere_m0(N), mfd.penalty_gamma(h, K_GENERIC))
    assert abs(Op - Op.conj().T).max() <= 1e-14 * abs(Op).max()


def test_adjoint_is_backward_difference():
    """D_i' is the conjugate transpose: (D' g)_r = (g_{r-1} - g_r)/h - i k_i (g_{r-1} + g_r)/2 along axis i."""
    N = 5
    h = 1.0 / N
    D1, _, _ = mfd.D_blocks(N, K_GENERIC, h)
    g = np.random.default_rng(0).standard_normal(N ** 3) + 1j
    G = g.reshape(N, N, N)
    Gm = np.roll(G, 1, axis=2)
    expect = (Gm - G) / h - 1j * K_GENERIC[0] * (Gm + G) / 2
    assert np.allclose((D1.conj().T @ g).reshape(N, N, N), expect)


def test_proposition_3_1_spectrum_union():
    """Spectrum of A M0 A' + gamma B'B = nonzero spec(A M0 A') U gamma * nonzero spec(B'B) (Proposition 3.1);
    dim ker A M0 A' = N^3 at k != 0, exactly N^3 compensation eigenvalues, and no zero eigenvalue."""
    N = 6
    h = 1.0 / N
    m0 = sphere_m0(N)
    g = mfd.penalty_gamma(h, K_GENERIC)
    w = np.linalg.eigvalsh(mfd.compensated_operator(N, K_GENERIC, h, m0, g).toarray())
    wa = np.linalg.eigvalsh(mfd.curl_part(N, K_GENERIC, h, m0).toarray())
    wb = np.linalg.eigvalsh(mfd.compensation_part(N, K_GENERIC, h).toarray())
    za = wa < 1e-10 * wa.max()
    zb = wb < 1e-10 * wb.max()
    assert za.sum() == N ** 3
    assert (~zb).sum() == N ** 3
    assert w.min() > 1e-3
    union = np.sort(np.concatenate([wa[~za], g * wb[~zb]]))
    assert np.max(np.abs(union - w)) < 1e-12 * w.max()
    # the compensation eigenvalues are gamma * sigma(m), independent of eps
    assert np.allclose(np.sort(wb[~zb]), np.sort(spectrum.sigma_grid(N, h, K_GENERIC).ravel()), rtol=1e-10,
                       atol=1e-10 * wb.max())


def test_kernel_at_gamma_point_is_three_dimensional():
    """At k = 0 the compensated operator has exactly 3 zero eigenvalues, the constant fields (Remark in Sec. 4.5)."""
    N = 6
    h = 1.0 / N
    k0 = np.zeros(3)
    Op = mfd.compensated_operator(N, k0, h, sphere_m0(N), mfd.penalty_gamma(h, k0))
    w = np.linalg.eigvalsh(Op.toarray())
    assert np.sum(w < 1e-9 * w.max()) == 3
    const = np.zeros((3 * N ** 3, 3))
    for c in range(3):
        const[c * N ** 3:(c + 1) * N ** 3, c] = 1.0
    assert abs(Op @ const).max() < 1e-10


def test_physical_eigenvalues_do_not_depend_on_gamma():
    """Remark pnt_criterion: once gamma lambda_1^B > lambda_m^A the lowest m eigenvalues are those of A M0 A'."""
    N = 6
    h = 1.0 / N
    m0 = sphere_m0(N)
    wa = np.linalg.eigvalsh(mfd.curl_part(N, K_GENERIC, h, m0).toarray())
    phys = np.sort(wa[wa > 1e-10 * wa.max()])[:8]
    for g in (64.0, 128.0, 1000.0):
        w = np.linalg.eigvalsh(mfd.compensated_operator(N, K_GENERIC, h, m0, g).toarray())[:8]
        assert np.allclose(w, phys, rtol=1e-11)


def test_preconditioner_blockwise_equals_product_form():
    """The blockwise matrix of eq. penalised_marix equals A A' + gamma B'B (Proposition commutativity_of_K_prime)."""
    N = 6
    h = 1.0 / N
    for korder in (1, 2):
        if N < 2 * korder:
            continue
        P = mfd.preconditioner_matrix(N, K_GENERIC, h, 7.5, korder)
        Pb = mfd.preconditioner_matrix_blocks(N, K_GENERIC, h, 7.5, korder)
        assert abs(P - Pb).max() < 1e-10 * abs(P).max()


def test_preconditioner_is_operator_at_unit_permittivity():
    N = 6
    h = 1.0 / N
    g = mfd.penalty_gamma(h, K_GENERIC)
    Op = mfd.compensated_operator(N, K_GENERIC, h, np.ones(3 * N ** 3), g)
    assert abs(Op - mfd.preconditioner_matrix(N, K_GENERIC, h, g)).max() <= 1e-14 * abs(Op).max()


def test_rayleigh_quotient_bound_of_preconditioned_operator():
    """Eigenvalues of P^{-1} Op lie in [min M0, max M0] = [1/13, 1] (Section 5.1's Rayleigh-quotient bound),
    and both ends are attained for the sphere structure."""
    N = 6
    h = 1.0 / N
    m0 = sphere_m0(N)
    g = mfd.penalty_gamma(h, K_GENERIC)
    Op = mfd.compensated_operator(N, K_GENERIC, h, m0, g).toarray()
    P = mfd.preconditioner_matrix(N, K_GENERIC, h, g).toarray()
    w = sla.eigh(Op, P, eigvals_only=True)
    assert w.min() >= 1 / 13 - 1e-9 and w.max() <= 1 + 1e-9
    assert abs(w.min() - 1 / 13) < 1e-6 and abs(w.max() - 1) < 1e-6


def test_vector_laplacian_corollary():
    """CURL CURL' + DIV' DIV = diag(L, L, L) with L = DIV DIV' (Corollary discrete_vec_lap_mat)."""
    N = 5
    h = 1.0 / N
    _, curl, div = mfd.grad_curl_div(N, K_GENERIC, h)
    V = (curl @ curl.conj().T + div.conj().T @ div).toarray()
    L = (div @ div.conj().T).toarray()
    n = N ** 3
    for i in range(3):
        for j in range(3):
            blk = V[i * n:(i + 1) * n, j * n:(j + 1) * n]
            assert np.allclose(blk, L if i == j else 0.0, atol=1e-10)
