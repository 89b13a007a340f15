"""Pins of the oracle's FFT preconditioner (Algorithm 5.1 with the 3x3 symbol) against a sparse direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import mfd, precond


@pytest.mark.parametrize("N,korder,variant", [(6, 1, "gamma"), (8, 1, "gamma"), (8, 2, "gamma"),
                                              (6, 1, "laplacian")])
def test_fft_solve_equals_sparse_solve(N, korder, variant):
    h = 1.0 / N
    k = np.array([0.7, -0.4, 1.9])
    g = mfd.penalty_gamma(h, k)
    gp = 1.0 if variant == "laplacian" else g
    P = mfd.preconditioner_matrix(N, k, h, gp, korder)
    rng = np.random.default_rng(N)
    r = rng.standard_normal(3 * N ** 3) + 1j * rng.standard_normal(3 * N ** 3)
    x_ref = spla.spsolve(P.tocsc(), r)
    x = precond.apply_preconditioner(r, N, h, k, g, korder, variant).ravel()
    assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))


def test_symbol_is_sherman_morrison_invertible():
    """Per mode the 3x3 symbol is sigma I + (gamma-1) conj(d) d^T; its inverse is
    (1/sigma)[I - (gamma-1)/(gamma sigma) conj(d) d^T]."""
    N = 6
    h = 1.0 / N
    k = np.array([0.3, 0.2, 0.1])
    g = 9.0
    P = precond.symbol_matrices(N, h, k, g)
    for idx in [(0, 0, 0), (1, 2, 3), (5, 0, 4)]:
        M = P[idx]
        sigma = np.trace(M).real / (g + 2)  # trace = 3 sigma + (gamma - 1) sigma
        # recover d up to a phase from the rank-1 part
        R1 = (M - sigma * np.eye(3)) / (g - 1)
        inv = (np.eye(3) - (g - 1) / (g * sigma) * R1) / sigma
        assert np.allclose(inv @ M, np.eye(3), atol=1e-12)


def test_gamma_point_mode_zero_is_pseudo_inverse():
    """At k = 0 the constant mode is singular; the solve returns the minimum-norm solution on the complement."""
    N = 6
    h = 1.0 / N
    k = np.zeros(3)
    g = 2.0 / h
    P = mfd.preconditioner_matrix(N, k, h, g).toarray()
    rng = np.random.default_rng(1)
    r = rng.standard_normal(3 * N ** 3) + 1j * rng.standard_normal(3 * N ** 3)
    x = precond.apply_preconditioner(r, N, h, k, g).ravel()
    x_ref = np.linalg.pinv(P, rcond=1e-10, hermitian=True) @ r
    assert np.max(np.abs(x - x_ref)) < 1e-9 * np.max(np.abs(x_ref))
