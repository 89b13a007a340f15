"""The FFT-based preconditioner solve (Section 5.2, Algorithm 5.1), FP64.

Algorithm 5.1 applies the FFT along each dimension, divides by the diagonal symbol, and applies the inverse FFT
along each dimension. For the preconditioner P = A A' + gamma B'B of eq. penalised_marix the three field components
couple, so the "divide" step becomes a solve with the 3x3 symbol matrix of each mode: entries
gamma|d_i|^2 + sum_{j != i} |d_j|^2 on the diagonal and (gamma - 1) conj(d_i) d_j off it (D_i -> d_i, D_i' -> conj d_i,
by the corollary in Section 5.2). With ``variant='laplacian'`` the matrix is the vector Laplacian of Corollary
discrete_vec_lap_mat (gamma = 1), whose symbol is the scalar diagonal d_{1,i} + d_{2,j} + d_{3,k} of Algorithm 5.1.

General lattice (Section 4.2.2, and the corollary discrete_vec_lap_mat, which the paper states for general lattices):
the same 3x3 solve with the symbols d_i of D_hat_i, which mix the three mode indices; the Laplacian variant stays
diagonal (|d|^2 I) but is no longer a sum of per-axis terms.

Reading for k = 0: the symbol matrix of mode 0 vanishes (the constant fields span the kernel); that mode's solution
is set to 0, which is the exact pseudo-inverse on the complement of the kernel.
"""
from __future__ import annotations

import numpy as np

from .spectrum import axis_symbols, lattice_symbols


def symbol_matrices(N: int, h: float, kvec, gamma: float, korder: int = 1, variant: str = "gamma",
                    lattice=None) -> np.ndarray:
    """The 3x3 symbol of P for every mode, shape (N, N, N, 3, 3) on the (z, y, x) mode grid."""
    if lattice is None:
        d1 = axis_symbols(N, h, kvec[0], korder)
        d2 = axis_symbols(N, h, kvec[1], korder)
        d3 = axis_symbols(N, h, kvec[2], korder)
        dz, dy, dx = np.meshgrid(d3, d2, d1, indexing="ij")
        d = np.stack([dx, dy, dz], axis=-1)  # component order (1, 2, 3) = (x, y, z)
    else:
        d = lattice_symbols(N, h, kvec, korder, lattice)
    g = 1.0 if variant == "laplacian" else gamma
    P = np.zeros((N, N, N, 3, 3), dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            if i == j:
                P[..., i, i] = g * np.abs(d[..., i]) ** 2 + sum(np.abs(d[..., l]) ** 2 for l in range(3) if l != i)
            else:
                P[..., i, j] = (g - 1.0) * np.conj(d[..., i]) * d[..., j]
    return P


def apply_preconditioner(R: np.ndarray, N: int, h: float, kvec, gamma: float, korder: int = 1,
                         variant: str = "gamma", lattice=None) -> np.ndarray:
    """W = P^{-1} R for one face field R of shape (3, N, N, N) (Algorithm 5.1 with the 3x3 symbol)."""
    R = np.asarray(R, dtype=np.complex128).reshape(3, N, N, N)
    B = R
    for axis in (3, 2, 1):  # FFT along each dimension
        B = np.fft.fft(B, axis=axis)
    P = symbol_matrices(N, h, kvec, gamma, korder, variant, lattice)
    rhs = np.moveaxis(B, 0, -1)  # (N, N, N, 3)
    sol = np.zeros_like(rhs)
    singular = np.abs(np.linalg.det(P)) == 0.0
    ok = ~singular
    sol[ok] = np.linalg.solve(P[ok], rhs[ok][..., None])[..., 0]
    B = np.moveaxis(sol, -1, 0)
    for axis in (3, 2, 1):  # inverse FFT along each dimension
        B = np.fft.ifft(B, axis=axis)
    return B


def apply_preconditioner_block(R: np.ndarray, N: int, h: float, kvec, gamma: float, korder: int = 1,
                               variant: str = "gamma", lattice=None) -> np.ndarray:
    """Column-wise P^{-1} on a block R of shape (3 N^3, m)."""
    out = np.empty_like(np.asarray(R, dtype=np.complex128))
    for j in range(R.shape[1]):
        out[:, j] = apply_preconditioner(R[:, j], N, h, kvec, gamma, korder, variant, lattice).ravel()
    return out
