"""Explicit sparse matrices of the MFD operators (Section 4.2 and 4.3), FP64 / complex128.

Vector layout: a grid function on the N^3 periodic grid is flattened with x fastest, i.e. index (z*N + y)*N + x, so
that K_1 = I (x) I (x) D1/h acts on x (eq. blocks). A vector field is the concatenation of its three components.

General lattices (Section 2's coordinate change x = A y and Section 4.2.2): ``lattice`` is the matrix A whose columns
are the translation vectors a_1, a_2, a_3. The grid lives on the unit cube of y (period e_n, spacing h = 1/N); the
field components stay Cartesian. With b = A^{-1}, K_hat_i = sum_j b_ji K_j replaces K_i and L_i is unchanged, so
D_hat_i = K_hat_i + i L_i. ``lattice=None`` is the cube itself (A = I): the operators of Section 4.2.1 unchanged.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.sparse as sp

# Table 1: coefficients (c_1..c_k), (d_1..d_k) of the 2k-th order symmetric stencils.
# Reading: for k = 3 the table prints c_1 = 25/64; the consistency condition sum_s c_s (2s-1) = 1 (first derivative
# exact on linear functions) only holds with 75/64, which is taken here.
TABLE1 = {
    1: ((Fraction(1),), (Fraction(1, 2),)),
    2: ((Fraction(9, 8), Fraction(-1, 24)), (Fraction(9, 16), Fraction(-1, 16))),
    3: ((Fraction(75, 64), Fraction(-25, 384), Fraction(3, 640)),
        (Fraction(75, 128), Fraction(-25, 256), Fraction(3, 256))),
    4: ((Fraction(1225, 1024), Fraction(-245, 3072), Fraction(49, 5120), Fraction(-5, 7168)),
        (Fraction(1225, 2048), Fraction(-245, 2048), Fraction(49, 2048), Fraction(-5, 2048))),
}


def stencil_coefficients(korder: int):
    """(c, d) as float tuples for the 2*korder-th order scheme (Table 1, eq. 2kfdm)."""
    c, d = TABLE1[korder]
    return tuple(float(x) for x in c), tuple(float(x) for x in d)


def circ(a) -> sp.csr_matrix:
    """Circ(a) of eq. circ_def: row i is a cyclically shifted right by i, i.e. Circ(a)[i, j] = a[(j - i) mod N]."""
    a = list(a)
    N = len(a)
    rows, cols, vals = [], [], []
    for t in range(N):
        if a[t] != 0:
            for i in range(N):
                rows.append(i)
                cols.append((i + t) % N)
                vals.append(a[t])
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64), (rows, cols)), shape=(N, N))


def generator_D1(N: int, korder: int) -> list:
    """v_1^{(k)} = (-c_1, c_1, c_2, ..., c_k, 0, ..., 0, -c_k, ..., -c_2) (Section 4.2.1)."""
    c, _ = stencil_coefficients(korder)
    k = len(c)
    if N < 2 * k:
        raise ValueError("grid too small for the stencil width")
    v = [0.0] * N
    v[0] = -c[0]
    for s in range(1, k + 1):
        v[s] += c[s - 1]
    for s in range(2, k + 1):
        v[N - s + 1] += -c[s - 1]
    return v


def generator_D0(N: int, korder: int) -> list:
    """v_0^{(k)} = (d_1, d_1, d_2, ..., d_k, 0, ..., 0, d_k, ..., d_2) (Section 4.2.1)."""
    _, d = stencil_coefficients(korder)
    k = len(d)
    if N < 2 * k:
        raise ValueError("grid too small for the stencil width")
    v = [0.0] * N
    v[0] = d[0]
    for s in range(1, k + 1):
        v[s] += d[s - 1]
    for s in range(2, k + 1):
        v[N - s + 1] += d[s - 1]
    return v


def lattice_inverse(lattice) -> np.ndarray:
    """b = A^{-1} for the lattice matrix A (columns a_1, a_2, a_3); rejects a singular or non-3x3 matrix."""
    A = np.asarray(lattice, dtype=np.float64)
    if A.shape != (3, 3) or not np.all(np.isfinite(A)) or abs(np.linalg.det(A)) < 1e-300:
        raise ValueError("lattice must be a finite, non-singular 3x3 matrix")
    return np.linalg.inv(A)


def D_blocks(N: int, kvec, h: float, korder: int = 1, lattice=None):
    """[D_1, D_2, D_3] with D_i = K_i + i L_i (eqs. discre, blocks), as sparse N^3 x N^3 complex matrices.
    With ``lattice`` = A, K_i is replaced by K_hat_i = sum_j b_ji K_j, b = A^{-1} (Section 4.2.2)."""
    I = sp.identity(N, format="csr", dtype=np.float64)
    D1 = circ(generator_D1(N, korder)) / h
    D0 = circ(generator_D0(N, korder))
    K = [sp.kron(I, sp.kron(I, D1)), sp.kron(I, sp.kron(D1, I)), sp.kron(D1, sp.kron(I, I))]
    if lattice is not None:
        b = lattice_inverse(lattice)
        K = [(b[0, i] * K[0] + b[1, i] * K[1] + b[2, i] * K[2]).tocsr() for i in range(3)]
    L = [sp.kron(I, sp.kron(I, kvec[0] * D0)), sp.kron(I, sp.kron(kvec[1] * D0, I)),
         sp.kron(kvec[2] * D0, sp.kron(I, I))]
    return [(K[i] + 1j * L[i]).tocsr() for i in range(3)]


def grad_curl_div(N: int, kvec, h: float, korder: int = 1, lattice=None):
    """GRAD_k (N->E), CURL_k (E->F), DIV_k (F->C) block matrices of eq. discrete_2nd_block (eq. unified_mat for a
    general lattice)."""
    D1, D2, D3 = D_blocks(N, kvec, h, korder) if lattice is None else D_blocks(N, kvec, h, korder, lattice=lattice)
    grad = sp.vstack([D1, D2, D3]).tocsr()
    curl = sp.bmat([[None, -D3, D2], [D3, None, -D1], [-D2, D1, None]]).tocsr()
    div = sp.hstack([D1, D2, D3]).tocsr()
    return grad, curl, div


def penalty_gamma(h: float, kvec) -> float:
    """gamma = 2 max{1/h, |k|^{-2}} (eq. pnt_number). Reading: at k = 0 the |k|^{-2} term is dropped (gamma = 2/h),
    since the Remark after Algorithm 4.1 states gamma = O(1) suffices there."""
    k2 = float(np.dot(kvec, kvec))
    if k2 == 0.0:
        return 2.0 / h
    return 2.0 * max(1.0 / h, 1.0 / k2)


def compensated_operator(N: int, kvec, h: float, m0: np.ndarray, gamma: float, korder: int = 1, lattice=None):
    """Op = A M0 A' + gamma B'B with A = CURL_k, B = DIV_k and M0 = diag(m0) on edges (eq. Ker_comp)."""
    _, A, B = grad_curl_div(N, kvec, h, korder, lattice)
    M0 = sp.diags(np.asarray(m0, dtype=np.float64).ravel())
    Ah = A.conj().T
    Bh = B.conj().T
    return (A @ M0 @ Ah + gamma * (Bh @ B)).tocsr()


def curl_part(N: int, kvec, h: float, m0: np.ndarray, korder: int = 1, lattice=None):
    """A M0 A' alone (the uncompensated operator of eq. first_view_mfdm)."""
    _, A, _ = grad_curl_div(N, kvec, h, korder, lattice)
    M0 = sp.diags(np.asarray(m0, dtype=np.float64).ravel())
    return (A @ M0 @ A.conj().T).tocsr()


def compensation_part(N: int, kvec, h: float, korder: int = 1, lattice=None):
    """B'B alone."""
    _, _, B = grad_curl_div(N, kvec, h, korder, lattice)
    return (B.conj().T @ B).tocsr()


def half_operators(N: int, kvec, h: float, korder: int = 1, lattice=None):
    """(A', B): faces -> edges and faces -> cells, used by the recompute step of Algorithm 4.1."""
    _, A, B = grad_curl_div(N, kvec, h, korder, lattice)
    return A.conj().T.tocsr(), B.tocsr()


def preconditioner_matrix(N: int, kvec, h: float, gamma: float, korder: int = 1, lattice=None):
    """P = A A' + gamma B'B (Section 5.1), the operator with M0 = I."""
    _, A, B = grad_curl_div(N, kvec, h, korder, lattice)
    return (A @ A.conj().T + gamma * (B.conj().T @ B)).tocsr()


def preconditioner_matrix_blocks(N: int, kvec, h: float, gamma: float, korder: int = 1, lattice=None):
    """P written blockwise as in eq. penalised_marix: diagonal gamma D_i D_i' + sum_{j != i} D_j D_j',
    off-diagonal (gamma - 1) D_i' D_j."""
    D = D_blocks(N, kvec, h, korder, lattice)
    Dh = [Di.conj().T for Di in D]
    blocks = [[None] * 3 for _ in range(3)]
    for i in range(3):
        diag = gamma * (D[i] @ Dh[i])
        for j in range(3):
            if j != i:
                diag = diag + D[j] @ Dh[j]
        blocks[i][i] = diag
        for j in range(3):
            if j != i:
                blocks[i][j] = (gamma - 1.0) * (Dh[i] @ D[j])
    return sp.bmat(blocks).tocsr()
