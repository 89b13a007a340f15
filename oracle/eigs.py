"""Reference eigenpairs of the compensated operator, FP64.

* ``lowest_dense`` / ``lowest_sparse``: the plain definition -- the smallest eigenvalues of the explicitly built
  Hermitian matrix Op = A M0 A' + gamma B'B (eq. Ker_comp), by LAPACK (dense) or ARPACK shift-invert (sparse).
* ``lobpcg``: an independent block LOBPCG (the eigensolver of Section 5.1; the paper cites Knyazev and gives no
  internals). Steps per iteration: residuals R = AX - X Theta, preconditioned directions W = T R, Rayleigh-Ritz on
  span[X, W, P] through an orthonormal basis, X <- Ritz vectors, P <- the [W, P] part of the Ritz update.
* ``recompute_check``: Algorithm 4.1's lambda_re = |M0^{1/2} A' x|^2 / |x|^2 and its comparison with lambda.
* ``solve_kpoint``: Algorithm 4.1 end to end (solve, recompute, double gamma while spurious values remain).

Readings (where the paper is silent):
* Convergence: column j is converged when |A x_j - theta_j x_j| <= tol * |theta_j| * |x_j|.
* Algorithm 4.1's equality test: |lambda - lambda_re| <= 10 * tol * lambda; at most ``max_doublings`` doublings.
  Its "goto line 1" re-solve starts from the current block with the spurious columns replaced by fresh random ones.
* k = 0 (Remark after eq. penalised_marix): instead of a shift, the 3 constant fields spanning the kernel are
  projected out of every block (exact, since the kernel is an invariant subspace), and the lowest nonzero
  eigenvalues are reported.
* Bloch vectors are first reduced into the first Brillouin zone of the cubic cell, k - 2 pi round(k / 2 pi)
  (Section 2 takes k in the first Brillouin zone); a vector equivalent to 0 becomes exactly 0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import mfd
from .precond import apply_preconditioner_block


def reduce_to_first_zone(kvec, a: float = 1.0) -> np.ndarray:
    k = np.asarray(kvec, dtype=np.float64)
    g = 2.0 * np.pi / a
    return k - g * np.round(k / g)


def reduce_by_reciprocal_lattice(kvec, lattice) -> np.ndarray:
    """k - 2 pi A^{-T} n with n = round(A^T k / 2 pi): the Bloch vector moved by the nearest reciprocal-lattice vector
    of the cell A in fractional coordinates (the cube's reduction for A = a I); a k whose fractional coordinates are
    all within 1e-12 of integers is equivalent to 0 and becomes exactly 0 (Section 2: k is taken in one zone)."""
    k = np.asarray(kvec, dtype=np.float64)
    A = np.asarray(lattice, dtype=np.float64)
    f = A.T @ k / (2.0 * np.pi)
    n = np.round(f)
    if np.all(np.abs(f - n) <= 1e-12):
        return np.zeros(3)
    return k - 2.0 * np.pi * np.linalg.solve(A.T, n)


def _herm(M):
    return 0.5 * (M + M.conj().T)


def lowest_dense(Op, m: int, skip: int = 0):
    """The m smallest eigenvalues (after skipping ``skip``) and eigenvectors of Op by LAPACK eigh."""
    A = Op.toarray() if hasattr(Op, "toarray") else np.asarray(Op)
    w, V = sla.eigh(_herm(A), subset_by_index=[0, skip + m - 1])
    return w[skip:], V[:, skip:]


def lowest_sparse(Op, m: int, skip: int = 0, tol: float = 1e-14):
    """The m smallest eigenvalues (after skipping ``skip``) of Hermitian PSD Op by ARPACK shift-invert about -1."""
    w, V = spla.eigsh(Op.tocsc(), k=m + skip, sigma=-1.0, which="LM", tol=tol)
    order = np.argsort(w)
    return w[order][skip:], V[:, order][:, skip:]


def constant_projector(N: int):
    """Projector removing the per-component mean (the k = 0 kernel) from each column of a face block."""
    n = N ** 3

    def project(Y):
        Y = np.array(Y, dtype=np.complex128, copy=True)
        for c in range(3):
            Y[c * n:(c + 1) * n] -= Y[c * n:(c + 1) * n].mean(axis=0, keepdims=True)
        return Y

    return project


def orthonormal_transform(S: np.ndarray, drop: float = 1e-12) -> np.ndarray:
    """C such that S C has orthonormal columns spanning span(S) up to numerically dependent directions.

    Columns are scaled to unit norm, the Gram matrix is diagonalised and directions with eigenvalue below
    ``drop`` times the largest are discarded; a second pass restores orthonormality to rounding level.
    """
    nrm = np.linalg.norm(S, axis=0)
    nrm[nrm == 0] = 1.0
    C = np.diag(1.0 / nrm)
    Q = S @ C
    w, V = np.linalg.eigh(_herm(Q.conj().T @ Q))
    keep = w > drop * w.max()
    C = C @ (V[:, keep] / np.sqrt(w[keep]))
    Q = S @ C
    w2, V2 = np.linalg.eigh(_herm(Q.conj().T @ Q))
    return C @ (V2 / np.sqrt(w2))


def lobpcg(apply_A, apply_T, X0: np.ndarray, nconv: int, tol: float, maxiter: int = 500, project=None):
    """Block LOBPCG for the smallest eigenpairs; returns (theta, X, iterations, relative residuals).

    ``apply_A``/``apply_T`` map an (n, p) block to an (n, p) block. AX and AP are recomputed with apply_A every
    iteration (no drift).
    """
    X = np.array(X0, dtype=np.complex128, copy=True)
    m = X.shape[1]
    if project is not None:
        X = project(X)
    X = X @ orthonormal_transform(X)
    AX = apply_A(X)
    theta, U = np.linalg.eigh(_herm(X.conj().T @ AX))
    X = X @ U
    AX = apply_A(X)
    P = None
    res = None
    for it in range(maxiter + 1):
        R = AX - X * theta[None, :]
        res = np.linalg.norm(R, axis=0) / (np.abs(theta) * np.linalg.norm(X, axis=0))
        if np.all(res[:nconv] <= tol) or it == maxiter:
            return theta, X, it, res
        W = apply_T(R)
        if project is not None:
            W = project(W)
        S = np.hstack([X, W] if P is None else [X, W, P])
        C = orthonormal_transform(S)
        Q = S @ C
        AQ = apply_A(Q)
        thall, U = np.linalg.eigh(_herm(Q.conj().T @ AQ))
        coef = C @ U[:, :m]
        theta = thall[:m]
        Xn = S @ coef
        P = S[:, m:] @ coef[m:]
        X = Xn
        if project is not None:
            X = project(X)
            P = project(P)
        AX = apply_A(X)
    return theta, X, maxiter, res


def recompute_check(X: np.ndarray, theta: np.ndarray, m0: np.ndarray, Ah, tol: float):
    """Algorithm 4.1: lambda_re = |M0^{1/2} A' x|^2 / |x|^2; flags columns whose value differs from lambda."""
    E = Ah @ X
    lam_re = np.sum(np.asarray(m0).ravel()[:, None] * np.abs(E) ** 2, axis=0) / np.sum(np.abs(X) ** 2, axis=0)
    spurious = np.abs(lam_re - theta) > 10.0 * tol * np.abs(theta)
    return lam_re, spurious


def spurious_columns(lam_re: np.ndarray, theta: np.ndarray, nbands: int, tol: float) -> np.ndarray:
    """Columns to discard before the re-solve of Algorithm 4.1: the first nbands by the equality test, the guard
    columns (not converged to tol) when lambda_re < lambda / 2, i.e. when the compensation part dominates."""
    strict = np.abs(lam_re - theta) > 10.0 * tol * np.abs(theta)
    loose = lam_re < 0.5 * theta
    return np.where(np.arange(theta.size) < nbands, strict, loose)


def solve_kpoint(N: int, kvec, m0: np.ndarray, nbands: int, tol: float, guard: int = 2, korder: int = 1,
                 gamma: float | None = None, variant: str = "gamma", X0: np.ndarray | None = None,
                 maxiter: int = 500, max_doublings: int = 8, seed: int = 0, lattice=None):
    """Algorithm 4.1 with the LOBPCG above and the FFT preconditioner of Algorithm 5.1 (on the cell ``lattice`` when
    given: Section 4.2.2's operators and symbols, k reduced by its reciprocal lattice).

    Returns a dict with eigenvalues (nbands), eigenvectors, iterations, residuals, the final gamma and the number
    of gamma doublings.
    """
    from .rng import initial_block

    h = 1.0 / N
    k = reduce_to_first_zone(kvec) if lattice is None else reduce_by_reciprocal_lattice(kvec, lattice)
    g = mfd.penalty_gamma(h, k) if gamma is None else float(gamma)
    m = nbands + guard
    project = constant_projector(N) if not np.any(k) else None
    if X0 is None:
        X0 = initial_block(seed, 0, 3 * N ** 3, m)
    lat = {} if lattice is None else {"lattice": lattice}
    Ah, _ = mfd.half_operators(N, k, h, korder, **lat)
    total_it = 0
    for doubling in range(max_doublings + 1):
        Op = mfd.compensated_operator(N, k, h, m0, g, korder, **lat)
        theta, X, it, res = lobpcg(lambda Y: Op @ Y,
                                   lambda Y: apply_preconditioner_block(Y, N, h, k, g, korder, variant, **lat),
                                   X0, nbands, tol, maxiter, project)
        total_it += it
        lam_re, spurious = recompute_check(X[:, :nbands], theta[:nbands], m0, Ah, tol)
        if not np.any(spurious):
            break
        if doubling == max_doublings:
            break
        g *= 2.0
        # "goto line 1" (Algorithm 4.1), warm-started: the physical eigenvectors are kept; the spurious ones are
        # gamma-independent exact eigenvectors of B'B that LOBPCG would never leave, so they are replaced by fresh
        # random columns (stream shifted by the doubling count)
        lam_all, _ = recompute_check(X, theta, m0, Ah, tol)
        bad = spurious_columns(lam_all, theta, nbands, tol)
        X0 = X.copy()
        fresh = initial_block(seed + 7919 * (doubling + 1), 0, X.shape[0], m)
        X0[:, bad] = fresh[:, bad]
    return {"evals": theta[:nbands], "evecs": X[:, :nbands], "iters": total_it, "resid": res[:nbands],
            "gamma": g, "doublings": doubling, "spurious": spurious, "lam_re": lam_re}
