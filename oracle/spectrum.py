"""Exact discrete spectrum of the compensated operator for a homogeneous permittivity.

Derivation (from Section 5.2): every circulant is diagonalised by the DFT (eq. diag_of_circ). On the Fourier mode
f_r = exp(i theta r), theta = 2 pi m / N, the generalised circulants act as

    D1^{(k)} f = exp(i theta/2) * 2i * sum_s c_s sin((s - 1/2) theta) * f,
    D0^{(k)} f = exp(i theta/2) * 2  * sum_s d_s cos((s - 1/2) theta) * f,

so D_i has the symbol d_i = i exp(i theta_i / 2) (S_i + k_i Z_i) with S = (2/h) sum c_s sin((s-1/2)theta) and
Z = 2 sum d_s cos((s-1/2)theta), and |d_i|^2 = (S_i + k_i Z_i)^2. Per mode, A A' = |d|^2 I - conj(d) d^T and
B'B = conj(d) d^T. With M0 = I / eps0 the 3x3 block (1/eps0)(|d|^2 I - conj(d) d^T) + gamma conj(d) d^T has the
eigenvalue gamma |d|^2 on conj(d) and |d|^2 / eps0 (twice) on its orthogonal complement. This is the spectrum union
of Proposition 3.1 with lambda^A = sigma / eps0 (multiplicity 2) and lambda^B = sigma (multiplicity 1).

General lattice (Section 4.2.2): D_hat_i = sum_j b_ji K_j + i L_i has the symbol
d_i = i (sum_j b_ji exp(i theta_j / 2) S_j + k_i exp(i theta_i / 2) Z_i), which depends on all three mode indices.
The 3x3 block argument above holds for any complex vector d (the identity [a]x [b]x = b a^T - (a.b) I needs no
reality), so the spectrum keeps the same form with sigma = |d|^2 = sum_i |d_i|^2.
"""
from __future__ import annotations

import numpy as np

from .mfd import stencil_coefficients


def axis_symbol_parts(N: int, h: float, korder: int = 1):
    """S(m), Z(m) for m = 0..N-1 (numpy FFT ordering)."""
    c, d = stencil_coefficients(korder)
    theta = 2.0 * np.pi * np.arange(N) / N
    S = np.zeros(N)
    Z = np.zeros(N)
    for s in range(1, len(c) + 1):
        S += c[s - 1] * np.sin((s - 0.5) * theta)
        Z += d[s - 1] * np.cos((s - 0.5) * theta)
    return (2.0 / h) * S, 2.0 * Z


def axis_symbols(N: int, h: float, k_i: float, korder: int = 1) -> np.ndarray:
    """Complex symbol d_i(m) of D_i along one axis."""
    S, Z = axis_symbol_parts(N, h, korder)
    theta = 2.0 * np.pi * np.arange(N) / N
    return 1j * np.exp(0.5j * theta) * (S + k_i * Z)


def lattice_symbols(N: int, h: float, kvec, korder: int = 1, lattice=None) -> np.ndarray:
    """Symbols d_i(m) of D_hat_i on the (z, y, x) mode grid, shape (N, N, N, 3), components (1, 2, 3) last.
    ``lattice=None`` is A = I, where d_i depends on the i-th mode index only."""
    S, Z = axis_symbol_parts(N, h, korder)
    theta = 2.0 * np.pi * np.arange(N) / N
    ph = np.exp(0.5j * theta)
    b = np.eye(3) if lattice is None else np.linalg.inv(np.asarray(lattice, dtype=np.float64))
    # per-axis factors broadcast onto the (z, y, x) grid: axis j (1 = x, 2 = y, 3 = z) is grid dimension 2 - j
    shape = [(1, 1, N), (1, N, 1), (N, 1, 1)]
    PS = [(ph * S).reshape(shape[j]) for j in range(3)]
    PZ = [(ph * Z).reshape(shape[j]) for j in range(3)]
    d = np.zeros((N, N, N, 3), dtype=np.complex128)
    for i in range(3):
        d[..., i] = 1j * (b[0, i] * PS[0] + b[1, i] * PS[1] + b[2, i] * PS[2] + kvec[i] * PZ[i])
    return d


def sigma_grid(N: int, h: float, kvec, korder: int = 1, lattice=None) -> np.ndarray:
    """sigma(m) = sum_i (S_i + k_i Z_i)^2 on the (z, y, x) mode grid (sum_i |d_i|^2 for a general lattice)."""
    if lattice is not None:
        return np.sum(np.abs(lattice_symbols(N, h, kvec, korder, lattice)) ** 2, axis=-1)
    S, Z = axis_symbol_parts(N, h, korder)
    s1 = (S + kvec[0] * Z) ** 2
    s2 = (S + kvec[1] * Z) ** 2
    s3 = (S + kvec[2] * Z) ** 2
    return s3[:, None, None] + s2[None, :, None] + s1[None, None, :]


def homogeneous_spectrum(N: int, h: float, kvec, eps0: float, gamma: float, korder: int = 1,
                         lattice=None) -> np.ndarray:
    """All 3 N^3 eigenvalues of A M0 A' + gamma B'B with M0 = I/eps0, ascending."""
    sig = sigma_grid(N, h, kvec, korder, lattice).ravel()
    return np.sort(np.concatenate([sig / eps0, sig / eps0, gamma * sig]))


def homogeneous_physical_spectrum(N: int, h: float, kvec, eps0: float, korder: int = 1,
                                  lattice=None) -> np.ndarray:
    """The nonzero spectrum of A M0 A' alone (each sigma/eps0 twice), ascending."""
    sig = sigma_grid(N, h, kvec, korder, lattice).ravel()
    return np.sort(np.concatenate([sig / eps0, sig / eps0]))


def exact_continuum_eigs(kvec, l: float, count: int, nmax: int = 4) -> np.ndarray:
    """Lowest ``count`` values of |k + 2 pi n / l|^2 over n in Z^3, each twice (eq. exact_eig, two polarisations)."""
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    w = np.sum((np.asarray(kvec)[None, :] + 2 * np.pi / l * n) ** 2, axis=1)
    return np.sort(np.repeat(w, 2))[:count]


def exact_continuum_eigs_lattice(kvec, lattice, count: int, nmax: int = 4) -> np.ndarray:
    """Lowest ``count`` values of |k + G|^2 over the reciprocal lattice G = 2 pi A^{-T} n, n in Z^3, each twice: the
    free-space bands of a medium with eps = 1 whose fields are periodic under the columns of A (Section 2)."""
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    G = 2.0 * np.pi * n @ np.linalg.inv(np.asarray(lattice, dtype=np.float64))  # rows: (A^{-T} n)^T
    w = np.sum((np.asarray(kvec, dtype=np.float64)[None, :] + G) ** 2, axis=1)
    return np.sort(np.repeat(w, 2))[:count]
