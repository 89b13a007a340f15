"""Planted mistakes in the oracle (on the CPU, by monkeypatching) must make its pins fail.

Each case swaps one oracle function for a plausible wrong version and re-runs the check of a pin; the pin has to
reject it. This shows the pins are sharp enough to catch dropped terms, wrong conjugations and typos.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import geometry, mfd, spectrum


def table2_N10_errors():
    N = 10
    l = 2 * np.pi
    h = l / N
    k = np.array([0.5, 0.0, 0.0])
    Op = mfd.compensated_operator(N, k, h, np.ones(3 * N ** 3), mfd.penalty_gamma(h, k), 1)
    w = sla.eigh(Op.toarray(), eigvals_only=True, subset_by_index=[0, 5])
    return np.abs(w - np.array([0.25] * 4 + [1.25] * 2))


def table2_pin_holds():
    e = table2_N10_errors()
    return np.allclose(e[2:], [8.17e-03, 8.17e-03, 3.25e-02, 3.25e-02], rtol=0.006)


def test_pin_passes_unplanted():
    assert table2_pin_holds()


def test_planted_missing_inverse_h(monkeypatch):
    orig = mfd.D_blocks

    def wrong(N, kvec, h, korder=1):
        return orig(N, kvec, 1.0, korder)  # forgets the 1/h of K_i = D1/h
    monkeypatch.setattr(mfd, "D_blocks", wrong)
    assert not table2_pin_holds()


def test_planted_backward_average(monkeypatch):
    """D0 averaging (f_r + f_{r-1}) / 2 instead of (f_r + f_{r+1}) / 2 puts the shift on the wrong half cell."""
    orig = mfd.generator_D0

    def wrong(N, korder):
        v = orig(N, korder)
        return [v[0]] + v[2:] + [v[1]]
    monkeypatch.setattr(mfd, "generator_D0", wrong)
    assert not table2_pin_holds()


def test_planted_transpose_without_conjugate(monkeypatch):
    """Using A^T instead of A' gives a non-Hermitian operator; the Hermitian pin rejects it."""
    def wrong(N, kvec, h, m0, gamma, korder=1):
        import scipy.sparse as sp
        _, A, B = mfd.grad_curl_div(N, kvec, h, korder)
        return (A @ sp.diags(np.ravel(m0)) @ A.T + gamma * (B.T @ B)).tocsr()
    monkeypatch.setattr(mfd, "compensated_operator", wrong)
    N = 6
    Op = mfd.compensated_operator(N, np.array([0.4, 0.2, -0.3]), 1 / N, np.ones(3 * N ** 3), 12.0)
    assert abs(Op - Op.conj().T).max() > 1e-3


def test_planted_eps_instead_of_inverse(monkeypatch):
    """M0 = eps instead of eps^{-1}: the preconditioned spectrum leaves [1/13, 1]."""
    monkeypatch.setattr(geometry, "m0_from_structure", lambda N, s, e: geometry.eps_edges(N, s, e))
    N = 6
    h = 1.0 / N
    k = np.array([0.41, 0.23, -0.37])
    s = wl.sc_single_sphere()
    m0 = geometry.m0_from_structure(N, s.as_array(), s.eps_bg)
    g = mfd.penalty_gamma(h, k)
    w = sla.eigh(mfd.compensated_operator(N, k, h, m0, g).toarray(),
                 mfd.preconditioner_matrix(N, k, h, g).toarray(), eigvals_only=True)
    assert w.max() > 1 + 1e-6


def test_planted_printed_table1_typo(monkeypatch):
    """With the printed k = 3 coefficient c_1 = 25/64 the 6th-order closed form misses Table 4 by orders of
    magnitude."""
    from fractions import Fraction
    c, d = mfd.TABLE1[3]
    monkeypatch.setitem(mfd.TABLE1, 3, ((Fraction(25, 64),) + c[1:], d))
    N = 10
    h = 2 * np.pi / N
    k = np.array([0.5, 0.0, 0.0])
    lam = spectrum.homogeneous_spectrum(N, h, k, 1.0, mfd.penalty_gamma(h, k), 3)[2]
    assert abs(abs(lam - 0.25) - 1.00e-04) > 1e-3
