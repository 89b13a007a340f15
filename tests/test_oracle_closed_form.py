"""Pins of the oracle's operator build and closed-form spectrum against the paper's printed numbers and exact
mathematics (Tables 1-5, eq. exact_eig)."""
import os

import numpy as np
import pytest

from oracle import eigs, mfd, spectrum

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tables_2_5_isotropic.txt")
# The paper's own eigensolver leaves absolute errors up to 2.7e-14 on modes the scheme resolves exactly
# (rows 1-2 of Tables 2-5); printed values below that level carry that noise.
PAPER_SOLVER_FLOOR = 5e-14


def golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        o, N, r, ex, pe = line.split()
        rows.append((int(o), int(N), int(r), float(ex), float(pe)))
    return rows


def table_setup(N):
    l = 2 * np.pi
    h = l / N
    k = np.array([np.pi / l, 0.0, 0.0])
    return h, k


def test_golden_fixture_complete():
    rows = golden_rows()
    assert len(rows) == 4 * 4 * 6
    assert {r[0] for r in rows} == {2, 4, 6, 8}
    assert {r[1] for r in rows} == {10, 20, 40, 80}


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_tables_2_to_5_closed_form(order):
    """Every printed error of Tables 2-5 is reproduced by the exact discrete spectrum."""
    for o, N, r, exact, printed in golden_rows():
        if o != order:
            continue
        h, k = table_setup(N)
        lam = spectrum.homogeneous_spectrum(N, h, k, 1.0, mfd.penalty_gamma(h, k), order // 2)[r - 1]
        err = abs(lam - exact)
        if r <= 2:
            # modes the scheme resolves exactly: error zero up to rounding, printed values are solver noise
            assert err < 1e-13 and printed < PAPER_SOLVER_FLOOR
        else:
            assert abs(err - printed) <= max(0.006 * printed, PAPER_SOLVER_FLOOR), (o, N, r, err, printed)


def test_exact_values_are_eq_exact_eig():
    """The 'exact' column equals |k + 2 pi n / l|^2 (eq. exact_eig) for the lowest modes."""
    h, k = table_setup(10)
    ex = spectrum.exact_continuum_eigs(k, 2 * np.pi, 6)
    assert np.allclose(ex, [0.25, 0.25, 0.25, 0.25, 1.25, 1.25])


@pytest.mark.parametrize("korder", [1, 2])
def test_table2_4_by_dense_kronecker_build(korder):
    """The explicitly built Kronecker operator, solved by LAPACK, reproduces Table 2 (order 2) and Table 3
    (order 4) at N = 10: pins the operator build independently of the closed form."""
    N = 10
    h, k = table_setup(N)
    Op = mfd.compensated_operator(N, k, h, np.ones(3 * N ** 3), mfd.penalty_gamma(h, k), korder)
    w, _ = eigs.lowest_dense(Op, 6)
    errs = np.abs(w - np.array([0.25] * 4 + [1.25] * 2))
    printed = {1: [8.17e-03, 8.17e-03, 3.25e-02, 3.25e-02], 2: [1.05e-03, 1.05e-03, 1.43e-03, 1.43e-03]}[korder]
    assert np.all(errs[:2] < 1e-12)
    assert np.allclose(errs[2:], printed, rtol=0.006)


def test_table2_N20_by_oracle_lobpcg():
    """Table 2 at N = 20 through the oracle's LOBPCG on the Kronecker-built operator (eps = 1)."""
    N = 20
    h, k = table_setup(N)
    g = mfd.penalty_gamma(h, k)
    Op = mfd.compensated_operator(N, k, h, np.ones(3 * N ** 3), g, 1)
    from oracle.precond import apply_preconditioner_block
    from oracle.rng import initial_block
    # rows 5-6 sit in an 8-fold degenerate cluster that a small block converges to only slowly; rows 1-4 are
    # checked here, rows 5-6 by the dense N = 10 build and the closed form
    theta, X, it, res = eigs.lobpcg(lambda Y: Op @ Y, lambda Y: apply_preconditioner_block(Y, N, h, k, g),
                                    initial_block(3, 0, 3 * N ** 3, 6), 4, 1e-11)
    errs = np.abs(theta[:4] - np.array([0.25] * 4))
    assert np.allclose(errs[2:], [2.05e-03, 2.05e-03], rtol=0.006)
    assert np.all(errs[:2] < 1e-12)


@pytest.mark.parametrize("N,korder,eps0", [(4, 1, 1.0), (6, 1, 2.5), (5, 1, 13.0), (8, 2, 3.0), (8, 3, 1.0),
                                           (8, 4, 0.5)])
def test_closed_form_equals_dense_full_spectrum(N, korder, eps0):
    """All 3N^3 eigenvalues of the Kronecker-built operator equal the Fourier-symbol closed form."""
    h = 1.0 / N
    k = np.array([0.37, -1.21, 0.83])
    g = mfd.penalty_gamma(h, k)
    Op = mfd.compensated_operator(N, k, h, np.full(3 * N ** 3, 1.0 / eps0), g, korder)
    w = np.linalg.eigvalsh(Op.toarray())
    cf = spectrum.homogeneous_spectrum(N, h, k, eps0, g, korder)
    assert np.max(np.abs(w - cf)) <= 1e-12 * np.max(cf)


@pytest.mark.parametrize("korder", [1, 2, 3, 4])
def test_table1_moment_conditions(korder):
    """Table 1's stencils are the 2k-th order staggered ones: sum c_s (2s-1) = 1, sum c_s (2s-1)^(2p+1) = 0 and
    2 sum d_s = 1, sum d_s (2s-1)^(2p) = 0 for p = 1..k-1 (Taylor expansion about the half point)."""
    c, d = mfd.TABLE1[korder]
    k = len(c)
    assert sum(cs * (2 * s - 1) for s, cs in enumerate(c, 1)) == 1
    assert 2 * sum(d) == 1
    for p in range(1, k):
        assert sum(cs * (2 * s - 1) ** (2 * p + 1) for s, cs in enumerate(c, 1)) == 0
        assert sum(ds * (2 * s - 1) ** (2 * p) for s, ds in enumerate(d, 1)) == 0


def test_table1_printed_c1_for_k3_fails_consistency():
    """The printed k = 3 value c_1 = 25/64 violates the first-derivative condition; 75/64 satisfies it."""
    from fractions import Fraction
    c = mfd.TABLE1[3][0]
    assert c[0] == Fraction(75, 64)
    printed = (Fraction(25, 64),) + c[1:]
    assert sum(cs * (2 * s - 1) for s, cs in enumerate(printed, 1)) != 1


def test_circulant_convention():
    """Circ(a) rows are right shifts (eq. circ_def) and D1 = Circ(-1, 1, 0, ...) is the forward difference."""
    D1 = mfd.circ(mfd.generator_D1(5, 1)).toarray()
    f = np.arange(5.0) ** 2
    assert np.allclose(D1 @ f, np.roll(f, -1) - f)
    D0 = mfd.circ(mfd.generator_D0(5, 1)).toarray()
    assert np.allclose(D0 @ f, 0.5 * (np.roll(f, -1) + f))
