"""Complex64 Gram products through the C ABI (pc_gram_pair, pc_gram): for complex64 panels whose length is a
multiple of 16 these run on the tensor cores (TF32 operands, three-term split, FP32 accumulation); other lengths take
the CUDA-core kernel. Both must match the FP64 product of the same FP32 inputs to FP32 accuracy.

Tolerance: every output is a sum of K = 2L real products accumulated in FP32 over chunks and added in FP64, so its
error is bounded by a small multiple of 2^-24 sqrt(K / chunks) sum_l |a_l| |b_l|; the tests use
4e-6 * (|A|^H |B|) elementwise. A missing lo term of the split would leave errors of 2^-12 .. 2^-11 relative, which
the constant-magnitude case below exposes (its values 1 + 2^-12 are not TF32 numbers).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    b.build()
    import paper_2503_19379_gb300 as p
    return p


def rand_c64(seed, shape):
    g = np.random.default_rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check(got, A, B, rel=4e-6):
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    ref = np.einsum("bil,bjl->bij", A64.conj(), B64)
    bound = np.einsum("bil,bjl->bij", np.abs(A64.real) + np.abs(A64.imag), np.abs(B64.real) + np.abs(B64.imag))
    err = np.abs(got - ref)
    assert np.all(err <= rel * bound + 1e-30), float(np.max(err / (bound + 1e-300)))


@pytest.mark.parametrize("nb,p,L", [(2, 48, 98304), (3, 64, 4096), (1, 8, 16), (4, 16, 3 * 32 ** 3), (2, 33, 1600),
                                    (5, 1, 512), (2, 13, 777), (1, 40, 3 * 48 ** 3), (40, 48, 3 * 16 ** 3)])
def test_gram_pair_c64(pcmod, nb, p, L):
    S = rand_c64(p * 7 + L, (nb, p, L))
    AS = (S * np.random.default_rng(L).uniform(0.5, 4.0, L)[None, None, :]).astype(np.complex64)
    G, H = pcmod.gram_pair(dev(S), dev(AS))
    G, H = G.cpu().numpy(), H.cpu().numpy()
    check(G, S, S)
    check(H, S, AS)
    for b in range(nb):
        assert np.array_equal(G[b], G[b].conj().T) and np.array_equal(H[b], H[b].conj().T)


@pytest.mark.parametrize("nb,p,q,L", [(2, 16, 32, 98304), (3, 10, 20, 4096), (1, 64, 64, 2048), (2, 64, 17, 1024),
                                      (2, 5, 3, 800), (1, 12, 24, 999)])
def test_gram_c64(pcmod, nb, p, q, L):
    A = rand_c64(p + q, (nb, p, L))
    B = rand_c64(p * q + 1, (nb, q, L))
    G = pcmod.gram(dev(A), dev(B)).cpu().numpy()
    check(G, A, B)


def test_gram_pair_split_exposes_lo(pcmod):
    """Entries (1 + 2^-12) times a unit phase in {1, i, -1, -i}: TF32 keeps 10 mantissa bits, so hi = 1 and
    lo = 2^-12; without the hi.lo and lo.hi terms every diagonal entry would be low by 2^-11 relative."""
    nb, p, L = 2, 24, 8192
    g = np.random.default_rng(3)
    ph = np.array([1, 1j, -1, -1j], dtype=np.complex64)[g.integers(0, 4, (nb, p, L))]
    S = (np.float32(1.0 + 2.0 ** -12) * ph).astype(np.complex64)
    AS = (S * np.float32(3.0)).astype(np.complex64)
    G, H = pcmod.gram_pair(dev(S), dev(AS))
    G, H = G.cpu().numpy(), H.cpu().numpy()
    x2 = (1.0 + 2.0 ** -12) ** 2
    for b in range(nb):
        assert np.allclose(np.diag(G[b]).real, L * x2, rtol=2e-6, atol=0)
        assert np.allclose(np.diag(H[b]).real, 3 * L * x2, rtol=2e-6, atol=0)
    check(G, S, S, rel=2e-6)
    check(H, S, AS, rel=2e-6)


@pytest.mark.parametrize("nb,p,q,L", [(3, 48, 16, 3 * 32 ** 3), (2, 32, 16, 4096), (2, 40, 9, 3 * 16 ** 3),
                                      (4, 8, 3, 512), (1, 64, 16, 2048), (2, 57, 19, 3 * 32 ** 3),
                                      (1, 64, 40, 2048)])
def test_gram_pair_coupled_c64(pcmod, nb, p, q, L):
    """G = S^H S, H = S^H AS and RQ = R^H S from one pass over [S | AS | R] (the mixed solve's pencil and coupling
    block). (57, 19) is the pencil of 12 bands with 7 guard columns (MMA N = 2 * 64 + 32 = 160, the widest one pass
    takes); the last case (2 p + q beyond 160 MMA columns) takes the separate pair and general products."""
    S = rand_c64(p + 3 * q + L, (nb, p, L))
    AS = (S * np.random.default_rng(L + 1).uniform(0.5, 4.0, L)[None, None, :]).astype(np.complex64)
    R = rand_c64(q + 17, (nb, q, L))
    G, H, RQ = pcmod.gram_pair_coupled(dev(S), dev(AS), dev(R))
    G, H, RQ = G.cpu().numpy(), H.cpu().numpy(), RQ.cpu().numpy()
    check(G, S, S)
    check(H, S, AS)
    check(RQ, R, S)
    for b in range(nb):
        assert np.array_equal(G[b], G[b].conj().T) and np.array_equal(H[b], H[b].conj().T)
