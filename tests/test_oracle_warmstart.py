"""Pins of the warm-start network's FP64 reference (oracle/warmstart.py): every hand-written backward pass against
central finite differences of its forward pass, the layers against special cases with known answers, the subspace
loss against its invariances, Adam against its closed-form first step, and a short training run that lowers the
loss on eigenvectors of the method itself."""
import numpy as np
import pytest

import workloads as wl
from oracle import eigs, geometry, mfd, warmstart as ws

NB, C1, C2, N = 2, 4, 6, 8


def small_params(seed=1):
    p = ws.init_params(C1, C2, NB, seed)
    g = np.random.default_rng(seed + 100)
    # move FiLM and the biases off their special initial values so that every path carries gradient
    for k in ("Fa", "fa", "Fc", "fc", "b1", "b2", "bh", "bv"):
        p[k] = 0.3 * g.standard_normal(p[k].shape)
    return p


def random_sample(seed=2):
    g = np.random.default_rng(seed)
    m0 = g.uniform(0.1, 1.0, (3, N, N, N))
    k = g.uniform(-3, 3, 3)
    V, _ = np.linalg.qr(g.standard_normal((3 * N ** 3, NB)) + 1j * g.standard_normal((3 * N ** 3, NB)))
    lam = g.uniform(1.0, 30.0, NB)
    return m0, k, V, lam


def fd_check(p, sample, key, count=6, h=1e-6, seed=0):
    """Central differences of the total loss in `count` random entries of parameter `key` vs backward()."""
    m0, k, V, lam = sample
    _, cache = ws.loss(p, m0, k, V, lam, NB)
    g = ws.backward(p, cache)[key]
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(count):
        idx = tuple(rng.integers(0, s) for s in p[key].shape)
        old = p[key][idx]
        p[key][idx] = old + h
        lp, _ = ws.loss(p, m0, k, V, lam, NB)
        p[key][idx] = old - h
        lm, _ = ws.loss(p, m0, k, V, lam, NB)
        p[key][idx] = old
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - g[idx]) / max(1e-6, abs(fd) + abs(g[idx])))
    return worst


@pytest.mark.parametrize("key", ws.PARAM_ORDER)
def test_backward_matches_finite_differences(key):
    p = small_params()
    assert fd_check(p, random_sample(), key) < 1e-6


def test_subspace_loss_gradient_matches_finite_differences():
    g = np.random.default_rng(4)
    X = g.standard_normal((60, 3)) + 1j * g.standard_normal((60, 3))
    V, _ = np.linalg.qr(g.standard_normal((60, 3)) + 1j * g.standard_normal((60, 3)))
    _, dX = ws.subspace_loss(X, V)
    h = 1e-6
    for (i, j) in [(0, 0), (17, 2), (59, 1)]:
        for unit, part in ((1.0, "re"), (1j, "im")):
            Xp = X.copy()
            Xp[i, j] += h * unit
            Xm = X.copy()
            Xm[i, j] -= h * unit
            fd = (ws.subspace_loss(Xp, V)[0] - ws.subspace_loss(Xm, V)[0]) / (2 * h)
            an = dX[i, j].real if part == "re" else dX[i, j].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_subspace_loss_invariances():
    """0 when span(X) = span(V), whatever the basis (phases, rotations); nb when X is orthogonal to V; unchanged by
    X -> X R."""
    g = np.random.default_rng(5)
    Q, _ = np.linalg.qr(g.standard_normal((40, 6)) + 1j * g.standard_normal((40, 6)))
    V, W = Q[:, :3], Q[:, 3:]
    R = g.standard_normal((3, 3)) + 1j * g.standard_normal((3, 3))
    assert abs(ws.subspace_loss(V @ R, V)[0]) < 1e-12
    assert abs(ws.subspace_loss(W @ R, V)[0] - 3.0) < 1e-12
    X = g.standard_normal((40, 3)) + 1j * g.standard_normal((40, 3))
    assert abs(ws.subspace_loss(X, V)[0] - ws.subspace_loss(X @ R, V)[0]) < 1e-10


def test_conv_delta_kernel_is_subsampling():
    """A kernel with only the centre tap (identity over channels) picks u[c, 2q]: the stride-2 sampling."""
    g = np.random.default_rng(6)
    u = g.standard_normal((3, 8, 8, 8))
    W = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        W[c, c, 1, 1, 1] = 1.0
    out = ws.conv_s2_forward(u, W, np.zeros(3))
    assert np.array_equal(out, u[:, ::2, ::2, ::2])


def test_conv_is_circular_and_shift_equivariant():
    """Shifting the input by 2 points shifts the output by 1 (stride 2, periodic), and a tap at offset -1 wraps."""
    g = np.random.default_rng(7)
    u = g.standard_normal((2, 8, 8, 8))
    W = g.standard_normal((3, 2, 3, 3, 3))
    b = g.standard_normal(3)
    out = ws.conv_s2_forward(u, W, b)
    out_s = ws.conv_s2_forward(np.roll(u, 2, axis=3), W, b)
    assert np.allclose(out_s, np.roll(out, 1, axis=3), atol=1e-13)
    Wt = np.zeros((1, 1, 3, 3, 3))
    Wt[0, 0, 1, 1, 0] = 1.0  # dx = 0: reads x = 2q - 1, i.e. x = 7 for q = 0
    o = ws.conv_s2_forward(u[:1], Wt, np.zeros(1))
    assert o[0, 0, 0, 0] == u[0, 0, 0, 7]


def test_upsample_exactness():
    """Rows sum to 1 (constants reproduced); points on the coarse lattice copy it exactly; the fine values between two
    coarse points are on the straight line between them."""
    U = ws.upsample_matrix(16)
    assert np.allclose(U.sum(axis=1), 1.0)
    c = np.random.default_rng(8).standard_normal((4, 4, 4))
    f = ws.upsample_forward(c, U)
    assert np.array_equal(f[::4, ::4, ::4], c)
    assert np.allclose(f[0, 0, 1], 0.75 * c[0, 0, 0] + 0.25 * c[0, 0, 1])
    assert np.allclose(f[0, 0, 14], 0.5 * c[0, 0, 3] + 0.5 * c[0, 0, 0])  # periodic wrap
    d = np.random.default_rng(9).standard_normal((16, 16, 16))
    assert np.isclose(np.sum(ws.upsample_backward(d, U) * c), np.sum(d * f))  # the adjoint


def test_film_identity_and_k_periodicity():
    """With Fa = fa = Fc = fc = 0 the FiLM layer passes u2 through; the outputs are periodic in k with period 2 pi."""
    p = ws.init_params(C1, C2, NB, 3)
    m0, k, _, _ = random_sample(10)
    X, y, cache = ws.forward(p, m0, k, NB)
    assert np.array_equal(cache["z"], cache["u2"])
    X2, y2, _ = ws.forward(p, m0, k + 2 * np.pi * np.array([1.0, -1.0, 0.0]), NB)
    assert np.allclose(X2, X, atol=1e-12) and np.allclose(y2, y, atol=1e-12)


def test_adam_first_step_closed_form():
    """After one step m^ = g and v^ = g^2, so every entry moves by -lr g / (|g| + eps)."""
    p = {k: np.ones(3) for k in ws.PARAM_ORDER}
    g = {k: np.array([2.0, -0.5, 1e-3]) for k in ws.PARAM_ORDER}
    st = ws.adam_init(p)
    ws.adam_step(p, g, st, lr=0.01)
    for k in ws.PARAM_ORDER:
        assert np.allclose(p[k], 1.0 - 0.01 * g[k] / (np.abs(g[k]) + 1e-8), rtol=0, atol=1e-15)


def method_samples(nsamp=3, nb=NB):
    """(m0, k, V, lambda) from dense eigensolves of the compensated operator on small random structures."""
    out = []
    for s in range(nsamp):
        st = wl.random_structure(s)
        m0 = geometry.m0_from_structure(N, st.as_array(), st.eps_bg)
        k = np.array([0.3 + 0.4 * s, -0.5, 0.8])
        h = 1.0 / N
        Op = mfd.compensated_operator(N, k, h, m0.ravel(), mfd.penalty_gamma(h, k), 1)
        lam, V = eigs.lowest_dense(Op, nb)
        out.append((m0, k, V, lam))
    return out


def test_training_lowers_the_loss_on_method_eigenvectors():
    """40 Adam steps on 3 structures solved by the method (dense at N = 8) lower the mean loss by a clear margin."""
    samples = method_samples()
    p = ws.init_params(C1, C2, NB, 0)
    st = ws.adam_init(p)
    first, _ = ws.batch_loss_and_grad(p, samples, NB)
    for _ in range(40):
        L, g = ws.batch_loss_and_grad(p, samples, NB)
        ws.adam_step(p, g, st, lr=3e-3)
    last, _ = ws.batch_loss_and_grad(p, samples, NB)
    assert last < 0.8 * first


def test_planted_backward_mistake_is_caught(monkeypatch):
    """A transposed convolution that scatters with the forward roll direction (a plausible sign slip) fails the
    finite-difference pin of W1."""
    def wrong(u, W, dout):
        du = np.zeros_like(u)
        dW = np.zeros_like(W)
        for dz, dy, dx in ws._taps():
            dW[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", dout, ws._window(u, dz, dy, dx))
            buf = np.zeros_like(u)
            buf[:, ::2, ::2, ::2] = np.einsum("oc,ozyx->czyx", W[:, :, dz, dy, dx], dout)
            du += np.roll(buf, shift=(-(dz - 1), -(dy - 1), -(dx - 1)), axis=(1, 2, 3))
        return du, dW, dout.sum(axis=(1, 2, 3))
    monkeypatch.setattr(ws, "conv_s2_backward", wrong)
    assert fd_check(small_params(), random_sample(), "W1") > 1e-3


def test_library_initial_parameters_follow_the_reference_layout():
    """The training driver's flat initial parameters have the library's count and the reference's layout: FiLM at
    the identity and zero biases, so the first forward pass of both starts from the same kind of model."""
    from paper_2503_19379_gb300 import warmstart as lws
    flat = lws.init_params(8, seed=3)
    ref = ws.init_params(8, 16, 8, 3)
    assert flat.size == sum(v.size for v in ref.values())
    off = 0
    for k in ws.PARAM_ORDER:
        part = flat[off:off + ref[k].size]
        if k[0] in "bf" or k in ("Fa", "Fc"):
            assert np.all(part == 0.0), k
        off += ref[k].size
