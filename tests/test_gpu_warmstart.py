"""The learned warm start's kernels (pc_ws_forward, pc_ws_backward, pc_ws_adam) against the FP64 reference of the
network (oracle/warmstart.py), and a short training run on the device against the same run of the reference.

The network is FP32 on the device and FP64 in the reference; both take the same FP32-rounded parameters and inputs.
Tolerances: the forward outputs are sums of at most 81 + 27 * 8 + 16 products per value, so FP32 rounding leaves
a relative error of a few 1e-7 of the largest output (checked at 2e-5); the gradients sum up to (N/2)^3 = 512
products per entry over a mean of S samples (checked at 1e-3 of the largest entry of each parameter group, which
also absorbs the rare pre-activation within FP32 rounding of zero whose ReLU decision can differ).
"""
import numpy as np
import pytest

from oracle import warmstart as ws

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C1, C2 = 8, 16  # PC_WS_C1, PC_WS_C2 of include/pc.h


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    import os
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2503_19379_gb300 as p
    return p


def params64(nb, seed):
    p = ws.init_params(C1, C2, nb, seed)
    g = np.random.default_rng(seed + 50)
    for k in ("Fa", "fa", "Fc", "fc", "b1", "b2", "bh", "bv"):
        p[k] = 0.2 * g.standard_normal(p[k].shape)
    # the device holds FP32 parameters: give the reference the same values
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


def flat(p):
    return np.concatenate([p[k].ravel() for k in ws.PARAM_ORDER]).astype(np.float32)


def unflat(v, p_like):
    out, o = {}, 0
    for k in ws.PARAM_ORDER:
        n = p_like[k].size
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(p_like[k].shape)
        o += n
    return out


def inputs(N, nb, S, nstruct, seed):
    g = np.random.default_rng(seed)
    m0 = g.uniform(1.0 / 13.0, 1.0, (nstruct, 3, N, N, N)).astype(np.float32)
    sidx = g.integers(0, nstruct, S).astype(np.int32)
    kpts = g.uniform(-3.5, 3.5, (S, 3))
    V = np.empty((S, nb, 3 * N ** 3), dtype=np.complex64)
    for s in range(S):
        q, _ = np.linalg.qr(g.standard_normal((3 * N ** 3, nb)) + 1j * g.standard_normal((3 * N ** 3, nb)))
        V[s] = q.T.astype(np.complex64)
    lam = g.uniform(2.0, 60.0, (S, nb))
    return m0, sidx, kpts, V, lam


@pytest.mark.parametrize("N,nb,S", [(16, 4, 3), (32, 8, 2)])
def test_forward_backward_match_reference(pcmod, N, nb, S):
    p = params64(nb, seed=N + nb)
    m0, sidx, kpts, V, lam = inputs(N, nb, S, nstruct=2, seed=7 * N + nb)
    net = pcmod.WarmStart(N, nb, S, params=torch.from_numpy(flat(p)))
    assert net.P == flat(p).size
    m0d = torch.from_numpy(m0).cuda()
    sd = torch.from_numpy(sidx).cuda()
    X, y = net.forward(m0d, sd, kpts)
    Xh = X.cpu().numpy().reshape(S, nb, -1)
    yh = y.cpu().numpy()
    w_val = 0.1
    samples = []
    for s in range(S):
        m0s = m0[sidx[s]].astype(np.float64)
        Xr, yr, _ = ws.forward(p, m0s, kpts[s], nb)
        assert np.max(np.abs(Xh[s].T - Xr)) <= 2e-5 * np.max(np.abs(Xr))
        assert np.max(np.abs(yh[s] - yr)) <= 2e-5 * max(1.0, np.max(np.abs(yr)))
        samples.append((m0s, kpts[s], V[s].T.astype(np.complex128), lam[s]))
    grad, loss = net.backward(m0d, sd, X, y, torch.from_numpy(V).cuda(), torch.from_numpy(lam).cuda(), w_val)
    gh = unflat(grad.cpu().numpy(), p)
    lref, gref = ws.batch_loss_and_grad(p, samples, nb, w_val)
    assert abs(float(loss.mean()) - lref) <= 1e-4 * max(1.0, abs(lref))
    for s in range(S):
        ls, _ = ws.loss(p, *samples[s], nb, w_val)
        assert abs(float(loss[s]) - ls) <= 1e-4 * max(1.0, abs(ls))
    for k in ws.PARAM_ORDER:
        scale = np.max(np.abs(gref[k]))
        assert np.max(np.abs(gh[k] - gref[k])) <= 1e-3 * scale + 1e-7, k


def test_adam_matches_reference(pcmod):
    nb = 4
    p = params64(nb, seed=3)
    g = np.random.default_rng(9)
    grads = [g.standard_normal(flat(p).size).astype(np.float32) * 0.01 for _ in range(3)]
    net = pcmod.WarmStart(16, nb, 1, params=torch.from_numpy(flat(p)))
    ref = {k: v.copy() for k, v in p.items()}
    st = ws.adam_init(ref)
    for gv in grads:
        net.adam(torch.from_numpy(gv).cuda(), lr=2e-3)
        ws.adam_step(ref, unflat(gv, p), st, lr=2e-3)
    got = unflat(net.params.cpu().numpy(), p)
    for k in ws.PARAM_ORDER:
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-6, k


def test_training_run_matches_reference(pcmod):
    """Twelve Adam steps on a fixed batch of four samples, on the device and in the reference from the same start:
    the loss histories agree, and the loss falls."""
    N, nb, S = 16, 4, 4
    p = params64(nb, seed=21)
    m0, sidx, kpts, V, lam = inputs(N, nb, S, nstruct=3, seed=5)
    net = pcmod.WarmStart(N, nb, S, params=torch.from_numpy(flat(p)))
    m0d, sd = torch.from_numpy(m0).cuda(), torch.from_numpy(sidx).cuda()
    Vd, lamd = torch.from_numpy(V).cuda(), torch.from_numpy(lam).cuda()
    samples = [(m0[sidx[s]].astype(np.float64), kpts[s], V[s].T.astype(np.complex128), lam[s]) for s in range(S)]
    ref = {k: v.copy() for k, v in p.items()}
    st = ws.adam_init(ref)
    hist_dev, hist_ref = [], []
    for _ in range(12):
        X, y = net.forward(m0d, sd, kpts)
        grad, loss = net.backward(m0d, sd, X, y, Vd, lamd, 0.1)
        net.adam(grad, lr=3e-3)
        hist_dev.append(float(loss.mean()))
        lr_, gr = ws.batch_loss_and_grad(ref, samples, nb, 0.1)
        ws.adam_step(ref, gr, st, lr=3e-3)
        hist_ref.append(lr_)
    hist_dev, hist_ref = np.array(hist_dev), np.array(hist_ref)
    assert np.max(np.abs(hist_dev - hist_ref) / hist_ref) <= 2e-3
    assert hist_dev[-1] < hist_dev[0]
