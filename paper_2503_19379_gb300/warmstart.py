"""Training and evaluation of the learned warm start on the device (the warm-start workload: seeded random
structures of 1-8 spheres in a cubic cell, eigenvectors from the solver itself).

Every numerical step runs in libpc: the solves (pc_solve), the network's forward and backward passes and Adam
(pc_ws_*). This module only orders the calls and keeps the training set resident on the device: the eigenvectors
as complex64, M0 per structure as float32, the eigenvalues as float64.
"""
from __future__ import annotations

import numpy as np

from . import pc


def make_dataset(N: int, structures, kpts, nbands: int, tol: float = 1e-6, precision: int = pc.PC_PREC_MIXED):
    """Solve every structure at every k-point and keep (M0, k, eigenvectors, eigenvalues) on the device.

    structures: list of (spheres [n][5], eps_bg); kpts: array [nk][3]. Returns a dict of torch tensors:
    m0 [ns][3][N][N][N] float32, sidx [ns nk] int32, k (host) [ns nk][3], V [ns nk][nbands][3][N][N][N] complex64,
    lam [ns nk][nbands] float64, iters [ns nk] (the random-start iteration counts)."""
    torch = pc._torch()
    kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
    nk = kpts.shape[0]
    m0s, V, lam, sidx, ks, iters = [], [], [], [], [], []
    for si, (spheres, eps_bg) in enumerate(structures):
        eps = pc.eps_spheres(N, spheres, eps_bg)
        solver = pc.Solver(N, eps, precision=precision)
        out = solver.solve(kpts, nbands, tol, want_vectors=True)
        solver.close()
        m0s.append(torch.from_numpy(1.0 / eps).float())
        V.append(out["evecs"].to(torch.complex64))
        lam.append(torch.from_numpy(out["evals"]))
        sidx += [si] * nk
        ks.append(kpts)
        iters.append(out["iters"])
    return {
        "m0": torch.stack(m0s).cuda(),
        "sidx": torch.tensor(sidx, dtype=torch.int32, device="cuda"),
        "k": np.concatenate(ks),
        "V": torch.cat(V),
        "lam": torch.cat(lam).cuda(),
        "iters": np.concatenate(iters),
    }


def train(data, nbands: int, epochs: int, batch: int, lr: float = 1e-3, seed: int = 0, w_val: float = 0.1,
          params=None):
    """Adam over mini-batches of `batch` samples (the sample order reshuffled each epoch by a seeded generator).
    Returns the network and the mean loss of every epoch."""
    torch = pc._torch()
    N = data["m0"].shape[-1]
    nsamp = data["V"].shape[0]
    net = pc.WarmStart(N, nbands, batch, params=params)
    if params is None:
        net.params.copy_(torch.from_numpy(init_params(nbands, seed)))
    rng = np.random.default_rng(seed)
    history = []
    for _ in range(epochs):
        order = rng.permutation(nsamp)
        losses = []
        for b0 in range(0, nsamp - batch + 1, batch):
            idx = torch.from_numpy(order[b0:b0 + batch]).cuda()
            sidx = data["sidx"][idx].contiguous()
            X, y = net.forward(data["m0"], sidx, data["k"][order[b0:b0 + batch]])
            grad, loss = net.backward(data["m0"], sidx, X, y, data["V"][idx].contiguous(),
                                      data["lam"][idx].contiguous(), w_val)
            net.adam(grad, lr=lr)
            losses.append(float(loss.mean()))
        history.append(float(np.mean(losses)) if losses else float("nan"))
    return net, history


def init_params(nbands: int, seed: int = 0) -> np.ndarray:
    """Seeded initial parameters in the library's flat order: He-normal convolutions and head, zero biases, FiLM at
    the identity."""
    g = np.random.default_rng(seed)
    C1, C2 = pc.PC_WS_C1, pc.PC_WS_C2
    parts = [
        g.standard_normal(C1 * 3 * 27) * np.sqrt(2.0 / (3 * 27)), np.zeros(C1),
        g.standard_normal(C2 * C1 * 27) * np.sqrt(2.0 / (C1 * 27)), np.zeros(C2),
        np.zeros(C2 * 6), np.zeros(C2), np.zeros(C2 * 6), np.zeros(C2),
        g.standard_normal(6 * nbands * C2) * np.sqrt(1.0 / C2), np.zeros(6 * nbands),
        g.standard_normal(nbands * (C2 + 6)) * np.sqrt(1.0 / (C2 + 6)), np.zeros(nbands),
    ]
    return np.concatenate(parts).astype(np.float32)


def evaluate(net, N: int, structures, kpts, nbands: int, tol: float = 1e-6, precision: int = pc.PC_PREC_MIXED):
    """Iterations to tolerance from the random block and from the network's block, on the given structures (held
    out from training), with the eigenvalues of both solves. Returns a dict of arrays [ns][nk]."""
    torch = pc._torch()
    kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
    nk = kpts.shape[0]
    out = {"iters_random": [], "iters_warm": [], "max_rel_diff": []}
    for spheres, eps_bg in structures:
        eps = pc.eps_spheres(N, spheres, eps_bg)
        solver = pc.Solver(N, eps, precision=precision)
        base = solver.solve(kpts, nbands, tol)
        m0 = torch.from_numpy(1.0 / eps).float().cuda()[None]
        X0 = []
        for k0 in range(0, nk, net.S):
            kk = kpts[k0:k0 + net.S]
            pad = net.S - kk.shape[0]
            kb = np.concatenate([kk, np.zeros((pad, 3))]) if pad else kk
            X, _ = net.forward(m0, torch.zeros(net.S, dtype=torch.int32, device="cuda"), kb)
            X0.append(X[:kk.shape[0]])
        warm = solver.solve(kpts, nbands, tol, x0=torch.cat(X0).contiguous())
        solver.close()
        out["iters_random"].append(base["iters"])
        out["iters_warm"].append(warm["iters"])
        out["max_rel_diff"].append(float(np.max(np.abs(warm["evals"] - base["evals"]) / base["evals"])))
    return {k: np.asarray(v) for k, v in out.items()}
