"""FP64 reference of the learned warm start for the block eigensolver (test infrastructure only).

The paper has no network: this is the warm-start model the project defines for LOBPCG (Section 5.1's initial block
X is "random" there). A small 3D convolutional encoder reads the edge permittivity of a structure and, conditioned on
the Bloch vector k, predicts an initial block X0 of nb face fields and guesses of the nb lowest eigenvalues. Every
layer below is written out plainly, forward and backward by hand; the backward passes are pinned by central finite
differences, so the CUDA kernels have a checked reference for both directions.

Model (parameters in a dict of float64 arrays, shapes in brackets):
* input  u0 = M0 = 1/eps at the three edge sets, 3 channels on the N^3 grid;
* conv1  3 -> C1 channels, 3x3x3 kernel, stride 2, circular padding, bias, ReLU          -> (N/2)^3  [W1, b1]
* conv2  C1 -> C2, same form                                                              -> (N/4)^3  [W2, b2]
* k features phi(k) = (sin k_1, sin k_2, sin k_3, cos k_1, cos k_2, cos k_3): periodic under k -> k + 2 pi e_i,
  the reduction the solver applies to k on the cube;
* FiLM   z = (1 + Fa phi + fa) * u2 + (Fc phi + fc), per channel                              [Fa, fa, Fc, fc]
* head   1x1x1 conv C2 -> 6 nb channels: band b, component c, (re, im)                        [Wh, bh]
* upsampling by 4 per axis, periodic linear interpolation, to the N^3 face grid: X0 (nb, 3, N, N, N) complex;
* value head  y = Wv [mean(z); phi] + bv, the guesses of log lambda_b                          [Wv, bv]

Loss for one sample (eps, k, V, lambda) with V (3N^3 x nb) the orthonormal eigenvectors the solver returned:
* subspace term  L_X = nb - tr(G^{-1} B B^H), G = X^H X, B = X^H V: nb minus the squared cosines of the principal
  angles between span(X) and span(V). It is invariant under X -> X R for any invertible R (phases, rotations inside
  degenerate clusters), as an initial block for a subspace method should be;
* value term     L_y = sum_b (y_b - log lambda_b)^2, weighted by w_val.
Its gradient with respect to X (real and imaginary parts) is -2 [(I - X G^{-1} X^H) V B^H G^{-1}].

Adam (Kingma and Ba, 2015) updates the parameters.
"""
from __future__ import annotations

import numpy as np

PARAM_ORDER = ("W1", "b1", "W2", "b2", "Fa", "fa", "Fc", "fc", "Wh", "bh", "Wv", "bv")


# ---------------------------------------------------------------------------------------------------------------- init
def init_params(C1: int, C2: int, nb: int, seed: int = 0) -> dict:
    """Seeded parameters: He-normal convolutions, zero biases, FiLM at the identity (Fa = Fc = 0)."""
    g = np.random.default_rng(seed)
    p = {
        "W1": g.standard_normal((C1, 3, 3, 3, 3)) * np.sqrt(2.0 / (3 * 27)),
        "b1": np.zeros(C1),
        "W2": g.standard_normal((C2, C1, 3, 3, 3)) * np.sqrt(2.0 / (C1 * 27)),
        "b2": np.zeros(C2),
        "Fa": np.zeros((C2, 6)),
        "fa": np.zeros(C2),
        "Fc": np.zeros((C2, 6)),
        "fc": np.zeros(C2),
        "Wh": g.standard_normal((6 * nb, C2)) * np.sqrt(1.0 / C2),
        "bh": np.zeros(6 * nb),
        "Wv": g.standard_normal((nb, C2 + 6)) * np.sqrt(1.0 / (C2 + 6)),
        "bv": np.zeros(nb),
    }
    return p


# ------------------------------------------------------------------------------------------------------------ layers
def _taps():
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                yield dz, dy, dx


def _window(u: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """u[c, 2q + d - 1] (circular) for every output point q: roll by -(d - 1), keep every second point."""
    r = np.roll(u, shift=(-(dz - 1), -(dy - 1), -(dx - 1)), axis=(1, 2, 3))
    return r[:, ::2, ::2, ::2]


def conv_s2_forward(u: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[o, q] = b[o] + sum_{c, d} W[o, c, d] u[c, 2q + d - 1 (mod n)]: 3x3x3 kernel, stride 2, circular."""
    C, n = u.shape[0], u.shape[1]
    out = np.zeros((W.shape[0], n // 2, n // 2, n // 2)) + b[:, None, None, None]
    for dz, dy, dx in _taps():
        out += np.einsum("oc,czyx->ozyx", W[:, :, dz, dy, dx], _window(u, dz, dy, dx))
    return out


def conv_s2_backward(u: np.ndarray, W: np.ndarray, dout: np.ndarray):
    """Gradients (du, dW, db) of conv_s2_forward given dL/dout: du is the transposed (scatter) stencil."""
    du = np.zeros_like(u)
    dW = np.zeros_like(W)
    for dz, dy, dx in _taps():
        dW[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", dout, _window(u, dz, dy, dx))
        buf = np.zeros_like(u)
        buf[:, ::2, ::2, ::2] = np.einsum("oc,ozyx->czyx", W[:, :, dz, dy, dx], dout)
        du += np.roll(buf, shift=(dz - 1, dy - 1, dx - 1), axis=(1, 2, 3))
    db = dout.sum(axis=(1, 2, 3))
    return du, dW, db


def relu_forward(a: np.ndarray) -> np.ndarray:
    return np.maximum(a, 0.0)


def relu_backward(a: np.ndarray, dout: np.ndarray) -> np.ndarray:
    """Subgradient 0 at a = 0."""
    return dout * (a > 0.0)


def k_features(kvec) -> np.ndarray:
    k = np.asarray(kvec, dtype=np.float64)
    return np.concatenate([np.sin(k), np.cos(k)])


def upsample_matrix(n: int, factor: int = 4) -> np.ndarray:
    """U (n x n/factor): fine point i = factor j + r takes (1 - r/factor) c_j + (r/factor) c_{j+1}, periodic."""
    m = n // factor
    U = np.zeros((n, m))
    for i in range(n):
        j, r = divmod(i, factor)
        U[i, j] += 1.0 - r / factor
        U[i, (j + 1) % m] += r / factor
    return U


def upsample_forward(c: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Separable interpolation of the last three axes (z, y, x) of c by U."""
    return np.einsum("Zz,Yy,Xx,...zyx->...ZYX", U, U, U, c)


def upsample_backward(dout: np.ndarray, U: np.ndarray) -> np.ndarray:
    """The transpose: U^T along each of the last three axes."""
    return np.einsum("Zz,Yy,Xx,...ZYX->...zyx", U, U, U, dout)


# ------------------------------------------------------------------------------------------------------- the network
def forward(p: dict, m0: np.ndarray, kvec, nb: int):
    """X0 (3 N^3 x nb complex, the block's columns) and the guesses y (nb) of log lambda; plus the cache for backward."""
    m0 = np.asarray(m0, dtype=np.float64).reshape(3, *np.shape(m0)[-3:])
    n = m0.shape[1]
    a1 = conv_s2_forward(m0, p["W1"], p["b1"])
    u1 = relu_forward(a1)
    a2 = conv_s2_forward(u1, p["W2"], p["b2"])
    u2 = relu_forward(a2)
    phi = k_features(kvec)
    sa = 1.0 + p["Fa"] @ phi + p["fa"]
    sc = p["Fc"] @ phi + p["fc"]
    z = sa[:, None, None, None] * u2 + sc[:, None, None, None]
    h = np.einsum("oc,czyx->ozyx", p["Wh"], z) + p["bh"][:, None, None, None]
    m = n // 4
    hc = h.reshape(nb, 3, 2, m, m, m)
    coarse = hc[:, :, 0] + 1j * hc[:, :, 1]
    U = upsample_matrix(n)
    X = upsample_forward(coarse, U).reshape(nb, -1).T
    feat = np.concatenate([z.mean(axis=(1, 2, 3)), phi])
    y = p["Wv"] @ feat + p["bv"]
    cache = dict(m0=m0, a1=a1, u1=u1, a2=a2, u2=u2, phi=phi, sa=sa, z=z, U=U, feat=feat, n=n, nb=nb)
    return X, y, cache


def subspace_loss(X: np.ndarray, V: np.ndarray):
    """L_X = nb - tr(G^{-1} B B^H) and dL/d(Re X) + i dL/d(Im X); V has orthonormal columns."""
    G = X.conj().T @ X
    B = X.conj().T @ V
    Gi = np.linalg.inv(G)
    BB = B @ B.conj().T
    L = V.shape[1] - float(np.real(np.trace(Gi @ BB)))
    grad_conj = V @ B.conj().T @ Gi - X @ Gi @ BB @ Gi  # d f / d conj(X) of f = tr(G^{-1} B B^H)
    return L, -2.0 * grad_conj


def loss(p: dict, m0, kvec, V, lam, nb: int, w_val: float = 0.1):
    """Total loss of one sample and the cache pieces backward needs."""
    X, y, cache = forward(p, m0, kvec, nb)
    LX, dX = subspace_loss(X, V)
    ly = np.log(np.asarray(lam, dtype=np.float64))
    Ly = float(np.sum((y - ly) ** 2))
    cache.update(dX=dX, dy=w_val * 2.0 * (y - ly))
    return LX + w_val * Ly, cache


def backward(p: dict, cache: dict) -> dict:
    """dL/dparam for every parameter, from the loss cache (chain rule through each layer above, in reverse)."""
    nb, n = cache["nb"], cache["n"]
    m = n // 4
    g = {}
    # value head
    dy = cache["dy"]
    g["Wv"] = np.outer(dy, cache["feat"])
    g["bv"] = dy.copy()
    dfeat = p["Wv"].T @ dy
    C2 = p["Wh"].shape[1]
    dz = np.broadcast_to((dfeat[:C2] / (m ** 3))[:, None, None, None], cache["z"].shape).copy()
    dphi = dfeat[C2:].copy()
    # X = upsample(coarse) as columns; dX holds dL/dRe + i dL/dIm
    dXf = cache["dX"].T.reshape(nb, 3, n, n, n)
    dcoarse = upsample_backward(dXf, cache["U"])
    dh = np.stack([dcoarse.real, dcoarse.imag], axis=2).reshape(6 * nb, m, m, m)
    g["Wh"] = np.einsum("ozyx,czyx->oc", dh, cache["z"])
    g["bh"] = dh.sum(axis=(1, 2, 3))
    dz += np.einsum("oc,ozyx->czyx", p["Wh"], dh)
    # FiLM
    u2, phi, sa = cache["u2"], cache["phi"], cache["sa"]
    dsa = np.sum(dz * u2, axis=(1, 2, 3))
    dsc = dz.sum(axis=(1, 2, 3))
    g["Fa"] = np.outer(dsa, phi)
    g["fa"] = dsa
    g["Fc"] = np.outer(dsc, phi)
    g["fc"] = dsc
    dphi += p["Fa"].T @ dsa + p["Fc"].T @ dsc  # (k is an input: dphi is not used further)
    du2 = sa[:, None, None, None] * dz
    # encoder
    da2 = relu_backward(cache["a2"], du2)
    du1, g["W2"], g["b2"] = conv_s2_backward(cache["u1"], p["W2"], da2)
    da1 = relu_backward(cache["a1"], du1)
    _, g["W1"], g["b1"] = conv_s2_backward(cache["m0"], p["W1"], da1)
    return g


# ---------------------------------------------------------------------------------------------------------- training
def adam_init(p: dict) -> dict:
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p: dict, g: dict, st: dict, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, bias-corrected, p -= lr m^/(sqrt v^ + eps)."""
    st["t"] += 1
    t = st["t"]
    for k in PARAM_ORDER:
        st["m"][k] = b1 * st["m"][k] + (1.0 - b1) * g[k]
        st["v"][k] = b2 * st["v"][k] + (1.0 - b2) * g[k] ** 2
        mh = st["m"][k] / (1.0 - b1 ** t)
        vh = st["v"][k] / (1.0 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def batch_loss_and_grad(p: dict, samples, nb: int, w_val: float = 0.1):
    """Mean loss and gradient over samples = [(m0, k, V, lam), ...]."""
    total = 0.0
    acc = {k: np.zeros_like(v) for k, v in p.items()}
    for m0, kvec, V, lam in samples:
        L, cache = loss(p, m0, kvec, V, lam, nb, w_val)
        g = backward(p, cache)
        total += L
        for k in acc:
            acc[k] += g[k]
    s = len(samples)
    return total / s, {k: v / s for k, v in acc.items()}
