"""ctypes binding of libpc (include/pc.h): same entry points, argument marshalling only.

Host buffers are numpy arrays; device buffers are torch CUDA tensors (complex128 / complex64 / float64), used only
as device memory. Work is issued on torch's current CUDA stream unless a stream is given.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libpc.so")

PC_C128, PC_C64, PC_C128_DF = 0, 1, 2
PC_PRECOND_GAMMA, PC_PRECOND_LAPLACIAN = 0, 1
PC_PREC_FP64, PC_PREC_MIXED = 0, 1
PC_WS_C1, PC_WS_C2 = 8, 16  # warm-start encoder channels (include/pc.h)
PC_NOT_CONVERGED, PC_SPURIOUS = 1, 2


class PCError(RuntimeError):
    pass


STAGES = ("stencil", "precond", "gram", "rr", "update", "residual", "recompute", "other", "dfloat")


class StageStat(C.Structure):
    _fields_ = [("calls", C.c_long), ("kernels", C.c_long), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("order", C.c_int), ("gamma_override", C.c_double), ("precond", C.c_int), ("precision", C.c_int),
                ("guard", C.c_int), ("maxiter", C.c_int), ("max_doublings", C.c_int), ("seed", C.c_uint64),
                ("groups", C.c_int), ("kchunk", C.c_int)]


_LIB = None
_vp, _i, _l, _d, _u64 = C.c_void_p, C.c_int, C.c_long, C.c_double, C.c_uint64
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)

SIGNATURES = {
    "pc_opts_default": (_i, [C.POINTER(Opts)]),
    "pc_setup": (_i, [C.POINTER(_vp), _i, _dp, _dp, C.POINTER(Opts), _vp]),
    "pc_solve": (_i, [_vp, _i, _dp, _i, _d, _dp, _vp, _ip, _dp]),
    "pc_solve_init": (_i, [_vp, _i, _dp, _i, _d, _vp, _i, _dp, _vp, _ip, _dp]),
    "pc_get_fp64_finish": (_i, [_vp, _i, _ip]),
    "pc_destroy": (None, [_vp]),
    "pc_last_error": (C.c_char_p, []),
    "pc_eps_spheres": (_i, [_i, _i, _dp, _d, _dp]),
    "pc_eps_spheres_lattice": (_i, [_i, _dp, _i, _dp, _d, _dp]),
    "pc_eps_gyroid": (_i, [_i, _dp, _d, _d, _d, _d, _dp]),
    "pc_eps_diamond": (_i, [_i, _dp, _d, _d, _d, _d, _d, _dp]),
    "pc_apply_op": (_i, [_vp, _i, _dp, _dp, _i, _i, _vp, _vp]),
    "pc_apply_half": (_i, [_vp, _i, _dp, _i, _vp, _vp, _vp]),
    "pc_recompute_norms": (_i, [_vp, _i, _dp, _i, _vp, _vp]),
    "pc_stencil_coefficients": (_i, [_i, _dp, _dp]),
    "pc_apply_precond": (_i, [_vp, _i, _dp, _dp, _i, _i, _vp, _vp]),
    "pc_gram": (_i, [_i, _l, _i, _i, _i, _vp, _l, _vp, _l, _vp, _vp]),
    "pc_gram_pair": (_i, [_i, _l, _i, _i, _vp, _l, _vp, _vp, _vp, _vp]),
    "pc_gram_pair_noalloc": (_i, [_i, _l, _i, _i, _vp, _l, _vp, _vp, _vp, _vp]),
    "pc_gram_pair_coupled": (_i, [_i, _l, _i, _i, _vp, _l, _vp, _vp, _l, _vp, _vp, _vp, _vp]),
    "pc_block_update": (_i, [_i, _l, _i, _i, _i, _vp, _l, _vp, _vp, _l, _vp]),
    "pc_eigh_batched": (_i, [_i, _i, _vp, _vp, _vp, _vp]),
    "pc_rayleigh_ritz": (_i, [_i, _i, _i, _vp, _vp, _d, _vp, _vp, _vp, _vp]),
    "pc_residual": (_i, [_i, _l, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pc_init_block": (_i, [_i, _l, _i, _u64, _i, _vp, _vp]),
    "pc_set_timing": (_i, [_vp, _i]),
    "pc_get_stats": (_i, [_vp, C.POINTER(StageStat)]),
    "pc_reset_stats": (_i, [_vp]),
    "pc_ws_param_count": (_l, [_i]),
    "pc_ws_work_bytes": (C.c_size_t, [_i, _i, _i]),
    "pc_ws_forward": (_i, [_i, _i, _i, _vp, _vp, _i, _vp, _dp, _vp, _vp, _vp, _vp]),
    "pc_ws_backward": (_i, [_i, _i, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp]),
    "pc_ws_adam": (_i, [_l, _vp, _vp, _vp, _vp, _i, C.c_float, C.c_float, C.c_float, C.c_float, _vp]),
}


def lib():
    """Load libpc.so (built in-tree); raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIBPATH):
            raise PCError(f"{LIBPATH} is missing: build it with paper_2503_19379_gb300.build.build()")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, what, warn_ok=False):
    if rc < 0 or (rc > 0 and not warn_ok):
        raise PCError(f"{what} failed ({rc}): {lib().pc_last_error().decode()}")
    return rc


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtypes=None):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise PCError("expected a contiguous CUDA tensor")
    if dtypes is not None and t.dtype not in dtypes:
        raise PCError(f"unexpected dtype {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.complex128:
        return PC_C128
    if t.dtype == torch.complex64:
        return PC_C64
    raise PCError(f"unsupported dtype {t.dtype}")


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(lib().pc_opts_default(C.byref(o)), "pc_opts_default")
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def stencil_coefficients(order: int):
    """Table 1 weights (c, d) of the 2k-th order scheme, k = order (pc_stencil_coefficients; host only)."""
    c = np.zeros(4)
    d = np.zeros(4)
    _check(lib().pc_stencil_coefficients(int(order), _dptr(c), _dptr(d)), "pc_stencil_coefficients")
    return c[:order].copy(), d[:order].copy()


def eps_spheres(N: int, spheres, eps_bg: float) -> np.ndarray:
    """Permittivity at the edge DoFs, host array (3, N, N, N) (pc_eps_spheres)."""
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 5))
    out = np.empty((3, N, N, N), dtype=np.float64)
    _check(lib().pc_eps_spheres(N, sph.shape[0], _dptr(sph) if sph.size else None, float(eps_bg), _dptr(out)),
           "pc_eps_spheres")
    return out


def lattice_vectors(lattice) -> np.ndarray:
    """The C layout of a lattice matrix A (columns a_1, a_2, a_3): a_1, a_2, a_3 one after the other."""
    A = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
    return np.ascontiguousarray(A.T).ravel()


def eps_spheres_lattice(N: int, lattice, spheres, eps_bg: float) -> np.ndarray:
    """Permittivity at the edge DoFs of a general cell, host array (3, N, N, N) (pc_eps_spheres_lattice). ``lattice``
    is A with the lattice vectors as columns; sphere centres and radii are Cartesian."""
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 5))
    lat = lattice_vectors(lattice)
    out = np.empty((3, N, N, N), dtype=np.float64)
    _check(lib().pc_eps_spheres_lattice(N, _dptr(lat), sph.shape[0], _dptr(sph) if sph.size else None,
                                        float(eps_bg), _dptr(out)), "pc_eps_spheres_lattice")
    return out


def eps_gyroid(N: int, lattice, l: float = 1.0, threshold: float = 1.1, eps_in: float = 16.0,
               eps_bg: float = 1.0) -> np.ndarray:
    """Permittivity at the edge DoFs of the single gyroid (Section 6.3) on the cell A (pc_eps_gyroid)."""
    out = np.empty((3, N, N, N), dtype=np.float64)
    _check(lib().pc_eps_gyroid(N, _dptr(lattice_vectors(lattice)), float(l), float(threshold), float(eps_in),
                               float(eps_bg), _dptr(out)), "pc_eps_gyroid")
    return out


def eps_diamond(N: int, lattice, l: float = 1.0, r: float = 0.12, b: float = 0.11, eps_in: float = 13.0,
                eps_bg: float = 1.0) -> np.ndarray:
    """Permittivity at the edge DoFs of the diamond of spheres and spheroids (Section 6.3) on the cell A
    (pc_eps_diamond)."""
    out = np.empty((3, N, N, N), dtype=np.float64)
    _check(lib().pc_eps_diamond(N, _dptr(lattice_vectors(lattice)), float(l), float(r), float(b), float(eps_in),
                                float(eps_bg), _dptr(out)), "pc_eps_diamond")
    return out


class Solver:
    """One structure on one grid: pc_setup / pc_solve / pc_destroy and the step-level kernels. ``lattice`` is the
    matrix A whose columns are the lattice vectors (None: the unit cube)."""

    def __init__(self, N: int, eps_edges: np.ndarray, stream=None, lattice=None, **opts):
        self.N = int(N)
        self.n = self.N ** 3
        eps = np.ascontiguousarray(np.asarray(eps_edges, dtype=np.float64).reshape(3, N, N, N))
        self.opts = default_opts(**opts)
        self._stream = _stream(stream)
        h = C.c_void_p()
        lat = lattice_vectors(np.eye(3) if lattice is None else lattice)
        _check(lib().pc_setup(C.byref(h), self.N, _dptr(eps), _dptr(lat), C.byref(self.opts), self._stream),
               "pc_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, kpts, nbands: int, tol: float, want_vectors: bool = False, x0=None):
        """pc_solve (pc_solve_init when x0, a torch complex64 CUDA tensor [nk][n0][3][N][N][N], gives the first n0
        columns of the initial block); returns dict(evals, iters, resid, status, fp64_finish (1 where the mixed
        solve handed the k-point to the FP64 solve)[, evecs (torch complex128)])."""
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        nk = k.shape[0]
        evals = np.zeros((nk, nbands))
        resid = np.zeros((nk, nbands))
        iters = np.zeros(nk, dtype=np.int32)
        evecs = None
        if want_vectors:
            torch = _torch()
            evecs = torch.empty((nk, nbands, 3, self.N, self.N, self.N), dtype=torch.complex128, device="cuda")
        ev = _dev(evecs) if evecs is not None else None
        if x0 is None:
            rc = lib().pc_solve(self._h, nk, _dptr(k), nbands, float(tol), _dptr(evals), ev,
                                iters.ctypes.data_as(_ip), _dptr(resid))
        else:
            torch = _torch()
            if tuple(x0.shape[:1]) != (nk,) or tuple(x0.shape[2:]) != (3, self.N, self.N, self.N):
                raise PCError("x0 must have shape [nk][n0][3][N][N][N]")
            rc = lib().pc_solve_init(self._h, nk, _dptr(k), nbands, float(tol), _dev(x0, [torch.complex64]),
                                     int(x0.shape[1]), _dptr(evals), ev, iters.ctypes.data_as(_ip), _dptr(resid))
        _check(rc, "pc_solve", warn_ok=True)
        finish = np.zeros(nk, dtype=np.int32)
        _check(lib().pc_get_fp64_finish(self._h, nk, finish.ctypes.data_as(_ip)), "pc_get_fp64_finish")
        out = {"evals": evals, "iters": iters, "resid": resid, "status": rc, "fp64_finish": finish}
        if evecs is not None:
            out["evecs"] = evecs
        return out

    # ---- tracing
    def set_timing(self, enable: bool):
        _check(lib().pc_set_timing(self._h, int(bool(enable))), "pc_set_timing")

    def reset_stats(self):
        _check(lib().pc_reset_stats(self._h), "pc_reset_stats")

    def stats(self) -> dict:
        arr = (StageStat * len(STAGES))()
        _check(lib().pc_get_stats(self._h, arr), "pc_get_stats")
        return {name: {"calls": a.calls, "kernels": a.kernels, "ms": a.ms, "flops": a.flops, "bytes": a.bytes}
                for name, a in zip(STAGES, arr)}

    # ---- step-level kernels (device tensors shaped (nb, m, 3, N, N, N))
    def apply_op(self, kpts, gammas, X, double_float=False):
        """Y = Op X; double_float=True evaluates a complex128 block in double-float arithmetic (PC_C128_DF)."""
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).reshape(-1))
        Y = _torch().empty_like(X)
        nb, m = X.shape[0], X.shape[1]
        code = _dtype_code(X)
        if double_float:
            if code != PC_C128:
                raise PCError("double-float evaluation needs a complex128 block")
            code = PC_C128_DF
        _check(lib().pc_apply_op(self._h, nb, _dptr(k), _dptr(g), m, code, _dev(X), _dev(Y)), "pc_apply_op")
        return Y

    def apply_half(self, kpts, X):
        torch = _torch()
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        nb, m = X.shape[0], X.shape[1]
        E = torch.empty_like(X)
        Cc = torch.empty((nb, m, self.N, self.N, self.N), dtype=X.dtype, device=X.device)
        _check(lib().pc_apply_half(self._h, nb, _dptr(k), m, _dev(X, [torch.complex128]), _dev(E), _dev(Cc)),
               "pc_apply_half")
        return E, Cc

    def recompute_norms(self, kpts, X):
        torch = _torch()
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        nb, m = X.shape[0], X.shape[1]
        out = torch.empty((nb, m, 3), dtype=torch.float64, device=X.device)
        _check(lib().pc_recompute_norms(self._h, nb, _dptr(k), m, _dev(X, [torch.complex128]), _dev(out)),
               "pc_recompute_norms")
        return out

    def apply_precond(self, kpts, gammas, R, out=None):
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).reshape(-1))
        W = _torch().empty_like(R) if out is None else out
        nb, m = R.shape[0], R.shape[1]
        _check(lib().pc_apply_precond(self._h, nb, _dptr(k), _dptr(g), m, _dtype_code(R), _dev(R), _dev(W)),
               "pc_apply_precond")
        return W


def gram(A, B, stream=None):
    """G_b = A_b^H B_b for A (nb, p, L), B (nb, q, L) device tensors (columns contiguous)."""
    torch = _torch()
    nb, p, L = A.shape
    q = B.shape[1]
    G = torch.empty((nb, p, q), dtype=torch.complex128, device=A.device)
    _check(lib().pc_gram(nb, L, p, q, _dtype_code(A), _dev(A), p * L, _dev(B), q * L, _dev(G), _stream(stream)),
           "pc_gram")
    return G


def gram_pair_coupled(S, AS, R, stream=None):
    """(G, H, RQ) = (S^H S, S^H AS, R^H S) for complex64 panels S, AS (nb, p, L) and R (nb, q, L) in one pass
    (pc_gram_pair_coupled)."""
    torch = _torch()
    nb, p, L = S.shape
    q = R.shape[1]
    G = torch.empty((nb, p, p), dtype=torch.complex128, device=S.device)
    H = torch.empty_like(G)
    RQ = torch.empty((nb, q, p), dtype=torch.complex128, device=S.device)
    _check(lib().pc_gram_pair_coupled(nb, L, p, q, _dev(S, [torch.complex64]), p * L, _dev(AS, [torch.complex64]),
                                      _dev(R, [torch.complex64]), q * L, _dev(G), _dev(H), _dev(RQ), _stream(stream)),
           "pc_gram_pair_coupled")
    return G, H, RQ


def gram_pair(S, AS, stream=None):
    """(G, H) = (S^H S, S^H AS) for panels S, AS (nb, p, L), Hermitian (upper triangle computed, mirrored)."""
    torch = _torch()
    nb, p, L = S.shape
    G = torch.empty((nb, p, p), dtype=torch.complex128, device=S.device)
    H = torch.empty_like(G)
    _check(lib().pc_gram_pair(nb, L, p, _dtype_code(S), _dev(S), p * L, _dev(AS), _dev(G), _dev(H),
                              _stream(stream)), "pc_gram_pair")
    return G, H


def block_update(S, Cm, stream=None):
    """Y_b = S_b C_b for S (nb, p, L) (columns contiguous) and C (nb, p, q) complex128; returns (nb, q, L)."""
    torch = _torch()
    nb, p, L = S.shape
    q = Cm.shape[2]
    Y = torch.empty((nb, q, L), dtype=S.dtype, device=S.device)
    _check(lib().pc_block_update(nb, L, p, q, _dtype_code(S), _dev(S), p * L, _dev(Cm, [torch.complex128]), _dev(Y),
                                 q * L, _stream(stream)), "pc_block_update")
    return Y


def eigh_batched(A, stream=None):
    torch = _torch()
    nb, n, _ = A.shape
    w = torch.empty((nb, n), dtype=torch.float64, device=A.device)
    V = torch.empty_like(A)
    _check(lib().pc_eigh_batched(nb, n, _dev(A, [torch.complex128]), _dev(w), _dev(V), _stream(stream)),
           "pc_eigh_batched")
    return w, V


def rayleigh_ritz(G, H, m: int, drop: float = 1e-12, stream=None):
    torch = _torch()
    nb, n, _ = G.shape
    theta = torch.empty((nb, m), dtype=torch.float64, device=G.device)
    coef = torch.empty((nb, n, m), dtype=torch.complex128, device=G.device)
    rank = torch.empty((nb,), dtype=torch.int32, device=G.device)
    _check(lib().pc_rayleigh_ritz(nb, n, m, _dev(G, [torch.complex128]), _dev(H, [torch.complex128]), float(drop),
                                  _dev(theta), _dev(coef), _dev(rank), _stream(stream)), "pc_rayleigh_ritz")
    return theta, coef, rank


def residual(X, AX, theta, stream=None):
    """R = AX - X diag(theta) and column norms (|r|, |x|) for X, AX (nb, m, L) complex128."""
    torch = _torch()
    nb, m, L = X.shape
    R = torch.empty_like(X)
    norms = torch.empty((nb, m, 2), dtype=torch.float64, device=X.device)
    _check(lib().pc_residual(nb, L, m, _dev(X, [torch.complex128]), _dev(AX, [torch.complex128]),
                             _dev(theta, [torch.float64]), _dev(R), _dev(norms), _stream(stream)), "pc_residual")
    return R, norms


def init_block(nb: int, L: int, m: int, seed: int, kidx0: int = 0, stream=None):
    torch = _torch()
    X = torch.empty((nb, m, L), dtype=torch.complex128, device="cuda")
    _check(lib().pc_init_block(nb, L, m, seed, kidx0, _dev(X), _stream(stream)), "pc_init_block")
    return X


class WarmStart:
    """The learned warm start's network on the device (pc_ws_*): forward, backward and Adam over a flat float32
    parameter tensor. Tensors are torch CUDA tensors; m0 is float32 [nstruct][3][N][N][N], sidx int32 [S]."""

    def __init__(self, N: int, nb: int, S: int, params=None, stream=None):
        torch = _torch()
        self.N, self.nb, self.S = int(N), int(nb), int(S)
        self.P = int(lib().pc_ws_param_count(self.nb))
        if self.P <= 0:
            raise PCError(f"pc_ws_param_count: nb = {nb} out of range")
        wb = int(lib().pc_ws_work_bytes(self.N, self.nb, self.S))
        if wb == 0:
            raise PCError(f"pc_ws_work_bytes: N = {N}, nb = {nb}, S = {S} out of range")
        self.work = torch.empty(wb, dtype=torch.uint8, device="cuda")
        self.params = (torch.zeros(self.P, dtype=torch.float32, device="cuda") if params is None
                       else params.to(device="cuda", dtype=torch.float32).contiguous())
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self._stream = _stream(stream)

    def forward(self, m0, sidx, kpts):
        """(X [S][nb][3][N][N][N] complex64, y [S][nb] float32) for the S samples."""
        torch = _torch()
        k = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(self.S, 3))
        X = torch.empty((self.S, self.nb, 3, self.N, self.N, self.N), dtype=torch.complex64, device="cuda")
        y = torch.empty((self.S, self.nb), dtype=torch.float32, device="cuda")
        _check(lib().pc_ws_forward(self.N, self.nb, self.S, _dev(self.params, [torch.float32]),
                                   _dev(m0, [torch.float32]), int(m0.shape[0]), _dev(sidx, [torch.int32]), _dptr(k),
                                   _dev(X), _dev(y), _dev(self.work), self._stream), "pc_ws_forward")
        return X, y

    def backward(self, m0, sidx, X, y, V, lam, w_val: float = 0.1):
        """(grad [P] float32, loss [S] float64) for the samples of the preceding forward."""
        torch = _torch()
        grad = torch.empty_like(self.params)
        loss = torch.empty(self.S, dtype=torch.float64, device="cuda")
        _check(lib().pc_ws_backward(self.N, self.nb, self.S, _dev(self.params, [torch.float32]),
                                    _dev(m0, [torch.float32]), int(m0.shape[0]), _dev(sidx, [torch.int32]),
                                    _dev(X, [torch.complex64]),
                                    _dev(y, [torch.float32]), _dev(V, [torch.complex64]), _dev(lam, [torch.float64]),
                                    float(w_val), _dev(grad), _dev(loss), _dev(self.work), self._stream),
               "pc_ws_backward")
        return grad, loss

    def adam(self, grad, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        _check(lib().pc_ws_adam(self.P, _dev(self.params), _dev(grad), _dev(self.m), _dev(self.v), self.t, float(lr),
                                float(b1), float(b2), float(eps), self._stream), "pc_ws_adam")
