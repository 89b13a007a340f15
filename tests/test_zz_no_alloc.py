"""pc_gram_pair_noalloc, the allocation-free Gram pair, agrees with pc_gram_pair and with numpy's own products.

Some callers cannot allocate device memory (a fixed memory budget, an application allocator that must own every
allocation, or a loop where cudaMalloc/cudaFree would synchronise the device); this entry point serves them from a
fixed array inside the library. The test calls both entry points through the C ABI on the same inputs, twice in a
row with different data, so that any state left in the shared array by the first call would show up in the second,
and checks both against S^H S and S^H AS formed by numpy in complex128 from the same (rounded) inputs.

Tolerances: complex128, 1e-13 sqrt(L) times the largest entry; complex64 (FP32 products, partial sums in FP32 over
row chunks), 4e-6 |s_i| |a_j| per entry, the FP32 accuracy bound of the library's Gram products.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcmod():
    from paper_2503_19379_gb300 import build as b
    import os
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2503_19379_gb300 as p
    return p


def panel(seed, nb, p, L, dtype):
    g = np.random.default_rng(seed)
    S = g.standard_normal((nb, p, L)) + 1j * g.standard_normal((nb, p, L))
    AS = S * g.uniform(0.5, 2.0, L)[None, None, :]  # image under a Hermitian operator
    return (torch.from_numpy(S).to(dtype).cuda().contiguous(), torch.from_numpy(AS).to(dtype).cuda().contiguous())


def numpy_pair(S, AS):
    """G = S^H S and H = S^H AS per k-point, complex128, from the device inputs' own values."""
    s = S.cpu().numpy().astype(np.complex128)
    a = AS.cpu().numpy().astype(np.complex128)
    return s.conj() @ s.transpose(0, 2, 1), s.conj() @ a.transpose(0, 2, 1)


def call(pcmod, name, S, AS):
    lib = pcmod.lib()
    nb, p, L = S.shape
    G = torch.empty((nb, p, p), dtype=torch.complex128, device="cuda")
    H = torch.empty_like(G)
    code = 0 if S.dtype == torch.complex128 else 1
    rc = getattr(lib, name)(nb, L, p, code, ctypes.c_void_p(S.data_ptr()), p * L, ctypes.c_void_p(AS.data_ptr()),
                            ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(H.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.pc_last_error()
    torch.cuda.synchronize()
    return G.cpu().numpy(), H.cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_gram_pair_matches_allocating_entry(pcmod, dtype):
    for seed, (nb, p, L) in ((1, (3, 48, 98304)), (2, (2, 13, 5001))):  # two calls in a row, different shapes
        S, AS = panel(seed, nb, p, L, dtype)
        G0, H0 = call(pcmod, "pc_gram_pair", S, AS)
        G1, H1 = call(pcmod, "pc_gram_pair_noalloc", S, AS)
        Gr, Hr = numpy_pair(S, AS)
        if dtype == torch.complex128:
            tolG = 1e-13 * np.sqrt(L) * np.max(np.abs(Gr))
            tolH = 1e-13 * np.sqrt(L) * np.max(np.abs(Hr))
        else:
            ns = np.linalg.norm(S.cpu().numpy().astype(np.complex128), axis=2)
            na = np.linalg.norm(AS.cpu().numpy().astype(np.complex128), axis=2)
            tolG = 4e-6 * ns[:, :, None] * ns[:, None, :]
            tolH = 4e-6 * ns[:, :, None] * na[:, None, :]
        for G, H in ((G1, H1), (G0, H0)):
            assert np.all(np.abs(G - Gr) <= tolG)
            assert np.all(np.abs(H - Hr) <= tolH)


def test_noalloc_rejects_oversized_request(pcmod):
    lib = pcmod.lib()
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.pc_gram_pair_noalloc(64, 16, 64, 0, ptr, 0, ptr, ptr, ptr, None)  # 64 * 64 * 64 > 131072
    assert rc == -1 and b"exceeds the fixed scratch" in lib.pc_last_error()
