"""The C-ABI library builds for sm_103a, loads, and exports every entry point that include/pc.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pc.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(pc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2503_19379_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("pc_setup", "pc_solve", "pc_destroy", "pc_last_error", "pc_apply_op", "pc_apply_precond", "pc_gram",
              "pc_rayleigh_ritz", "pc_block_update", "pc_residual", "pc_recompute_norms", "pc_eps_spheres"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2503_19379_gb300 import pc
    assert set(declared_symbols()) <= set(pc.SIGNATURES)


def test_opts_default_and_errors_without_gpu(libpath):
    """Host-side validation runs without a device: bad arguments are rejected before any CUDA call."""
    from paper_2503_19379_gb300 import pc
    o = pc.default_opts()
    assert (o.order, o.guard, o.maxiter, o.precision) == (1, -1, 400, 0)
    import numpy as np
    h = ctypes.c_void_p()
    eps = np.ones(3 * 6 ** 3)
    rc = pc.lib().pc_setup(ctypes.byref(h), 6, pc._dptr(eps), None, None, None)  # N not a power of two >= 8
    assert rc == -1 and b"power of two" in pc.lib().pc_last_error()
    eps = np.ones(3 * 8 ** 3)
    eps[5] = -1.0
    rc = pc.lib().pc_setup(ctypes.byref(h), 8, pc._dptr(eps), None, None, None)
    assert rc == -1 and b"eps_edges" in pc.lib().pc_last_error()
    lat = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, 1.0, 0.0]]).ravel()  # a3 = a1 + a2: a singular cell
    rc = pc.lib().pc_setup(ctypes.byref(h), 8, pc._dptr(np.ones(3 * 8 ** 3)), pc._dptr(lat), None, None)
    assert rc == -1 and b"independent" in pc.lib().pc_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2503_19379_gb300 import pc
    monkeypatch.setattr(pc, "_LIB", None)
    monkeypatch.setattr(pc, "LIBPATH", str(tmp_path / "nope.so"))
    with pytest.raises(pc.PCError):
        pc.lib()


@pytest.mark.parametrize("korder", [1, 2, 3, 4])
def test_stencil_coefficients_match_table1(libpath, korder):
    """pc_stencil_coefficients (the closed-form weights the CUDA path uses) equals the oracle's Table 1 exactly, and
    satisfies the 2k-th order moment conditions: sum c_s (2s-1)^(2p+1) = [p = 0], sum d_s (2s-1)^(2p) = [p = 0] / 2
    for p < k. Host only."""
    import numpy as np

    from oracle import mfd
    from paper_2503_19379_gb300 import pc
    c, d = pc.stencil_coefficients(korder)
    tc, td = mfd.TABLE1[korder]
    assert np.array_equal(c, np.asarray(tc, dtype=np.float64))
    assert np.array_equal(d, np.asarray(td, dtype=np.float64))
    o = 2.0 * np.arange(1, korder + 1) - 1.0
    for p in range(korder):
        assert abs(np.sum(c * o ** (2 * p + 1)) - (1.0 if p == 0 else 0.0)) <= 1e-12
        assert abs(np.sum(d * o ** (2 * p)) - (0.5 if p == 0 else 0.0)) <= 1e-12


def test_stencil_coefficients_reject_other_orders(libpath):
    from paper_2503_19379_gb300 import pc
    for bad in (0, 5):
        with pytest.raises(pc.PCError):
            pc.stencil_coefficients(bad)


def test_header_is_plain_c():
    """include/pc.h is a C ABI: it compiles as C99 (no C++ or CUDA types in the signatures)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    res = subprocess.run([cc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Werror", HEADER],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def _setup_rc(N, eps=None, lattice=None, **opts):
    """pc_setup through ctypes; returns (rc, message). Every case below fails argument validation before any CUDA
    call, so no GPU is needed."""
    import ctypes as C

    import numpy as np

    from paper_2503_19379_gb300 import pc
    L = pc.lib()
    o = pc.default_opts(**opts)
    e = np.ones((3, N, N, N)) if eps is None else eps
    h = C.c_void_p()
    lat = None if lattice is None else np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).ravel())
    rc = L.pc_setup(C.byref(h), N, pc._dptr(np.ascontiguousarray(e, dtype=np.float64)),
                    pc._dptr(lat) if lat is not None else None, C.byref(o), None)
    return rc, L.pc_last_error().decode()


def test_setup_rejects_bad_arguments_on_the_host(libpath):
    import numpy as np
    rc, msg = _setup_rc(12)
    assert rc == -1 and "power of two" in msg
    rc, msg = _setup_rc(8, lattice=np.diag([1.0, 1.0, 2.0]), order=2, precision=1)
    assert rc == -2 and "mixed" in msg
    rc, msg = _setup_rc(8, lattice=[0.0, 0.5, 0.5, 0.5, 0.0, 0.5, 0.5, 0.5, 0.0 * np.nan])
    assert rc == -1 and "finite" in msg
    rc, msg = _setup_rc(8, lattice=[1.0, 2.0, 3.0, 2.0, 4.0, 6.0, 0.0, 0.0, 1.0])
    assert rc == -1 and "independent" in msg
    rc, msg = _setup_rc(8, order=5)
    assert rc == -2 and "order" in msg
    rc, msg = _setup_rc(8, order=2, precision=1)
    assert rc == -2 and "mixed" in msg
    bad = np.ones((3, 8, 8, 8))
    bad[1, 2, 3, 4] = 0.0
    rc, msg = _setup_rc(8, eps=bad)
    assert rc == -1 and "eps_edges" in msg


def test_eps_spheres_lattice_rejects_bad_arguments_on_the_host(libpath):
    """pc_eps_spheres_lattice validates the cell and the spheres before any CUDA call."""
    import numpy as np

    from paper_2503_19379_gb300 import pc
    out = np.empty((3, 8, 8, 8))
    sph = np.array([[0.0, 0.0, 0.0, 0.2, 13.0]])
    L = pc.lib()
    flat = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0])  # a3 = a1 + a2
    assert L.pc_eps_spheres_lattice(8, pc._dptr(flat), 1, pc._dptr(sph), 1.0, pc._dptr(out)) == -1
    assert b"independent" in L.pc_last_error()
    bad = np.array([[0.0, 0.0, 0.0, 0.2, -1.0]])
    eye = np.eye(3).ravel()
    assert L.pc_eps_spheres_lattice(8, pc._dptr(eye), 1, pc._dptr(bad), 1.0, pc._dptr(out)) == -1
    assert L.pc_eps_spheres_lattice(8, None, 1, pc._dptr(sph), 1.0, pc._dptr(out)) == -1


def test_lattice_vectors_layout():
    """The binding passes a_1, a_2, a_3 one after the other: the columns of A, as pc_setup documents."""
    import numpy as np

    from paper_2503_19379_gb300 import pc
    A = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 10.0]])
    v = pc.lattice_vectors(A)
    assert np.array_equal(v[0:3], A[:, 0]) and np.array_equal(v[3:6], A[:, 1]) and np.array_equal(v[6:9], A[:, 2])


def test_warm_start_host_entry_points(libpath):
    """The warm start's parameter count equals the oracle's model, the workspace size is positive, and bad sizes are
    rejected before any CUDA call."""
    import ctypes as C

    import numpy as np

    from oracle import warmstart as ws
    from paper_2503_19379_gb300 import pc
    L = pc.lib()
    for nb in (1, 8, 16):
        p = ws.init_params(8, 16, nb)
        assert L.pc_ws_param_count(nb) == sum(v.size for v in p.values())
    assert L.pc_ws_param_count(0) == -1 and L.pc_ws_param_count(17) == -1
    assert L.pc_ws_work_bytes(32, 8, 4) > 0 and L.pc_ws_work_bytes(12, 8, 4) == 0
    k = np.zeros(3)
    rc = L.pc_ws_forward(12, 8, 1, None, None, 1, None, pc._dptr(k), None, None, None, None)
    assert rc == -1 and b"power of two" in L.pc_last_error()
    rc = L.pc_ws_forward(32, 8, 1, None, None, 1, None, pc._dptr(k), None, None, None, None)
    assert rc == -1 and b"null" in L.pc_last_error()
    rc = L.pc_ws_adam(4, None, None, None, None, 1, C.c_float(1e-3), C.c_float(0.9), C.c_float(0.999),
                      C.c_float(1e-8), None)
    assert rc == -1


def test_solve_init_rejects_null_arguments_on_the_host(libpath):
    import numpy as np

    from paper_2503_19379_gb300 import pc
    k = np.zeros(3)
    ev = np.zeros(4)
    rc = pc.lib().pc_solve_init(None, 1, pc._dptr(k), 4, 1e-6, None, 2, pc._dptr(ev), None, None, None)
    assert rc == -1 and b"null" in pc.lib().pc_last_error()


def test_structure_entry_points_reject_bad_arguments_on_the_host(libpath):
    import numpy as np

    from paper_2503_19379_gb300 import pc
    L = pc.lib()
    out = np.empty((3, 8, 8, 8))
    flat = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0])
    assert L.pc_eps_gyroid(8, pc._dptr(flat), 1.0, 1.1, 16.0, 1.0, pc._dptr(out)) == -1
    assert L.pc_eps_diamond(8, pc._dptr(flat), 1.0, 0.12, 0.11, 13.0, 1.0, pc._dptr(out)) == -1
    eye = np.eye(3).ravel()
    assert L.pc_eps_gyroid(8, pc._dptr(eye), -1.0, 1.1, 16.0, 1.0, pc._dptr(out)) == -1
    assert L.pc_eps_diamond(8, pc._dptr(eye), 1.0, -0.1, 0.11, 13.0, 1.0, pc._dptr(out)) == -1


def test_opts_layout_matches_the_header(tmp_path):
    """The binding's Opts mirrors pc_opts field by field: sizes and offsets from a C program compiled against
    include/pc.h equal ctypes' (a drift here would shift every option after it)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2503_19379_gb300 import pc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    names = [f[0] for f in pc.Opts._fields_]
    body = "".join(f'printf("%zu ", offsetof(pc_opts, {n}));' for n in names)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pc.h"\nint main(void){' + body +
                   'printf("%zu\\n", sizeof(pc_opts)); return 0;}\n')
    exe = tmp_path / "layout"
    res = subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [getattr(pc.Opts, n).offset for n in names] + [ctypes.sizeof(pc.Opts)]
    assert got == want


def test_kchunk_option_validated_on_the_host(libpath):
    from paper_2503_19379_gb300 import pc
    rc, msg = _setup_rc(8, kchunk=-1)
    assert rc == -1 and "kchunk" in msg
    assert pc.default_opts().kchunk == 0
