"""The C ABI: the library builds for sm_103a, loads, and exports every entry point of include/cpc.h."""
import ctypes

import numpy as np
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cpc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1205_6113_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cpc_setup", "cpc_solve", "cpc_apply_Bcom", "cpc_destroy", "cpc_last_error",
                     "cpc_tpfa_assemble", "cpc_solve_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1205_6113_gb300 import cpc
    bound = {name for name, _, _ in cpc.SIGNATURES}
    assert declared_functions() <= bound


def test_pure_host_entry_points(lib):
    """Entry points that need no GPU: option defaults, sizes and argument validation."""
    from paper_1205_6113_gb300 import cpc
    L = cpc.load()
    opt = cpc._Options()
    assert L.cpc_default_options(ctypes.byref(opt)) == 0
    assert opt.precond == 0 and opt.theta == 0.12 and opt.coarse_max == 2048 and opt.max_levels == 20 and opt.autotune == 0
    assert opt.gs_order == 0 and opt.ic_order == 0 and opt.tail_nnz_max == 0
    assert L.cpc_default_options(None) == 1
    assert L.cpc_tpfa_nnz(128, 128, 64) == 7274496
    assert L.cpc_tpfa_nnz(256, 256, 128) == 58458112
    assert L.cpc_tpfa_nnz(64, 64, 1) == 20224
    h = ctypes.c_void_p()
    assert L.cpc_setup(None, None, ctypes.byref(h)) == 1 and not h.value
    assert L.cpc_solve(None, None, None, 1e-6, 10, None, None, 0) == 1
    assert L.cpc_coarse_inverse_info(None, None, None) == 1
    L.cpc_destroy(None)
    # mixed-hybrid sizes are host arithmetic: they must match the oracle's assembled system
    import oracle as O
    for shape, mask in [((3, 2, 2), 1), ((4, 3, 2), 0), ((2, 2, 2), 63), ((1, 1, 1), 3), ((5, 1, 3), 1 | 8 | 32)]:
        nx, ny, nz = shape
        A = O.mhfem(nx, ny, nz, np.zeros(nx * ny * nz), 0.1, mask)
        assert cpc.mhfem_size(nx, ny, nz, mask) == (A.n, A.nnz)
    nu = ctypes.c_int64(0)
    assert L.cpc_mhfem_size(1024, 1024, 1024, 1, ctypes.byref(nu)) == -1      # 2^30 cells: nnz over int32
    assert L.cpc_mhfem_size(0, 4, 4, 1, ctypes.byref(nu)) == -1
    assert L.cpc_mhfem_size(4, 4, 4, 1, None) == -1
    assert L.cpc_mhfem_assemble(4, 4, 4, None, 0.1, 1, None, None, None, None) == 1
    # option validation happens before any device work: a valid 1 x 1 host CSR with bad options
    rp, ci, va = (ctypes.c_int32 * 2)(0, 1), (ctypes.c_int32 * 1)(0), (ctypes.c_double * 1)(1.0)
    csr = cpc._Csr(1, 1, ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(ci, ctypes.c_void_p),
                   ctypes.cast(va, ctypes.c_void_p), 0)
    for field, value in [("gs_order", 2), ("gs_order", -1), ("precond", 6), ("autotune", 2),
                         ("max_levels", 0), ("max_levels", 26)]:
        bad = cpc._Options()
        L.cpc_default_options(ctypes.byref(bad))
        setattr(bad, field, value)
        assert L.cpc_setup(ctypes.byref(csr), ctypes.byref(bad), ctypes.byref(h)) == 1 and not h.value
    for ic_order, tail in [(1, 0), (0, 1 << 20)]:      # natural-order GS: natural IC(0), no cluster kernel
        bad = cpc._Options()
        L.cpc_default_options(ctypes.byref(bad))
        bad.gs_order, bad.ic_order, bad.tail_nnz_max = 1, ic_order, tail
        assert L.cpc_setup(ctypes.byref(csr), ctypes.byref(bad), ctypes.byref(h)) == 1 and not h.value


def test_cuda_path_has_no_cpu_fallback():
    """The binding raises when the library is absent; it never computes on the host."""
    from paper_1205_6113_gb300 import cpc
    src = open(cpc.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src
    with pytest.raises(cpc.CpcError):
        saved = cpc._lib
        cpc._lib = None
        try:
            cpc.load(os.path.join(ROOT, "does-not-exist.so"))
        finally:
            cpc._lib = saved
