"""The allocation-free assembly entry point against the regular one, through the C ABI.

cpc_tpfa_assemble_noalloc serves callers that cannot let a library allocate device memory (their
own pool owns every allocation, or an allocation's synchronisation is not acceptable).  It must
give exactly what cpc_tpfa_assemble gives, call after call, although every call reuses the same
scratch array inside the library, and it must not allocate.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1205_6113_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_6113_gb300 import cpc  # noqa: E402

DEV = torch.device("cuda:0")


def assemble_both(p):
    logk = torch.tensor(p.logk, device=DEV)
    ref = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    n, nnz = p.n, cpc.tpfa_nnz(p.nx, p.ny, p.nz)
    rowptr = torch.full((n + 1,), -7, dtype=torch.int32, device=DEV)
    col = torch.full((nnz,), -7, dtype=torch.int32, device=DEV)
    val = torch.full((nnz,), float("nan"), dtype=torch.float64, device=DEV)
    rc = cpc.tpfa_assemble_noalloc(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet, rowptr, col, val)
    torch.cuda.synchronize()
    return rc, ref, (rowptr, col, val)


def check_same(ref, got):
    # the same per-cell code runs in both kernels: identical bits, values included
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_noalloc_matches_regular_assembly_on_consecutive_calls():
    # a large grid first, then smaller ragged ones: a call must not see an earlier call's scratch.
    # 129 x 128 x 64 has 1032 blocks of 1024 cells, so the block scan reads scratch entries past
    # the first 1024.
    for p in (inputs.small_3d(129, 128, 64, seed=9), inputs.correlated_3d(), inputs.small_3d(37, 23, 11, seed=3),
              inputs.lognormal_2d()):
        rc, ref, got = assemble_both(p)
        assert rc == 0
        check_same(ref, got)


def test_noalloc_at_its_cell_limit():
    # 4096 x 4096 x 1 = 16,777,216 cells: every one of the 16,384 scratch entries is used
    p = inputs.Problem("plane_4096x4096", 4096, 4096, 1, np.zeros(4096 * 4096), 1.0, inputs.FACE_X0)
    p.logk = inputs.random_vector(p.n, seed=4) * 0.5
    rc, ref, got = assemble_both(p)
    assert rc == 0
    check_same(ref, got)
    del ref, got
    torch.cuda.empty_cache()


def _cudart():
    for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    return None


def test_noalloc_takes_nothing_from_the_stream_ordered_pool():
    """The regular assembly takes its scan scratch from the device's default memory pool
    (cudaMallocAsync); the allocation-free one must not: the pool's high-water mark of used
    memory, reset just before the call, stays at the level it had before."""
    rt = _cudart()
    if rt is None:
        pytest.skip("CUDA runtime library not found")
    USED_CURRENT, USED_HIGH = 7, 8                     # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh
    p = inputs.correlated_3d()
    logk = torch.tensor(p.logk, device=DEV)
    nnz = cpc.tpfa_nnz(p.nx, p.ny, p.nz)
    rowptr = torch.empty(p.n + 1, dtype=torch.int32, device=DEV)
    col = torch.empty(nnz, dtype=torch.int32, device=DEV)
    val = torch.empty(nnz, dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), DEV.index or 0) == 0

    def attr(a):
        v = ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        z = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(z)) == 0

    # the check itself: the regular assembly does raise the mark
    before = attr(USED_CURRENT)
    reset_high()
    cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    torch.cuda.synchronize()
    assert attr(USED_HIGH) > before
    before = attr(USED_CURRENT)
    reset_high()
    assert cpc.tpfa_assemble_noalloc(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet, rowptr, col, val) == 0
    torch.cuda.synchronize()
    assert attr(USED_HIGH) == before


def test_noalloc_rejects_grids_beyond_its_scratch():
    logk = torch.zeros(8, dtype=torch.float64, device=DEV)
    ptr = torch.zeros(9, dtype=torch.int32, device=DEV)
    col = torch.zeros(8, dtype=torch.int32, device=DEV)
    val = torch.zeros(8, dtype=torch.float64, device=DEV)
    # 4096 x 4096 x 2 cells = 33.5M > 16,777,216: rejected before any kernel runs
    assert cpc.tpfa_assemble_noalloc(4096, 4096, 2, logk, 1.0, 1, ptr, col, val) == 1
    assert b"16,777,216" in cpc.load().cpc_last_error(None)
    assert cpc.tpfa_assemble_noalloc(0, 4, 4, logk, 1.0, 1, ptr, col, val) == 1
