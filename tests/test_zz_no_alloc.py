"""The allocation-free assembly entry point against the regular one, through the C ABI.

cpc_tpfa_assemble_noalloc serves callers that cannot let a library allocate device memory (their
own pool owns every allocation, or an allocation's synchronisation is not acceptable).  It must
give exactly what cpc_tpfa_assemble gives, call after call, although every call reuses the same
scratch array inside the library.  This file is collected last on purpose.
"""
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
    for a, b in zip(ref[:2], got[:2]):
        assert torch.equal(a, b)
    ra, rb = ref[2].cpu().numpy(), got[2].cpu().numpy()
    assert np.all(np.isfinite(rb))
    assert np.max(np.abs(ra - rb)) <= 1e-14 * np.max(np.abs(ra))


def test_noalloc_matches_regular_assembly_on_consecutive_calls():
    # a large grid first, then a smaller ragged one: the second call must not see the first's scratch
    for p in (inputs.correlated_3d(), inputs.small_3d(37, 23, 11, seed=3), inputs.lognormal_2d()):
        rc, ref, got = assemble_both(p)
        assert rc == 0
        check_same(ref, got)


def test_noalloc_rejects_grids_beyond_its_scratch():
    logk = torch.zeros(8, dtype=torch.float64, device=DEV)
    ptr = torch.zeros(9, dtype=torch.int32, device=DEV)
    col = torch.zeros(8, dtype=torch.int32, device=DEV)
    val = torch.zeros(8, dtype=torch.float64, device=DEV)
    # 4096 x 4096 x 2 cells = 33.5M > 16,777,216: rejected before any kernel runs
    assert cpc.tpfa_assemble_noalloc(4096, 4096, 2, logk, 1.0, 1, ptr, col, val) == 1
    assert cpc.tpfa_assemble_noalloc(0, 4, 4, logk, 1.0, 1, ptr, col, val) == 1
