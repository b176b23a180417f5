"""Block PCG (O'Leary 1980; cpc_solve_block) against the oracle's block_pcg.

The oracle runs the same recurrences in NumPy with the oracle's preconditioner column by column
(pinned in test_oracle_pins.py: K = 1 is textbook PCG, finite termination, no more iterations than
the slowest column).  At tol 1e-10 the GPU's block iteration count is within 1 of the oracle's and
every column within 1e-8 (FP64 preconditioner; 1e-5 with FP32).  Ragged K (not a multiple of 32)
and both padded widths (32, 64) are covered; a rank-deficient block ends in a breakdown, a zero
column and AMG(ILU(0)) are rejected.  At 128 x 128 x 64 with 64 right-hand sides every column
reaches the tolerance on its true residual, in no more block iterations than the slowest single
solve.
"""
import numpy as np
import pytest

import oracle as O
from paper_1205_6113_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_6113_gb300 import cpc  # noqa: E402

DEV = torch.device("cuda:0")


def rhs_block(n, K, seed, cells=4):
    return np.ascontiguousarray(inputs.batch_rhs(n, K, cells_per_rhs=cells, seed=seed).T)   # [n, K]


@pytest.fixture(scope="module")
def small():
    A = O.tpfa_problem(inputs.small_3d(13, 11, 7, seed=21))
    orc = O.Oracle(A, coarse_max=64)
    return A, orc


def colerr(X, Y):
    return max(np.linalg.norm(X[:, k] - Y[:, k]) / np.linalg.norm(Y[:, k]) for k in range(Y.shape[1]))


@pytest.mark.parametrize("K", [1, 8, 13, 40, 64])
def test_block_cg_matches_oracle(small, K):
    A, orc = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64)
    Bh = rhs_block(A.n, K, seed=K)
    X, it, res, st = s.solve_block(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=300)
    s.close()
    ref = O.block_pcg(orc, Bh, op=O.BCO, tol=1e-10, maxit=300)
    assert st == 0 and ref["status"] == 0
    assert abs(it - ref["iters"]) <= 1
    assert colerr(X.cpu().numpy(), ref["X"]) <= 1e-8
    assert np.all(res < 1e-10)
    assert np.allclose(res, ref["res_hist"][-1], rtol=1e-3) or abs(it - ref["iters"]) == 1


def test_block_cg_one_column_is_pcg(small):
    A, orc = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64)
    b = inputs.random_vector(A.n, seed=2)
    bt = torch.tensor(b, device=DEV)
    X, it, res, st = s.solve_block(bt[:, None].contiguous(), tol=1e-10, maxit=300)
    x, its, sts, _ = s.solve(bt, tol=1e-10, maxit=300)
    s.close()
    assert st == 0 and sts == 0 and abs(it - its) <= 1
    x = x.cpu().numpy()
    assert np.linalg.norm(X.cpu().numpy()[:, 0] - x) <= 1e-8 * np.linalg.norm(x)


@pytest.mark.parametrize("which,op", [("amg", O.STILDE), ("ic0", O.B), ("bhat", O.BHAT)])
def test_block_cg_other_preconditioners(small, which, op):
    A, orc = small
    s = cpc.Solver(A.rowptr, A.col, A.val, precond=which, coarse_max=64)
    Bh = rhs_block(A.n, 16, seed=3)
    X, it, res, st = s.solve_block(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=600)
    s.close()
    ref = O.block_pcg(orc, Bh, op=op, tol=1e-10, maxit=600)
    assert st == 0 and ref["status"] == 0 and abs(it - ref["iters"]) <= 1
    assert colerr(X.cpu().numpy(), ref["X"]) <= 1e-8


@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16"])
def test_block_cg_mixed_precision(small, precision):
    A, orc = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, precision=precision, ic_order="colour")
    Bh = rhs_block(A.n, 24, seed=4)
    X, it, res, st = s.solve_block(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=300)
    s.close()
    ref = O.block_pcg(orc, Bh, op=O.BCO, tol=1e-10, maxit=300)
    assert st == 0 and abs(it - ref["iters"]) <= 2
    X = X.cpu().numpy()
    assert colerr(X, ref["X"]) <= 1e-5
    for k in (0, 23):
        assert np.linalg.norm(Bh[:, k] - A.matvec(X[:, k])) <= 1e-9 * np.linalg.norm(Bh[:, k])


def test_block_cg_breakdown_and_rejections(small):
    A, orc = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64)
    b = inputs.random_vector(A.n, seed=5)
    dup = torch.tensor(np.stack([b, b, 2.0 * b], axis=1), device=DEV)
    X, it, res, st = s.solve_block(dup, tol=1e-10, maxit=50, check=False)
    assert st == 4                                       # rank-deficient block: CG breakdown
    assert O.block_pcg(orc, dup.cpu().numpy(), op=O.BCO, tol=1e-10, maxit=50)["status"] == 4
    zero = torch.zeros(A.n, 2, dtype=torch.float64, device=DEV)
    zero[:, 0] = torch.tensor(b, device=DEV)
    with pytest.raises(cpc.CpcError):
        s.solve_block(zero, tol=1e-10, maxit=50)
    with pytest.raises(cpc.CpcError):
        s.solve_block(torch.zeros(A.n, 65, dtype=torch.float64, device=DEV), tol=1e-10, maxit=5)
    s.close()
    t = cpc.Solver(A.rowptr, A.col, A.val, precond="amg_ilu", coarse_max=64)
    with pytest.raises(cpc.CpcError):
        t.solve_block(torch.tensor(rhs_block(A.n, 4, seed=6), device=DEV), tol=1e-10, maxit=50)
    t.close()


def test_block_cg_full_size_64_rhs():
    p = inputs.correlated_3d()
    logk = torch.tensor(p.logk, device=DEV)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    s = cpc.Solver(rowptr, col, val, precision="fp32", ic_order="colour")
    Bh = rhs_block(p.n, 64, seed=5, cells=16)
    B = torch.tensor(Bh, device=DEV)
    X, it, res, st = s.solve_block(B, tol=1e-6, maxit=200)
    _, itb, stb = s.solve_batched(B, tol=1e-6, maxit=200)
    s.close()
    assert st == 0 and np.all(stb == 0)
    assert it <= int(np.max(itb))
    A = O.Csr(p.n, rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy())
    Xh = X.cpu().numpy()
    for k in range(0, 64, 7):
        assert np.linalg.norm(Bh[:, k] - A.matvec(Xh[:, k])) <= 1.0001e-6 * np.linalg.norm(Bh[:, k])
