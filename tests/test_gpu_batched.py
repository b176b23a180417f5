"""Batched PCG (K right-hand sides in lockstep, one CUDA graph) against single solves and the oracle.

Each column must reproduce the single-right-hand-side iteration: iteration counts within 1 and
solutions within 1e-8 of the single solve (same algorithm, different reduction layout), within
1e-8 of the oracle at tol 1e-10 (the FP64 parity gate) and within 1e-5 with the FP32
preconditioner.  The adjoint half must equal single solves of A lambda = G, G = X on the source
cells of each column.  At 128 x 128 x 64 with 64 right-hand sides every column must reach the
tolerance on its true FP64 residual.
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


def rhs_block(n, K, seed, cells=16):
    return np.ascontiguousarray(inputs.batch_rhs(n, K, cells_per_rhs=cells, seed=seed).T)   # [n, K]


@pytest.fixture(scope="module")
def small():
    p = inputs.small_3d(13, 11, 7, seed=21)
    A = O.tpfa_problem(p)
    return p, A


@pytest.mark.parametrize("K", [1, 7, 40, 64])
def test_batched_columns_match_single_solves(small, K):
    p, A = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour")
    Bh = rhs_block(A.n, K, seed=K, cells=4)
    X, it, st = s.solve_batched(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=500)
    X = X.cpu().numpy()
    assert np.all(st == 0)
    for k in range(K):
        xs, its, sts, _ = s.solve(torch.tensor(Bh[:, k].copy(), device=DEV), tol=1e-10, maxit=500)
        xs = xs.cpu().numpy()
        assert sts == 0 and abs(int(it[k]) - its) <= 1
        assert np.linalg.norm(X[:, k] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_batched_matches_oracle(small):
    p, A = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour")
    orc = O.Oracle(A, coarse_max=64, ic_colour_order=True)
    Bh = rhs_block(A.n, 32, seed=3, cells=4)
    X, it, st = s.solve_batched(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=500)
    X = X.cpu().numpy()
    for k in (0, 5, 31):
        ref = orc.pcg(Bh[:, k], op=O.BCO, tol=1e-10, maxit=500)
        assert abs(int(it[k]) - ref["iters"]) <= 2
        assert np.linalg.norm(X[:, k] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16"])
def test_batched_mixed_precision(small, precision):
    p, A = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour", precision=precision)
    orc = O.Oracle(A, coarse_max=64, ic_colour_order=True)
    Bh = rhs_block(A.n, 64, seed=4, cells=4)
    X, it, st = s.solve_batched(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=500)
    X = X.cpu().numpy()
    assert np.all(st == 0)
    for k in (0, 17, 63):
        ref = orc.pcg(Bh[:, k], op=O.BCO, tol=1e-10, maxit=500)
        assert np.linalg.norm(X[:, k] - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"])
        assert np.linalg.norm(Bh[:, k] - A.matvec(X[:, k])) <= 1e-9 * np.linalg.norm(Bh[:, k])


def test_batched_adjoint_in_one_graph(small):
    p, A = small
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour")
    Bh = rhs_block(A.n, 20, seed=5, cells=4)
    X, Lam, itf, ita = s.solve_batched_adjoint(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=500)
    X, Lam = X.cpu().numpy(), Lam.cpu().numpy()
    for k in (0, 9, 19):
        G = np.where(Bh[:, k] != 0, X[:, k], 0.0)
        ls, its, sts, _ = s.solve(torch.tensor(G, device=DEV), tol=1e-10, maxit=500)
        ls = ls.cpu().numpy()
        assert sts == 0 and abs(int(ita[k]) - its) <= 1
        assert np.linalg.norm(Lam[:, k] - ls) <= 1e-8 * np.linalg.norm(ls)
        xs, _, _, _ = s.solve(torch.tensor(Bh[:, k].copy(), device=DEV), tol=1e-10, maxit=500)
        assert np.linalg.norm(X[:, k] - xs.cpu().numpy()) <= 1e-8 * np.linalg.norm(xs.cpu().numpy())


def test_batched_full_size_64_rhs():
    p = inputs.correlated_3d()
    logk = torch.tensor(p.logk, device=DEV)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    s = cpc.Solver(rowptr, col, val, precision="fp32", ic_order="colour")
    Bh = rhs_block(p.n, 64, seed=5)
    B = torch.tensor(Bh, device=DEV)
    X, Lam, itf, ita = s.solve_batched_adjoint(B, tol=1e-6, maxit=500)
    A = O.Csr(p.n, rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy())
    Xh = X.cpu().numpy()
    for k in range(0, 64, 9):
        assert np.linalg.norm(Bh[:, k] - A.matvec(Xh[:, k])) <= 1.0001e-6 * np.linalg.norm(Bh[:, k])
    xs, its, sts, _ = s.solve(B[:, 3].contiguous(), tol=1e-6, maxit=500)
    assert sts == 0 and abs(int(itf[3]) - its) <= 1
    assert np.linalg.norm(Xh[:, 3] - xs.cpu().numpy()) <= 1e-6 * np.linalg.norm(xs.cpu().numpy())
    assert np.all(ita > 0)
