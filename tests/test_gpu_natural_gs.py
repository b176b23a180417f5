"""Natural-order ("standard") Gauss-Seidel smoother on the GPU (gs_order="natural") against the oracle.

The GPU groups the rows of each smoothed level by their wavefront in the lower-triangular dependency
graph of A_l.  That grouping is integer data and must equal, row for row, the wavefronts computed
here from the oracle's A_l (w(i) = 1 + max w(j) over coupled j < i, 0 when there is none).  Sweeps,
V-cycles and every preconditioner must match the oracle built with gs_natural=True to 1e-11; PCG
solves at tol 1e-10 agree to 1e-8 with equal iteration counts (the FP64 parity gate), 1e-5 with the
FP32 preconditioner.  The natural order needs natural-order IC(0) and no cluster kernel; other
combinations are rejected at setup.
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


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def wavefronts(A):
    """Level of every row in the lower-triangular dependency graph of A (natural order)."""
    w = np.zeros(A.n, np.int64)
    for i in range(A.n):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        lo = c[c < i]
        w[i] = 1 + w[lo].max() if lo.size else 0
    return w


PROBLEMS = {
    "correlated_13x11x7": lambda: O.tpfa_problem(inputs.small_3d(13, 11, 7, seed=21)),
    "lognormal_2d": lambda: O.tpfa_problem(inputs.lognormal_2d()),
    "mhfem_6x5x4": lambda: O.mhfem_problem(inputs.small_3d(6, 5, 4, seed=8))[0],
}


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def case(request):
    A = PROBLEMS[request.param]()
    orc = O.Oracle(A, coarse_max=64, gs_natural=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, gs_order="natural")
    yield A, orc, s
    s.close()


def test_wavefront_grouping_is_exact(case):
    A, orc, s = case
    assert s.nlevels == orc.nlevels >= 2
    for l in range(orc.nlevels - 1):
        w = wavefronts(orc.level_A(l))
        _, colour = s.level_splitting(l)
        assert np.array_equal(colour, w)
        assert s.level_info(l)["ncolours"] == int(w.max()) + 1


def test_sweeps_and_cycles_match_oracle(case):
    A, orc, s = case
    for l in range(orc.nlevels - 1):
        n = orc.level_sizes(l)["n"]
        x = inputs.random_vector(n, seed=30 + l)
        xt = torch.tensor(x, device=DEV)
        for op in (1, 2, 4):                           # forward sweep, backward sweep, V-cycle
            y = s.level_apply(l, op, xt).cpu().numpy()
            assert rel(y, orc.level_apply(l, op, x)) < 1e-11, (l, op)


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE), ("bhat", O.BHAT),
                                      ("amg_ilu", O.AMG_ILU)])
def test_preconditioners_match_oracle(case, which, op):
    A, orc, s = case
    r = inputs.random_vector(A.n, seed=7)
    z = s.apply(torch.tensor(r, device=DEV), which=which).cpu().numpy()
    assert rel(z, orc.apply(op, r)) < 1e-11


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE)])
def test_pcg_matches_oracle(case, which, op):
    A, orc, s = case
    b = inputs.random_vector(A.n, seed=9)
    ref = orc.pcg(b, op=op, tol=1e-10, maxit=500)
    t = cpc.Solver(A.rowptr, A.col, A.val, precond=which, coarse_max=64, gs_order="natural")
    x, iters, status, _ = t.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=500)
    t.close()
    assert status == 0 and abs(iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


def test_fp32_preconditioner_natural_order():
    A = PROBLEMS["correlated_13x11x7"]()
    orc = O.Oracle(A, coarse_max=64, gs_natural=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, gs_order="natural", precision="fp32")
    b = inputs.random_vector(A.n, seed=10)
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=500)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=500)
    s.close()
    assert status == 0 and abs(iters - ref["iters"]) <= 2
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"])


def test_batched_natural_order_matches_single_solves():
    A = PROBLEMS["correlated_13x11x7"]()
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, gs_order="natural")
    Bh = np.ascontiguousarray(inputs.batch_rhs(A.n, 8, cells_per_rhs=4, seed=12).T)
    X, it, st = s.solve_batched(torch.tensor(Bh, device=DEV), tol=1e-10, maxit=500)
    X = X.cpu().numpy()
    assert np.all(st == 0)
    for k in (0, 7):
        xs, its, sts, _ = s.solve(torch.tensor(Bh[:, k].copy(), device=DEV), tol=1e-10, maxit=500)
        xs = xs.cpu().numpy()
        assert sts == 0 and abs(int(it[k]) - its) <= 1
        assert np.linalg.norm(X[:, k] - xs) <= 1e-8 * np.linalg.norm(xs)
    s.close()


def test_rejected_combinations():
    A = PROBLEMS["correlated_13x11x7"]()
    with pytest.raises(cpc.CpcError):
        cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, gs_order="natural", ic_order="colour")
    with pytest.raises(cpc.CpcError):
        cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, gs_order="natural", tail_nnz_max=1 << 20)


def test_full_size_natural_order_iterations():
    """128 x 128 x 64 correlated field, tol 1e-6: the GPU takes the oracle's iteration count with
    the natural-order smoother, and the fine level has nx + ny + nz - 2 wavefronts."""
    p = inputs.correlated_3d()
    A = O.tpfa_problem(p)
    b = p.rhs()
    orc = O.Oracle(A, gs_natural=True)
    ref = orc.pcg(b, op=O.BCO, tol=1e-6, maxit=200)
    s = cpc.Solver(A.rowptr, A.col, A.val, gs_order="natural")
    assert s.level_info(0)["ncolours"] == p.nx + p.ny + p.nz - 2
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-6, maxit=200)
    s.close()
    assert status == 0 and abs(iters - ref["iters"]) <= 1
    x = x.cpu().numpy()
    assert np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b) <= 1e-6 * 1.0001
    assert np.linalg.norm(x - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
