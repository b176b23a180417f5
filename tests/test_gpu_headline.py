"""Parity at full size on the benchmark configuration: the 128 x 128 x 64 correlated-lognormal
two-point-flux matrix (1,048,576 unknowns), B_co with the red-black IC(0) ordering and the
multicolour Gauss-Seidel V-cycle, exactly the handle that bench.py times.

At this size the hierarchy has five levels with 12 to 24 colours on the coarse levels, so the
wide-batch colour-step kernels, the one-pass black-row B_co step (2) and the refined inverse of
the 1,823-row coarsest level (FP32 blocked Cholesky, then Newton-Schulz steps) all run.  The oracle (single-threaded FP64) needs a few seconds for its
setup and about half a second per preconditioner application here.

Gates: structure identical (splitting, colouring, level patterns), level values to 1e-12,
one B_co application to 1e-11, PCG run to 1e-10 within +-2 iterations of the oracle with
||x - x_oracle|| / ||x_oracle|| <= 1e-8 (FP64 preconditioner), or within -2/+5 iterations and
1e-5 (FP32 preconditioner: its rounding costs iterations near 1e-10), and the 1e-6 benchmark
solve within +-2 iterations with a true residual below 1e-6.
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
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def full():
    p = inputs.correlated_3d()
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, ic_colour_order=True)
    logk = torch.tensor(p.logk, device=DEV)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    assert np.array_equal(rowptr.cpu().numpy(), A.rowptr) and np.array_equal(col.cpu().numpy(), A.col)
    s = cpc.Solver(rowptr, col, val, precond="bco", precision="fp64", ic_order="colour")
    yield p, A, orc, s, (rowptr, col, val)
    s.close()


@pytest.fixture(scope="module")
def reference_solution(full):
    p, A, orc, _, _ = full
    b = p.rhs()
    return b, orc.pcg(b, op=O.BCO, tol=1e-10, maxit=200)


def test_full_size_hierarchy_matches_oracle(full):
    _, _, orc, s, _ = full
    assert s.nlevels == orc.nlevels >= 5
    for l in range(orc.nlevels):
        ptr, col, val = s.level_matrix(l)
        Ao = orc.level_A(l)
        assert np.array_equal(ptr, Ao.rowptr) and np.array_equal(col, Ao.col), l
        assert rel(val, Ao.val) < 1e-12, l
        if l + 1 < orc.nlevels:
            cf, colour = s.level_splitting(l)
            cfo, colo = orc.level_cf_colour(l)
            assert np.array_equal(cf, cfo), l
            assert np.array_equal(colour, colo), l
    assert s.level_info(0)["ncolours"] == 2
    assert max(s.level_info(l)["ncolours"] for l in range(1, s.nlevels - 1)) >= 12
    # the coarsest inverse: FP32 Cholesky refined to FP64 accuracy, and its solve equals the
    # oracle's dense Cholesky solve
    method, res = s.coarse_inverse_info()
    assert method == 1 and res <= 1e-12
    last = orc.nlevels - 1
    x = inputs.random_vector(orc.level_sizes(last)["n"], seed=70)
    y = s.level_apply(last, 3, torch.tensor(x, device=DEV)).cpu().numpy()
    assert rel(y, orc.level_apply(last, 3, x)) < 1e-11


def test_full_size_bco_application_matches_oracle(full):
    _, A, orc, s, _ = full
    r = inputs.random_vector(A.n, seed=71)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
    z2 = s.apply_Bcom(torch.tensor(r, device=DEV)).cpu().numpy()
    assert np.array_equal(z, z2)


def test_full_size_fp64_solve_matches_oracle(full, reference_solution):
    _, A, _, s, _ = full
    b, ref = reference_solution
    assert ref["status"] == 0
    x, iters, status, hist = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=200)
    x = x.cpu().numpy()
    assert status == 0 and abs(iters - ref["iters"]) <= 2
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-9 * np.linalg.norm(b)
    assert np.allclose(hist[:6], ref["res_hist"][:6], rtol=1e-8, atol=1e-15)


@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16"])
def test_full_size_mixed_precision_solve_matches_oracle(full, reference_solution, precision):
    _, A, _, _, csr = full
    b, ref = reference_solution
    s = cpc.Solver(*csr, precond="bco", precision=precision, ic_order="colour")
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=200)
    s.close()
    x = x.cpu().numpy()
    assert status == 0 and ref["iters"] - 2 <= iters <= ref["iters"] + 5
    assert np.linalg.norm(x - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-9 * np.linalg.norm(b)


def test_full_size_benchmark_tolerance(full):
    """The timed solve itself (tol 1e-6): the oracle's iteration count within +-2 and a true FP64
    residual below the tolerance, for B_co and for AMG alone (S~, two V-cycles)."""
    p, A, orc, s, csr = full
    b = p.rhs()
    for which, op, handle in [("bco", O.BCO, s), ("amg", O.STILDE, None)]:
        ref = orc.pcg(b, op=op, tol=1e-6, maxit=200)
        h = handle or cpc.Solver(*csr, precond=which, precision="fp64", ic_order="colour")
        x, iters, status, _ = h.solve(torch.tensor(b, device=DEV), tol=1e-6, maxit=200)
        if handle is None:
            h.close()
        x = x.cpu().numpy()
        assert status == 0 and abs(iters - ref["iters"]) <= 2, which
        assert np.linalg.norm(b - A.matvec(x)) <= 1e-6 * np.linalg.norm(b), which
        assert np.linalg.norm(x - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"]), which


def test_channel_field_full_size_parity():
    """The 256 x 256 x 128 channel field (8,388,608 unknowns, 1000:1 facies contrast, k_z / k =
    0.01), the largest workload: the GPU hierarchy built from the oracle's matrix equals the
    oracle's (splitting, colouring, patterns and values to the bit), and one B_co application
    equals the oracle's to 1e-11.  The oracle's setup here takes about half a minute."""
    p = inputs.channel_facies()
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, ic_colour_order=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, precond="bco", precision="fp64", ic_order="colour")
    assert s.nlevels == orc.nlevels >= 5
    for l in range(orc.nlevels):
        ptr, col, val = s.level_matrix(l)
        Ao = orc.level_A(l)
        assert np.array_equal(ptr, Ao.rowptr) and np.array_equal(col, Ao.col), l
        assert np.array_equal(val, Ao.val), l
        if l + 1 < orc.nlevels:
            cf, colour = s.level_splitting(l)
            cfo, colo = orc.level_cf_colour(l)
            assert np.array_equal(cf, cfo) and np.array_equal(colour, colo), l
    r = inputs.random_vector(A.n, seed=72)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    s.close()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
