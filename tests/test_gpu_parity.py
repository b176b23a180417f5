"""GPU (CUDA, through the C ABI) against the CPU oracle, element by element.

Tolerances: structural choices (C/F splitting, colouring, sparsity patterns) must be
identical; the hierarchy's FP64 values (interpolation, Galerkin products) are identical to the
bit (same formulas, products added in the same order, no fused multiply-adds); operator
applications (where the GPU's fused multiply-adds round differently) to
1e-11; PCG solutions run to tol 1e-10 agree to 1e-8 relative with iteration counts
within +-2 (the parity gate), and every GPU solve reaches its tolerance on the
true FP64 residual.
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


def gpu_matrix(p):
    logk = torch.tensor(p.logk, device=DEV)
    return cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)


PROBLEMS = {
    "lognormal2d_64x64": lambda: inputs.lognormal_2d(),
    "small3d_13x11x7": lambda: inputs.small_3d(13, 11, 7, seed=21),
    "small3d_33x17x9": lambda: inputs.small_3d(33, 17, 9, seed=22),
    "channels_40x36x10": lambda: inputs.channel_facies(40, 36, 10, seed=23),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=64)
    # the GPU handle is built from the oracle's CSR (host) so that both start from the same bits
    solver = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64)
    return p, A, orc, solver


def test_tpfa_assembly_matches_oracle(case):
    p, A, _, _ = case
    rowptr, col, val = gpu_matrix(p)
    assert np.array_equal(rowptr.cpu().numpy(), A.rowptr)
    assert np.array_equal(col.cpu().numpy(), A.col)
    assert rel(val.cpu().numpy(), A.val) < 1e-14


def test_tpfa_full_size_1m():
    p = inputs.correlated_3d()
    A = O.tpfa_problem(p)
    rowptr, col, val = gpu_matrix(p)
    assert np.array_equal(rowptr.cpu().numpy(), A.rowptr)
    assert np.array_equal(col.cpu().numpy(), A.col)
    assert rel(val.cpu().numpy(), A.val) < 1e-14


def test_hierarchy_matches_oracle(case):
    _, A, orc, s = case
    assert s.nlevels == orc.nlevels
    for l in range(orc.nlevels):
        ptr, col, val = s.level_matrix(l)
        Ao = orc.level_A(l)
        assert np.array_equal(ptr, Ao.rowptr), l
        assert np.array_equal(col, Ao.col), l
        # both sides add the Galerkin products of an entry in the same order, without fused
        # multiply-adds: the coarse operators are identical to the bit
        assert np.array_equal(val, Ao.val), l
        if l + 1 < orc.nlevels:
            cf, colour = s.level_splitting(l)
            cfo, colo = orc.level_cf_colour(l)
            assert np.array_equal(cf, cfo), l
            assert np.array_equal(colour, colo), l
            pp, pc, pv = s.level_interp(l)
            Po = orc.level_P(l)
            assert np.array_equal(pp, Po.rowptr) and np.array_equal(pc, Po.col), l
            assert np.array_equal(pv, Po.val), l


def test_ic0_factor_matches_oracle(case):
    _, _, orc, s = case
    assert rel(s.ic0_values(), orc.ic0_values()) < 1e-13


def test_level_operators_match_oracle(case):
    _, _, orc, s = case
    for l in range(orc.nlevels):
        n = orc.level_sizes(l)["n"]
        x = inputs.random_vector(n, seed=100 + l)
        xd = torch.tensor(x, device=DEV)
        last = l == orc.nlevels - 1
        ops = [3] if last else [0, 1, 2, 4]
        if last and l == 0:
            ops = [0, 3, 4]
        for op in ops:
            y = s.level_apply(l, op, xd).cpu().numpy()
            assert rel(y, orc.level_apply(l, op, x)) < 1e-11, (l, op)


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE), ("ic0", O.B), ("bhat", O.BHAT),
                                      ("amg_ilu", O.AMG_ILU)])
def test_preconditioner_matches_oracle(case, which, op):
    _, A, orc, s = case
    r = inputs.random_vector(A.n, seed=7)
    z = s.apply(torch.tensor(r, device=DEV), which=which).cpu().numpy()
    assert rel(z, orc.apply(op, r)) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_tail_matches_oracle(case, precision):
    """The coarse end of the V-cycle as one cluster kernel (an option, off by default): same B_co
    as the oracle, and fewer launches per iteration than the launch-per-step path."""
    _, A, orc, s = case
    t = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, precision=precision, tail_nnz_max=1 << 40)
    assert t.solve_launches()[0] < s.solve_launches()[0]
    r = inputs.random_vector(A.n, seed=17)
    z = t.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < (1e-11 if precision == "fp64" else 1e-5)
    b = inputs.random_vector(A.n, seed=18)
    x, it, st, _ = t.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=500)
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=500)
    assert st == 0 and abs(it - ref["iters"]) <= 2
    x = x.cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= (1e-8 if precision == "fp64" else 1e-5) * np.linalg.norm(ref["x"])
    t.close()


def test_blocked_cholesky_on_a_large_coarsest_level():
    """A coarsest level of 329 rows: the dense inverse goes through 11 panels of the blocked
    Cholesky (diagonal block, triangular solve, trailing update), the last one ragged.  The
    coarsest solve and a whole B_co application must equal the oracle's dense Cholesky solve."""
    p = inputs.small_3d(40, 40, 16, seed=51)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=512)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=512)
    last = s.nlevels - 1
    assert s.level_info(last)["n"] == orc.level_sizes(orc.nlevels - 1)["n"] > 32 * 8
    nc = s.level_info(last)["n"]
    x = inputs.random_vector(nc, seed=52)
    y = s.level_apply(last, 3, torch.tensor(x, device=DEV)).cpu().numpy()
    assert rel(y, orc.level_apply(orc.nlevels - 1, 3, x)) < 1e-11
    r = inputs.random_vector(A.n, seed=53)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
    # the FP32 Cholesky inverse refined by Newton-Schulz steps reached FP64 accuracy and was kept
    method, res = s.coarse_inverse_info()
    assert method == 1 and res <= 1e-12
    s.close()


def test_coarse_inverse_falls_back_to_fp64_cholesky():
    """A nearly singular M-matrix (diagonal excess 1e-9 over the row sums, so the smallest
    eigenvalue is about 1e-9): kappa(A_c) is about 6e9 on its 1,533-row coarsest level, beyond what
    an FP32 factorisation resolves, so the Newton-Schulz steps from the FP32 inverse do not
    converge and setup forms the FP64 Cholesky inverse instead.  That coarsest solve must equal the
    oracle's dense Cholesky solve within kappa * eps, and a well-shifted matrix of the same pattern
    keeps the refined inverse."""
    for shift, method_want in [(1e-9, 0), (1e-2, 1)]:
        ptr, col, val = inputs.long_range_2d(nx=64, ny=64, radius=1.5, seed=61, shift=shift)
        A = O.Csr(len(ptr) - 1, ptr, col, val)
        orc = O.Oracle(A)
        s = cpc.Solver(ptr, col, val)
        assert s.nlevels == orc.nlevels == 2
        method, res = s.coarse_inverse_info()
        assert method == method_want, (shift, method, res)
        assert res < (1e-7 if method == 0 else 1e-12)
        nc = s.level_info(1)["n"]
        x = inputs.random_vector(nc, seed=62)
        y = s.level_apply(1, 3, torch.tensor(x, device=DEV)).cpu().numpy()
        assert rel(y, orc.level_apply(1, 3, x)) < (1e-6 if method == 0 else 1e-12)
        s.close()


def test_chained_cycles_read_fresh_data():
    """Two V-cycles back to back (S~, and B_co's steps (1)-(3)) in one chain of dependent launches:
    each kernel starts while its predecessor still writes, so a kernel that read the previous
    cycle's vectors through the read-only cache got values of the previous cycle (2.5e-5 off the
    oracle on this grid before the fix).  Repeated applications must be identical and equal the
    oracle's, and the solve must match it far inside the parity gate."""
    p = inputs.small_3d(40, 40, 16, seed=51)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=512)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=512)
    r = inputs.random_vector(A.n, seed=53)
    for which, op in [("amg", O.STILDE), ("bco", O.BCO)]:
        ref = orc.apply(op, r)
        zs = [s.apply(torch.tensor(r, device=DEV), which=which).cpu().numpy() for _ in range(4)]
        assert all(np.array_equal(zs[0], z) for z in zs[1:]), which
        assert rel(zs[0], ref) < 1e-11, which
    b = p.rhs()
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=300)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=300)
    s.close()
    assert status == 0 and abs(iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-12 * np.linalg.norm(ref["x"])


def test_autotuned_layout_matches_oracle(case):
    """Chunk heights picked by timing (autotune) change the layout and the lanes per row, not the
    method: B_co still equals the oracle's."""
    _, A, orc, _ = case
    t = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, autotune=True)
    for l in range(t.nlevels - 1):
        assert t.level_layout(l)["C"] in (4, 8, 16, 32)
    r = inputs.random_vector(A.n, seed=19)
    z = t.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
    t.close()


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE), ("ic0", O.B), ("bhat", O.BHAT),
                                      ("amg_ilu", O.AMG_ILU)])
def test_pcg_matches_oracle(case, which, op):
    p, A, orc, _ = case
    s = cpc.Solver(A.rowptr, A.col, A.val, precond=which, coarse_max=64)
    b = p.rhs()
    ref = orc.pcg(b, op=op, tol=1e-10, maxit=3000)
    x, iters, status, hist = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=3000)
    x = x.cpu().numpy()
    assert status == 0 and ref["status"] == 0
    assert abs(iters - ref["iters"]) <= 2
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b) <= 1e-9
    assert hist[0] == 1.0 and hist[-1] < 1e-10
    # the first residuals agree tightly; later ones drift with rounding (CG amplifies it), so
    # only their order of magnitude is compared
    n = min(len(hist), len(ref["res_hist"]))
    m = min(n, 8)
    assert np.allclose(hist[:m], ref["res_hist"][:m], rtol=1e-8, atol=1e-15)
    assert np.all(np.abs(np.log10(hist[:n] / ref["res_hist"][:n])) < 0.5)


def test_pcg_tol_1e6_iteration_counts(case):
    p, A, orc, s = case
    b = p.rhs()
    ref = orc.pcg(b, op=O.BCO, tol=1e-6, maxit=3000)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-6, maxit=3000)
    assert status == 0
    assert abs(iters - ref["iters"]) <= 2
    x = x.cpu().numpy()
    assert np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b) <= 1e-6 * 1.0001


def test_spmv_matches_oracle(case):
    _, A, orc, s = case
    x = inputs.random_vector(A.n, seed=3)
    y = s.spmv(torch.tensor(x, device=DEV)).cpu().numpy()
    assert rel(y, orc.apply(O.A, x)) < 1e-13


# ------------------------------------------------------------------------------------------------
# Edge cases
# ------------------------------------------------------------------------------------------------
def test_single_level_and_ragged_sizes():
    for shape in [(5, 3, 2), (7, 5, 3), (31, 1, 1), (33, 1, 1)]:
        p = inputs.small_3d(*shape, seed=4)
        A = O.tpfa_problem(p)
        orc = O.Oracle(A, coarse_max=40)
        s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=40)
        assert s.nlevels == orc.nlevels
        b = inputs.random_vector(A.n, seed=5)
        ref = orc.pcg(b, op=O.BCO, tol=1e-12, maxit=200)
        x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-12, maxit=200)
        assert status == 0 and abs(iters - ref["iters"]) <= 2
        assert np.linalg.norm(x.cpu().numpy() - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8


@pytest.mark.parametrize("shape", [(16, 12, 8), (64, 1, 1), (32, 24, 1)])
def test_even_width_grids(shape):
    """Fine grids of even width (3-D, a 1-D line, a 2-D plane) in the diagonal form with the
    red-black colour-ordered IC(0): applications, the fine sweep and PCG against the oracle."""
    p = inputs.small_3d(*shape, seed=31)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=16, ic_colour_order=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=16, ic_order="colour")
    assert s.level_layout(0)["ndiag"] > 0
    r = inputs.random_vector(A.n, seed=32)
    rt = torch.tensor(r, device=DEV)
    for which, op in [("bco", O.BCO), ("amg", O.STILDE), ("bhat", O.BHAT)]:
        assert rel(s.apply(rt, which=which).cpu().numpy(), orc.apply(op, r)) < 1e-11
    y = s.level_apply(0, 1, rt).cpu().numpy()
    assert rel(y, orc.level_apply(0, 1, r)) < 1e-12
    b = inputs.random_vector(A.n, seed=33)
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=300)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=300)
    assert status == 0 and abs(iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    c = s.check_layouts()
    assert c["out_of_range"] == 0 and c["gs_races"] == 0 and c["triangular_races"] == 0
    s.close()


def test_zero_rhs_and_maxit():
    p = inputs.small_3d(9, 8, 6, seed=1)
    A = O.tpfa_problem(p)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=20)
    x, iters, status, hist = s.solve(torch.zeros(A.n, dtype=torch.float64, device=DEV), tol=1e-6)
    assert status == 0 and iters == 0 and not x.cpu().numpy().any()
    x, iters, status, hist = s.solve(torch.tensor(p.rhs(), device=DEV), tol=1e-14, maxit=2)
    assert status == 3 and iters == 2 and len(hist) == 3


def test_nan_rhs_is_breakdown():
    p = inputs.small_3d(9, 8, 6, seed=1)
    A = O.tpfa_problem(p)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=20)
    b = p.rhs()
    b[5] = np.nan
    _, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-6)
    assert status == 4


def test_invalid_csr_and_breakdown_codes():
    with pytest.raises(cpc.CpcError) as e:
        cpc.Solver(np.array([0, 2, 3]), np.array([1, 0, 1]), np.array([1.0, 2.0, 1.0]))
    assert e.value.code == 1
    with pytest.raises(cpc.CpcError) as e:      # second IC(0) pivot is 1 - 4 < 0
        cpc.Solver(np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([1.0, 2.0, 2.0, 1.0]))
    assert e.value.code == 2
    with pytest.raises(cpc.CpcError) as e:      # structurally unsymmetric
        cpc.Solver(np.array([0, 2, 3, 4]), np.array([0, 1, 1, 2]), np.array([4.0, -1.0, 4.0, 4.0]), coarse_max=1)
    assert e.value.code == 1


# ------------------------------------------------------------------------------------------------
# Mixed precision: the preconditioner in FP32 (and BF16 coarse operators), outer PCG in FP64
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16"])
def test_mixed_precision_solution(case, precision):
    p, A, orc, _ = case
    s = cpc.Solver(A.rowptr, A.col, A.val, precision=precision, coarse_max=64)
    b = p.rhs()
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=3000)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=3000)
    assert status == 0
    x = x.cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-5
    assert np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b) <= 1e-9
    assert iters <= ref["iters"] + 5


def test_mixed_precision_preconditioner_close(case):
    _, A, orc, _ = case
    s = cpc.Solver(A.rowptr, A.col, A.val, precision="fp32", coarse_max=64)
    r = inputs.random_vector(A.n, seed=8)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-4


def test_colour_ordered_ic0(case):
    p, A, _, _ = case
    orc = O.Oracle(A, coarse_max=64, ic_colour_order=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour")
    assert rel(s.ic0_values(), orc.ic0_values()) < 1e-13
    r = inputs.random_vector(A.n, seed=9)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11


def test_host_buffers_solve(case):
    p, A, orc, s = case
    b = p.rhs()
    x = np.zeros(A.n)
    iters, status = s.solve_host(b, x, tol=1e-10, maxit=3000)
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=3000)
    assert status == 0 and abs(iters - ref["iters"]) <= 2
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8


@pytest.mark.parametrize("radius,longest", [(14.0, 256), (20.0, 512)])
def test_galerkin_products_on_long_rows(radius, longest):
    """Strong 5-point couplings keep many coarse points while weak couplings out to `radius` make
    the Galerkin rows long: with radius 14 the rows of A P and R (A P) reach about 300 entries (the
    hash product's largest tables), with radius 20 more than 512 (the sort-based fallback).  The
    hierarchy must still equal the oracle's to the bit, and a B_co application to 1e-11.  IC(0) is
    taken in the colour order (its rows of several hundred entries go to the warp-per-row
    elimination), which keeps the dependent chain of the factorisation short."""
    ptr, col, val = inputs.long_range_2d(radius=radius)
    A = O.Csr(len(ptr) - 1, ptr, col, val)
    orc = O.Oracle(A, coarse_max=256, ic_colour_order=True)
    s = cpc.Solver(ptr, col, val, coarse_max=256, ic_order="colour")
    assert rel(s.ic0_values(), orc.ic0_values()) < 1e-13
    assert s.nlevels == orc.nlevels >= 3
    assert np.diff(orc.level_A(1).rowptr).max() > longest
    for l in range(orc.nlevels):
        lp, lc, lv = s.level_matrix(l)
        Ao = orc.level_A(l)
        assert np.array_equal(lp, Ao.rowptr) and np.array_equal(lc, Ao.col), l
        assert np.array_equal(lv, Ao.val), l
        if l + 1 < orc.nlevels:
            cf, colour = s.level_splitting(l)
            cfo, colo = orc.level_cf_colour(l)
            assert np.array_equal(cf, cfo) and np.array_equal(colour, colo), l
    r = inputs.random_vector(A.n, seed=61)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    s.close()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11


def test_disconnected_matrix_hierarchy():
    """A block-diagonal matrix of three independent grids: every level's graph has several
    components, and the parity 2-colouring must root each at its own smallest index (the union-find
    hooks larger roots under smaller ones).  Splitting, colours and Galerkin values equal the
    oracle's to the bit; one B_co application to 1e-11."""
    blocks = [O.tpfa_problem(q) for q in (inputs.small_3d(13, 11, 7, seed=71), inputs.small_3d(9, 9, 5, seed=72),
                                          inputs.lognormal_2d(20, 20, seed=73))]
    ptrs, cols, vals, off = [np.zeros(1, np.int32)], [], [], 0
    for B in blocks:
        ptrs.append(B.rowptr[1:] + ptrs[-1][-1])
        cols.append(B.col + off)
        vals.append(B.val)
        off += B.n
    ptr = np.concatenate(ptrs).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32)
    val = np.concatenate(vals)
    A = O.Csr(off, ptr, col, val)
    orc = O.Oracle(A, coarse_max=64)
    s = cpc.Solver(ptr, col, val, coarse_max=64)
    assert s.nlevels == orc.nlevels >= 3
    for l in range(orc.nlevels):
        lp, lc, lv = s.level_matrix(l)
        Ao = orc.level_A(l)
        assert np.array_equal(lp, Ao.rowptr) and np.array_equal(lc, Ao.col) and np.array_equal(lv, Ao.val), l
        if l + 1 < orc.nlevels:
            cf, colour = s.level_splitting(l)
            cfo, colo = orc.level_cf_colour(l)
            assert np.array_equal(cf, cfo) and np.array_equal(colour, colo), l
    _, colour0 = s.level_splitting(0)
    starts = np.cumsum([0] + [B.n for B in blocks[:-1]])
    assert s.level_info(0)["ncolours"] == 2 and all(colour0[i] == 0 for i in starts)
    r = inputs.random_vector(A.n, seed=74)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    s.close()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
