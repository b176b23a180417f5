"""The GPU solver on the mixed-hybrid (p, lambda) system of Section 4 / Section 5 Eq. alge_sys.

These matrices exercise paths that the two-point-flux workloads never reach:
- cell and face unknowns mixed in one system;
- positive off-diagonal couplings;
- a fine level that is not bipartite (peel-round colouring, no red-black fusion of B_co step (2));
- more than 8 distinct column offsets (SELL instead of the diagonal form).

Hierarchy, colourings and preconditioners must equal the oracle's, and the PCG runs must reach
the oracle's iterates.  AMG(ILU(0)) may lose positive definiteness here (Section 5): each side
then either converges or reports a CG breakdown, and where both converge they agree.
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

PROBLEMS = {
    "correlated_9x8x5": lambda: inputs.small_3d(9, 8, 5, seed=41),
    "channels_24x20x8": lambda: inputs.channel_facies(24, 20, 8, seed=43),
}


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    if not p.wells:
        p.wells = inputs.nine_wells(p)
    A, b = O.mhfem_problem(p)
    orc = O.Oracle(A, coarse_max=64)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64)
    yield p, A, b, orc, s
    s.close()


def test_hierarchy_and_colouring_match(case):
    _, A, _, orc, s = case
    assert s.nlevels == orc.nlevels
    assert s.level_info(0)["ncolours"] > 2                 # not bipartite
    assert s.level_layout(0)["ndiag"] == 0                  # too many offsets for the diagonal form
    for l in range(s.nlevels - 1):
        cf, colour = s.level_splitting(l)
        cfo, colo = orc.level_cf_colour(l)
        assert np.array_equal(cf, cfo) and np.array_equal(colour, colo), l


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE), ("ic0", O.B), ("bhat", O.BHAT),
                                      ("amg_ilu", O.AMG_ILU)])
def test_preconditioners_match(case, which, op):
    _, A, _, orc, s = case
    r = inputs.random_vector(A.n, seed=3)
    z = s.apply(torch.tensor(r, device=DEV), which=which).cpu().numpy()
    assert rel(z, orc.apply(op, r)) < 1e-11


@pytest.mark.parametrize("which,op", [("bco", O.BCO), ("amg", O.STILDE), ("bhat", O.BHAT)])
def test_pcg_matches(case, which, op):
    _, A, b, orc, _ = case
    s = cpc.Solver(A.rowptr, A.col, A.val, precond=which, coarse_max=64)
    x, it, st, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=1000)
    ref = orc.pcg(b, op=op, tol=1e-10, maxit=1000)
    assert st == 0 and ref["status"] == 0
    assert abs(it - ref["iters"]) <= 2
    x = x.cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    s.close()


def test_amg_ilu_breakdown_or_agreement(case):
    _, A, b, orc, _ = case
    s = cpc.Solver(A.rowptr, A.col, A.val, precond="amg_ilu", coarse_max=64)
    x, it, st, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-10, maxit=1000)
    ref = orc.pcg(b, op=O.AMG_ILU, tol=1e-10, maxit=1000)
    assert st in (0, 4) and ref["status"] in (0, 4)          # 4: CG breakdown (CPC_EBREAKDOWN)
    if st == 0 and ref["status"] == 0:
        assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    s.close()


def test_colour_ordered_ic0_on_non_bipartite_fine_level(case):
    _, A, b, _, _ = case
    orc = O.Oracle(A, coarse_max=64, ic_colour_order=True)
    s = cpc.Solver(A.rowptr, A.col, A.val, coarse_max=64, ic_order="colour")
    assert rel(s.ic0_values(), orc.ic0_values()) < 1e-13
    r = inputs.random_vector(A.n, seed=5)
    z = s.apply(torch.tensor(r, device=DEV), which="bco").cpu().numpy()
    assert rel(z, orc.apply(O.BCO, r)) < 1e-11
    s.close()


# ------------------------------------------------------------------------------------------------
# Device assembly (cpc_mhfem_assemble) against the oracle's assembly
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape,mask", [((9, 8, 5), inputs.FACE_X0), ((4, 3, 2), 0), ((3, 3, 3), 63),
                                        ((1, 1, 1), 3), ((7, 1, 4), 1 | 8 | 32), ((16, 12, 6), 4 | 16)])
def test_device_assembly_matches_oracle(shape, mask):
    nx, ny, nz = shape
    logk = 1.5 * inputs.random_vector(nx * ny * nz, seed=7)
    A = O.mhfem(nx, ny, nz, logk, 0.1, mask)
    rowptr, col, val = cpc.mhfem_assemble(nx, ny, nz, torch.tensor(logk, device=DEV), 0.1, mask)
    assert np.array_equal(rowptr.cpu().numpy(), A.rowptr)
    assert np.array_equal(col.cpu().numpy(), A.col)
    assert rel(val.cpu().numpy(), A.val) < 1e-14


def test_device_assembled_system_solves_like_oracle():
    """64 x 64 x 32 channel problem (530,432 unknowns) assembled on the device: B_co PCG takes the
    oracle's iteration count at tol 1e-6 and meets the tolerance on the true residual."""
    p = inputs.channel_facies(64, 64, 32, seed=45)
    p.wells = inputs.nine_wells(p)
    A, b = O.mhfem_problem(p)
    rowptr, col, val = cpc.mhfem_assemble(p.nx, p.ny, p.nz, torch.tensor(p.logk, device=DEV), p.kz_ratio,
                                          p.dirichlet)
    assert np.array_equal(col.cpu().numpy(), A.col)
    orc = O.Oracle(A)
    ref = orc.pcg(b, op=O.BCO, tol=1e-6, maxit=300)
    s = cpc.Solver(rowptr, col, val)
    x, iters, status, _ = s.solve(torch.tensor(b, device=DEV), tol=1e-6, maxit=300)
    s.close()
    assert status == 0 and abs(iters - ref["iters"]) <= 1
    x = x.cpu().numpy()
    assert np.linalg.norm(b - A.matvec(x)) <= 1.0001e-6 * np.linalg.norm(b)
