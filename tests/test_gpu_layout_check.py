"""The layout checker (cpc_check_layouts) on every kind of handle the solver builds.

Each smoothed level contributes its colour-grouped smoother copy, P and R (3 layouts); the fine
natural copy and the IC(0) factor's two triangular-solve copies add 3.  A sound handle has no index
out of range, every row exactly once per layout, no two coupled rows in one Gauss-Seidel colour
group and every factor entry's row in a later triangular-solve level than its column.
"""
import pytest

import oracle as O
from paper_1205_6113_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_6113_gb300 import cpc  # noqa: E402

SMALL = lambda: O.tpfa_problem(inputs.small_3d(13, 11, 7, seed=21))      # noqa: E731
CASES = {
    "tpfa_colour_ic": (SMALL, dict(coarse_max=64, ic_order="colour")),
    "tpfa_natural_ic": (SMALL, dict(coarse_max=64)),
    "tpfa_natural_gs": (SMALL, dict(coarse_max=64, gs_order="natural")),
    "tpfa_fp32_bf16_autotune": (SMALL, dict(coarse_max=64, ic_order="colour", precision="fp32_bf16", autotune=True)),
    "lognormal_2d": (lambda: O.tpfa_problem(inputs.lognormal_2d()), dict(coarse_max=64, ic_order="colour")),
    "mhfem": (lambda: O.mhfem_problem(inputs.small_3d(6, 5, 4, seed=8))[0], dict(coarse_max=64)),
    "ragged_1d": (lambda: O.tpfa_problem(inputs.small_3d(33, 1, 1, seed=4)), dict(coarse_max=8)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_layouts_are_sound(name):
    make, kw = CASES[name]
    A = make()
    s = cpc.Solver(A.rowptr, A.col, A.val, **kw)
    c = s.check_layouts()
    nl = s.nlevels
    s.close()
    assert c["out_of_range"] == 0 and c["coverage"] == 0
    assert c["gs_races"] == 0 and c["triangular_races"] == 0
    assert c["layouts"] == 3 * (nl - 1) + 3


def test_layouts_full_size():
    p = inputs.correlated_3d()
    logk = torch.tensor(p.logk, device=torch.device("cuda:0"))
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    for kw in (dict(ic_order="colour"), dict(gs_order="natural")):
        s = cpc.Solver(rowptr, col, val, **kw)
        c = s.check_layouts()
        nl = s.nlevels
        s.close()
        assert c == dict(out_of_range=0, coverage=0, gs_races=0, triangular_races=0, layouts=3 * (nl - 1) + 3)
