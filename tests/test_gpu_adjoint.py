"""Differentiable solve: adjoint gradient of a well-pressure misfit with respect to log k.

J = 1/2 sum_w (mean_w p - d_w)^2, A(log k) p = q, d from a solve on a perturbed field.
Checks: the gradient kernel against the oracle's (same lambda, p; 1e-13), the autograd gradient
against the oracle's adjoint gradient on a medium channel problem (solves at tol 1e-12; 1e-8), and
against central finite differences (h = 1e-4 in log k) on 20 random cells of the 256 x 256 x 128
channel problem (|g_fd - g| <= 1e-4 |g| + 1e-6 max|g|, the floor set by the solve tolerance).
"""
import numpy as np
import pytest

import oracle as O
from paper_1205_6113_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_6113_gb300 import adjoint, cpc  # noqa: E402

DEV = torch.device("cuda:0")


def grid_of(p):
    return adjoint.Grid(p.nx, p.ny, p.nz, p.kz_ratio, p.dirichlet)


@pytest.mark.parametrize("make", [lambda: inputs.small_3d(13, 11, 7, seed=3),
                                  lambda: inputs.small_3d(9, 8, 5, seed=4, dirichlet=inputs.FACE_X0 | inputs.FACE_Y1),
                                  lambda: inputs.channel_facies(40, 36, 10, seed=23)])
def test_gradient_kernel_matches_oracle(make):
    p = make()
    lam = inputs.random_vector(p.n, seed=1)
    x = inputs.random_vector(p.n, seed=2)
    ref = O.tpfa_gradient(p.nx, p.ny, p.nz, p.logk, p.kz_ratio, p.dirichlet, lam, x)
    g = cpc.tpfa_gradient(p.nx, p.ny, p.nz, torch.tensor(p.logk, device=DEV), p.kz_ratio, p.dirichlet,
                          torch.tensor(lam, device=DEV), torch.tensor(x, device=DEV)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))


def misfit_setup(p, seed=40):
    wells = inputs.well_columns(p)
    cells = torch.tensor(wells, device=DEV, dtype=torch.int64)
    q = torch.tensor(p.rhs(), device=DEV)
    grid = grid_of(p)
    with torch.no_grad():
        p_obs = adjoint.pressure(torch.tensor(inputs.perturbed_logk(p, seed=seed), device=DEV), q, grid, tol=1e-12)
        d = adjoint.well_pressures(p_obs, cells)
    return wells, cells, q, grid, d


def misfit(logk, q, grid, cells, d, tol=1e-12):
    p = adjoint.pressure(logk, q, grid, tol=tol)
    r = adjoint.well_pressures(p, cells) - d
    return 0.5 * (r * r).sum()


def test_autograd_gradient_matches_oracle_adjoint():
    p = inputs.channel_facies(48, 40, 16, seed=9)
    p.wells = inputs.nine_wells(p)
    wells, cells, q, grid, d = misfit_setup(p)
    logk = torch.tensor(p.logk, device=DEV, requires_grad=True)
    J = misfit(logk, q, grid, cells, d)
    J.backward()
    A = O.tpfa_problem(p)
    j_ref, g_ref = O.misfit_gradient(A, p, p.logk, wells, d.cpu().numpy())
    assert abs(J.item() - j_ref) <= 1e-8 * abs(j_ref)
    g = logk.grad.cpu().numpy()
    assert np.max(np.abs(g - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))


@pytest.mark.slow
def test_central_differences_on_full_channel_problem():
    """The 256 x 256 x 128 channelised case: 20 random cells, central differences h = 1e-4."""
    p = inputs.channel_facies()
    wells, cells, q, grid, d = misfit_setup(p)
    logk0 = torch.tensor(p.logk, device=DEV)
    logk = logk0.clone().requires_grad_(True)
    J = misfit(logk, q, grid, cells, d)
    J.backward()
    g = logk.grad.cpu().numpy()
    gmax = np.max(np.abs(g))
    rng = np.random.Generator(np.random.PCG64(20))
    h = 1e-4
    for c in rng.choice(p.n, size=20, replace=False):
        e = torch.zeros_like(logk0)
        e[c] = h
        with torch.no_grad():
            jp = misfit(logk0 + e, q, grid, cells, d).item()
            jm = misfit(logk0 - e, q, grid, cells, d).item()
        fd = (jp - jm) / (2 * h)
        assert abs(fd - g[c]) <= 1e-4 * abs(g[c]) + 1e-6 * gmax, (c, fd, g[c])
