"""Seeded synthetic inputs for the pressure-system workloads.

This module holds no arithmetic of the solver method: it only draws
permeability fields, well locations and well rates, and places the rates in a
right-hand-side vector.  Both the CUDA path and the CPU oracle consume what it
returns, so it imports neither of them.

The paper's matrices come from private reservoir models (Section 5, Table 1);
these generators stand in for them with structured grids whose permeability is
heterogeneous in the ways the paper describes (large jumps, strong anisotropy).

Cell (i, j, k) of an nx x ny x nz grid has the natural index
``i + nx * (j + ny * k)``; arrays are returned flat in that order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Dirichlet face bits (p = 0 on the face, half-cell transmissibility).
FACE_X0, FACE_X1, FACE_Y0, FACE_Y1, FACE_Z0, FACE_Z1 = 1, 2, 4, 8, 16, 32


@dataclass
class Problem:
    """A structured-grid pressure problem: log-permeability, anisotropy, boundary and wells."""

    name: str
    nx: int
    ny: int
    nz: int
    logk: np.ndarray            # float64[n], natural log of the horizontal permeability
    kz_ratio: float             # k_z = kz_ratio * k
    dirichlet: int              # bitmask of FACE_* faces held at p = 0
    wells: list = field(default_factory=list)   # [(cell_index, rate)]

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def idx(self, i: int, j: int, k: int = 0) -> int:
        return i + self.nx * (j + self.ny * k)

    def rhs(self) -> np.ndarray:
        """Right-hand side: each well's rate added at its cell (p_D = 0 adds nothing)."""
        return rhs_from_wells(self.n, self.wells)


def rhs_from_wells(n: int, wells) -> np.ndarray:
    b = np.zeros(n, dtype=np.float64)
    for c, q in wells:
        b[int(c)] += float(q)
    return b


def gaussian_field(shape, corr_len: float, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Correlated Gaussian field with covariance sigma^2 * exp(-(r/corr_len)^2).

    White noise convolved (periodically, by FFT) with exp(-2 r^2 / corr_len^2)
    has a covariance proportional to exp(-r^2 / corr_len^2); the result is then
    standardised to mean 0, standard deviation 1 and scaled by sigma.
    ``shape`` is (nz, ny, nx) so that the flattened array is in natural order.
    """
    noise = rng.standard_normal(shape)
    grids = np.meshgrid(*[np.minimum(np.arange(s), s - np.arange(s)) for s in shape], indexing="ij")
    r2 = sum(g.astype(np.float64) ** 2 for g in grids)
    kern = np.exp(-2.0 * r2 / (corr_len * corr_len))
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.fft.fftn(kern)))
    f = (f - f.mean()) / f.std()
    return (sigma * f).reshape(-1)


def lognormal_2d(nx=64, ny=64, seed=1) -> Problem:
    """64 x 64 five-point problem: iid log k ~ N(0, 1), p = 0 on the left edge, source +1 at (48, 48)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logk = rng.standard_normal(nx * ny)
    p = Problem("lognormal2d_%dx%d" % (nx, ny), nx, ny, 1, logk, 1.0, FACE_X0)
    p.wells = [(p.idx(min(48, nx - 1), min(48, ny - 1)), 1.0)]
    return p


def five_spot(p: Problem, kw: int) -> list:
    """Injector +1 at the centre, four producers -0.25 at the quarter points, all at layer kw."""
    nx, ny = p.nx, p.ny
    qx, qy = nx // 8, ny // 8
    return [(p.idx(nx // 2, ny // 2, kw), 1.0),
            (p.idx(qx, qy, kw), -0.25), (p.idx(qx, ny - qy, kw), -0.25),
            (p.idx(nx - qx, qy, kw), -0.25), (p.idx(nx - qx, ny - qy, kw), -0.25)]


def correlated_3d(nx=128, ny=128, nz=64, seed=2, sigma=2.0, corr_len=8.0, kz_ratio=0.1) -> Problem:
    """3-D seven-point problem: Gaussian-correlated lognormal k, k_z = 0.1 k, five-spot wells, p = 0 on x = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logk = gaussian_field((nz, ny, nx), corr_len, sigma, rng)
    p = Problem("correlated3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, logk, kz_ratio, FACE_X0)
    p.wells = five_spot(p, nz // 2)
    return p


def channel_facies(nx=256, ny=256, nz=128, seed=4, ntg=0.25, kz_ratio=0.01,
                   k_hi=1000.0, k_lo=1.0, width=12, thickness=6) -> Problem:
    """Binary facies: sinuous high-permeability channels over a low-permeability background.

    Channel centrelines follow y = y0 + a sin(2 pi x / lam + phi) with a ~ U[8, 32],
    lam ~ U[64, 256]; each channel is ``width`` cells wide and ``thickness`` layers
    thick.  Channels are added until the net-to-gross reaches ``ntg``.  Nine vertical
    wells on a 3 x 3 pattern with alternating signs (sum |q| = 9, each rate split
    evenly over the layers); p = 0 on x = 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    facies = np.zeros((nz, ny, nx), dtype=bool)
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    half = width / 2.0
    while facies.mean() < ntg:
        a = rng.uniform(8.0, 32.0)
        lam = rng.uniform(64.0, 256.0)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        y0 = rng.uniform(0.0, ny)
        z0 = int(rng.integers(0, max(1, nz - thickness + 1)))
        yc = y0 + a * np.sin(2.0 * np.pi * xs / lam + phi)            # [nx]
        band = np.abs(ys[:, None] - yc[None, :]) < half                # [ny, nx]
        facies[z0:z0 + thickness] |= band[None, :, :]
    logk = np.where(facies, np.log(k_hi), np.log(k_lo)).reshape(-1).astype(np.float64)
    p = Problem("channels3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, logk, kz_ratio, FACE_X0)
    p.wells = nine_wells(p)
    return p


def nine_wells(p: Problem) -> list:
    """3 x 3 vertical wells at the quarter points, sign (-1)^(a+b), |q| = 1 each, split over nz."""
    wells = []
    for a in range(3):
        for b in range(3):
            i = (a + 1) * p.nx // 4
            j = (b + 1) * p.ny // 4
            q = (1.0 if (a + b) % 2 == 0 else -1.0) / p.nz
            wells += [(p.idx(i, j, k), q) for k in range(p.nz)]
    return wells


def well_columns(p: Problem) -> list:
    """Cell indices of each of the nine vertical wells (for the well-pressure misfit)."""
    cols = []
    for a in range(3):
        for b in range(3):
            i = (a + 1) * p.nx // 4
            j = (b + 1) * p.ny // 4
            cols.append([p.idx(i, j, k) for k in range(p.nz)])
    return cols


def perturbed_logk(p: Problem, seed=40, scale=0.5) -> np.ndarray:
    """log k plus iid N(0, scale^2) noise: the field that produces the observed well pressures."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return p.logk + scale * rng.standard_normal(p.n)


def batch_rhs(n: int, nrhs=64, cells_per_rhs=16, seed=5) -> np.ndarray:
    """nrhs right-hand sides, each with rates U[-1, 1] at ``cells_per_rhs`` random cells; shape [nrhs, n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    B = np.zeros((nrhs, n), dtype=np.float64)
    for r in range(nrhs):
        cells = rng.choice(n, size=cells_per_rhs, replace=False)
        B[r, cells] = rng.uniform(-1.0, 1.0, size=cells_per_rhs)
    return B


def small_3d(nx, ny, nz, seed=7, sigma=1.5, corr_len=3.0, kz_ratio=0.1, dirichlet=FACE_X0) -> Problem:
    """Small correlated 3-D problem (ragged sizes) for parity tests; wells as a five-spot at mid depth."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logk = gaussian_field((nz, ny, nx), corr_len, sigma, rng)
    p = Problem("small3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, logk, kz_ratio, dirichlet)
    p.wells = five_spot(p, nz // 2)
    return p


def long_range_2d(nx=64, ny=64, radius=14.0, seed=60, shift=1e-2):
    """CSR (rowptr, col, val) of an SPD M-matrix on an nx x ny grid: strong couplings to the four
    grid neighbours (weights 0.5..1.5) and weak ones (weights 0.5e-3..1.5e-3) to every other point
    within Euclidean distance ``radius``; diagonal = the sum of the row's couplings + ``shift``.  The
    strong part keeps many coarse points, the weak part makes the Galerkin rows long; a tiny shift
    makes the matrix nearly singular (smallest eigenvalue about ``shift``, the constant vector)."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    r = int(np.floor(radius))
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()
    for dy in range(0, r + 1):
        for dx in range(-r, r + 1):
            if dy == 0 and dx <= 0:
                continue                               # each unordered pair once
            if dx * dx + dy * dy > radius * radius:
                continue
            ok = (ii + dx >= 0) & (ii + dx < nx) & (jj + dy < ny)
            a = (ii + nx * jj)[ok]
            b = a + dx + nx * dy
            strong = (dx, dy) in ((1, 0), (0, 1))
            w = (0.5 + rng.random(a.size)) * (1.0 if strong else 1e-3)
            rows += [a, b]
            cols += [b, a]
            vals += [-w, -w]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    diag = np.zeros(n)
    np.add.at(diag, rows, -vals)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag + shift])
    order = np.lexsort((cols, rows))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return rowptr, cols[order].astype(np.int32), vals[order].astype(np.float64)


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


# Workloads by name: the plain 2-D case, the 1M-unknown correlated case (FP64 and
# mixed precision share it), the 8.4M-unknown channel case and the batched case.
def workload(name: str) -> Problem:
    if name == "lognormal2d_64x64":
        return lognormal_2d()
    if name == "correlated3d_128x128x64":
        return correlated_3d()
    if name == "channels3d_256x256x128":
        return channel_facies()
    raise KeyError(name)
