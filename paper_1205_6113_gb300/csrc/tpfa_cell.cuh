// tpfa_cell.cuh -- the row of one cell of the two-point-flux matrix (Section 4, Eq. model with
// c = 0, unit cells), shared by the regular assembly (setup.cu) and the allocation-free one
// (noalloc.cu) so that both write the same entries in the same order with the same arithmetic.
#pragma once

namespace cpc {

// Entries of row c: 1 + the number of grid neighbours.
__device__ __forceinline__ int tpfa_row_len(int c, int nx, int ny, int nz) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    return 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
}

// Harmonic-mean transmissibility of a unit face between permeabilities a and b.
__device__ __forceinline__ double tpfa_harmonic(double a, double b) { return (2.0 * a * b) / (a + b); }

// Writes row c starting at entry `off`.  Entry order: z-, y-, x-, diagonal, x+, y+, z+ (ascending
// columns).  The diagonal sums the neighbour transmissibilities in that order, then the Dirichlet
// half-cell terms 2 k (2 k_z on z faces) in face order x0, x1, y0, y1, z0, z1 (bits of dmask).
// Vertical transmissibilities use k_z = kzr k.
__device__ __forceinline__ void tpfa_fill_row(int c, int nx, int ny, int nz, const double* logk, double kzr,
                                              int dmask, int off, int* col, double* val) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const int sxy = nx * ny;
    const double kc = exp(logk[c]);
    const double kzc = kzr * kc;
    int nb[6];
    double t[6];
    int cnt = 0;
    if (k > 0)      { nb[cnt] = c - sxy; t[cnt++] = tpfa_harmonic(kzc, kzr * exp(logk[c - sxy])); }
    if (j > 0)      { nb[cnt] = c - nx;  t[cnt++] = tpfa_harmonic(kc, exp(logk[c - nx])); }
    if (i > 0)      { nb[cnt] = c - 1;   t[cnt++] = tpfa_harmonic(kc, exp(logk[c - 1])); }
    const int nlow = cnt;
    if (i < nx - 1) { nb[cnt] = c + 1;   t[cnt++] = tpfa_harmonic(kc, exp(logk[c + 1])); }
    if (j < ny - 1) { nb[cnt] = c + nx;  t[cnt++] = tpfa_harmonic(kc, exp(logk[c + nx])); }
    if (k < nz - 1) { nb[cnt] = c + sxy; t[cnt++] = tpfa_harmonic(kzc, kzr * exp(logk[c + sxy])); }
    double d = 0.0;
    for (int q = 0; q < cnt; ++q) d += t[q];
    if ((dmask & 1) && i == 0)       d += 2.0 * kc;
    if ((dmask & 2) && i == nx - 1)  d += 2.0 * kc;
    if ((dmask & 4) && j == 0)       d += 2.0 * kc;
    if ((dmask & 8) && j == ny - 1)  d += 2.0 * kc;
    if ((dmask & 16) && k == 0)      d += 2.0 * kzc;
    if ((dmask & 32) && k == nz - 1) d += 2.0 * kzc;
    int p = off;
    for (int q = 0; q < nlow; ++q) { col[p] = nb[q]; val[p] = -t[q]; ++p; }
    col[p] = c; val[p] = d; ++p;
    for (int q = nlow; q < cnt; ++q) { col[p] = nb[q]; val[p] = -t[q]; ++p; }
}

}  // namespace cpc
