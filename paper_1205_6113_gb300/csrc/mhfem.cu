// mhfem.cu -- the mixed-hybrid (pressure, multiplier) system of Section 4 (Eq. alge_sys) for the
// lowest-order Raviart-Thomas element on unit bricks, assembled on the device.
//
// Unknowns: the n cell pressures first (cell (i,j,k) = i + nx (j + ny k)), then the face
// multipliers of the x-, y- and z-faces in that order, each family in (k, j, i) order, leaving out
// the faces of Dirichlet boundaries (p = 0 there, so they carry no unknown).  For a unit brick with
// diagonal permeability, the element matrix of the hybridised RT0 method couples a cell to each of
// its faces with -6 k_f (k_f = k on x and y faces, k_z on z faces), the cell to itself with
// sum_f 6 k_f, a face to itself with 4 k_f and to the opposite face of the same cell with 2 k_f.
// Summing the element matrices gives, in ascending column order:
//   cell row c:  (c, sum_f 6 k_f), then (f, -6 k_f) for its free faces;
//   face row f:  (L, -6 k_L), (R, -6 k_R) for its one or two cells L < R, (o_L, 2 k_L), (f, 4 k_L + 4 k_R),
//                (o_R, 2 k_R) with o_L, o_R the opposite faces of L and R (when free).
// Products and sums are rounded one at a time (no fused multiply-add), cell sums in face order,
// face diagonals in cell order, so the values follow the plain sequential assembly.
#include <cub/cub.cuh>

#include "handle.cuh"

namespace cpc {

namespace {

struct MhGrid {
    int nx, ny, nz, n;
    int d[6];                          // Dirichlet flags x0, x1, y0, y1, z0, z1
    int lx, ly, lz;                    // free faces per line along x, per plane column along y, planes along z
    int64_t fx, fy, fz;                // free faces per family
};

MhGrid mh_grid(int nx, int ny, int nz, int dmask) {
    MhGrid g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.n = nx * ny * nz;
    for (int q = 0; q < 6; ++q) g.d[q] = (dmask >> q) & 1;
    g.lx = nx + 1 - g.d[0] - g.d[1];
    g.ly = ny + 1 - g.d[2] - g.d[3];
    g.lz = nz + 1 - g.d[4] - g.d[5];
    g.fx = (int64_t)g.lx * ny * nz;
    g.fy = (int64_t)nx * g.ly * nz;
    g.fz = (int64_t)nx * ny * g.lz;
    return g;
}

// Unknown of face `a` (0..N) along direction dir through the line of cell (i, j, k), or -1.
__device__ __forceinline__ int mh_face(const MhGrid& g, int dir, int a, int i, int j, int k) {
    if (dir == 0) {
        if ((a == 0 && g.d[0]) || (a == g.nx && g.d[1])) return -1;
        return g.n + (k * g.ny + j) * g.lx + (a - g.d[0]);
    }
    if (dir == 1) {
        if ((a == 0 && g.d[2]) || (a == g.ny && g.d[3])) return -1;
        return (int)(g.n + g.fx + ((int64_t)k * g.ly + (a - g.d[2])) * g.nx + i);
    }
    if ((a == 0 && g.d[4]) || (a == g.nz && g.d[5])) return -1;
    return (int)(g.n + g.fx + g.fy + ((int64_t)(a - g.d[4]) * g.ny + j) * g.nx + i);
}

// Row r as a face: direction, face position a along it and the other two coordinates.
__device__ __forceinline__ void mh_face_of(const MhGrid& g, int r, int& dir, int& a, int& i, int& j, int& k) {
    int64_t q = r - g.n;
    if (q < g.fx) {
        dir = 0;
        a = (int)(q % g.lx) + g.d[0];
        const int line = (int)(q / g.lx);
        j = line % g.ny;
        k = line / g.ny;
        i = 0;
        return;
    }
    q -= g.fx;
    if (q < g.fy) {
        dir = 1;
        i = (int)(q % g.nx);
        const int t = (int)(q / g.nx);
        a = t % g.ly + g.d[2];
        k = t / g.ly;
        j = 0;
        return;
    }
    q -= g.fy;
    dir = 2;
    i = (int)(q % g.nx);
    const int t = (int)(q / g.nx);
    j = t % g.ny;
    a = t / g.ny + g.d[4];
    k = 0;
}

__device__ __forceinline__ int mh_cell(const MhGrid& g, int i, int j, int k) { return i + g.nx * (j + g.ny * k); }

// Cell along direction dir at position b of the line through (i, j, k).
__device__ __forceinline__ int mh_cell_at(const MhGrid& g, int dir, int b, int i, int j, int k) {
    return dir == 0 ? mh_cell(g, b, j, k) : dir == 1 ? mh_cell(g, i, b, k) : mh_cell(g, i, j, b);
}

__device__ __forceinline__ int mh_len(const MhGrid& g, int dir) { return dir == 0 ? g.nx : dir == 1 ? g.ny : g.nz; }

// Number of entries of row r.
__global__ void k_mh_rowlen(MhGrid g, int nunk, int* len) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nunk; r += gridDim.x * blockDim.x) {
        int c = 1;
        if (r < g.n) {
            const int i = r % g.nx, j = (r / g.nx) % g.ny, k = r / (g.nx * g.ny);
            const int pos[3] = {i, j, k};
            for (int dir = 0; dir < 3; ++dir)
                for (int s = 0; s < 2; ++s) c += mh_face(g, dir, pos[dir] + s, i, j, k) >= 0;
        } else {
            int dir, a, i, j, k;
            mh_face_of(g, r, dir, a, i, j, k);
            const int N = mh_len(g, dir);
            if (a >= 1) c += 1 + (mh_face(g, dir, a - 1, i, j, k) >= 0);         // L and o_L
            if (a <= N - 1) c += 1 + (mh_face(g, dir, a + 1, i, j, k) >= 0);     // R and o_R
        }
        len[r] = c;
    }
}

__global__ void k_mh_fill(MhGrid g, int nunk, const double* __restrict__ logk, double kzr, const int* __restrict__ rowptr,
                          int* __restrict__ col, double* __restrict__ val) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nunk; r += gridDim.x * blockDim.x) {
        int e = rowptr[r];
        if (r < g.n) {
            const int i = r % g.nx, j = (r / g.nx) % g.ny, k = r / (g.nx * g.ny);
            const double kc = exp(logk[r]);
            const double kz = __dmul_rn(kzr, kc);
            const double kf[3] = {kc, kc, kz};
            double cc = 0.0;
            for (int q = 0; q < 6; ++q) cc = __dadd_rn(cc, __dmul_rn(6.0, kf[q / 2]));
            col[e] = r;
            val[e++] = cc;
            const int pos[3] = {i, j, k};
            for (int dir = 0; dir < 3; ++dir)
                for (int s = 0; s < 2; ++s) {
                    const int f = mh_face(g, dir, pos[dir] + s, i, j, k);
                    if (f < 0) continue;
                    col[e] = f;
                    val[e++] = -__dmul_rn(6.0, kf[dir]);
                }
        } else {
            int dir, a, i, j, k;
            mh_face_of(g, r, dir, a, i, j, k);
            const int N = mh_len(g, dir);
            const bool hasL = a >= 1, hasR = a <= N - 1;
            double kL = 0.0, kR = 0.0;
            if (hasL) {
                const double c = exp(logk[mh_cell_at(g, dir, a - 1, i, j, k)]);
                kL = dir == 2 ? __dmul_rn(kzr, c) : c;
            }
            if (hasR) {
                const double c = exp(logk[mh_cell_at(g, dir, a, i, j, k)]);
                kR = dir == 2 ? __dmul_rn(kzr, c) : c;
            }
            if (hasL) { col[e] = mh_cell_at(g, dir, a - 1, i, j, k); val[e++] = -__dmul_rn(6.0, kL); }
            if (hasR) { col[e] = mh_cell_at(g, dir, a, i, j, k); val[e++] = -__dmul_rn(6.0, kR); }
            if (hasL) {
                const int o = mh_face(g, dir, a - 1, i, j, k);
                if (o >= 0) { col[e] = o; val[e++] = __dmul_rn(2.0, kL); }
            }
            double d = 0.0;
            if (hasL) d = __dadd_rn(d, __dmul_rn(4.0, kL));
            if (hasR) d = __dadd_rn(d, __dmul_rn(4.0, kR));
            col[e] = r;
            val[e++] = d;
            if (hasR) {
                const int o = mh_face(g, dir, a + 1, i, j, k);
                if (o >= 0) { col[e] = o; val[e++] = __dmul_rn(2.0, kR); }
            }
        }
    }
}

inline int mh_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

}  // namespace

// Unknowns and nonzeros of the system, from closed forms over grid lines (host only).
int64_t mhfem_size(int nx, int ny, int nz, int dmask, int64_t* nunk) {
    const MhGrid g = mh_grid(nx, ny, nz, dmask);
    const int64_t nfree = g.fx + g.fy + g.fz;
    *nunk = g.n + nfree;
    // cell-face incidences (each appears twice: cell row and face row) and face-face pairs
    auto along = [&](int N, int d0, int d1, int64_t lines) {
        int64_t inc = 0, pairs = 0;
        for (int a = 0; a < N; ++a) {                   // cell a with faces a and a + 1
            const bool fa = !(a == 0 && d0), fb = !(a + 1 == N && d1);
            inc += fa + fb;
            pairs += 2 * (fa && fb);
        }
        return std::make_pair(inc * lines, pairs * lines);
    };
    const auto x = along(nx, g.d[0], g.d[1], (int64_t)ny * nz);
    const auto y = along(ny, g.d[2], g.d[3], (int64_t)nx * nz);
    const auto z = along(nz, g.d[4], g.d[5], (int64_t)nx * ny);
    return g.n + nfree + 2 * (x.first + y.first + z.first) + (x.second + y.second + z.second);
}

void mhfem_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask, int* rowptr, int* col,
                    double* val, cudaStream_t s) {
    const MhGrid g = mh_grid(nx, ny, nz, dmask);
    int64_t nu = 0;
    mhfem_size(nx, ny, nz, dmask, &nu);
    const int nunk = (int)nu;
    Tmp<int> len(nunk + 1, s);
    CPC_CK(cudaMemsetAsync(len.get() + nunk, 0, sizeof(int), s));
    k_mh_rowlen<<<mh_blocks(nunk), 256, 0, s>>>(g, nunk, len.get());
    size_t tmp = 0;
    CPC_CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp, len.get(), rowptr, nunk + 1, s));
    Tmp<char> t(tmp, s);
    CPC_CK(cub::DeviceScan::ExclusiveSum(t.get(), tmp, len.get(), rowptr, nunk + 1, s));
    k_mh_fill<<<mh_blocks(nunk), 256, 0, s>>>(g, nunk, logk, kzr, rowptr, col, val);
    CPC_LAUNCH_CK();
}

}  // namespace cpc
