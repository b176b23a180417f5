/*
 * oracle.cpp -- reference oracle for combined-preconditioned conjugate gradients
 * (Hu, Wu, Wu, Xu, Zhang, Zhang, Zikatanov, "Combined Preconditioning with Applications in
 * Reservoir Simulation").
 *
 * TEST INFRASTRUCTURE ONLY.  This is plain, slow, single-threaded FP64 CPU code written to be
 * checked against the paper by eye.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load it; the CUDA library shares no code with it and never calls it.
 *
 * What it computes, in the paper's order:
 *   tpfa_assemble  two-point-flux discretisation of -div(a grad p) = f (Section 4, Eq. model, c = 0)
 *                  on a structured grid, harmonic-mean transmissibilities.
 *   ilu0           Algorithm 3.1 (ILU(k)) with k = 0; for SPD A this is IC(0) (Section 3.3).
 *   amg_setup      Section 3.2: A_l = P_l^T A_{l+1} P_l with a C/F splitting and interpolation.
 *                  The paper uses classical Ruge-Stueben coarsening; this oracle (like the CUDA
 *                  path) uses PMIS coarsening with a fixed hash and direct interpolation.
 *   vcycle         Algorithm 3.2 with Gauss-Seidel smoothers S_l (multicolour order), exact
 *                  coarsest solve.
 *   apply_bco      Algorithm 2.1 with u^{k,0} = 0, giving B_co of Eq. barB.
 *   apply_stilde   two V-cycles (AMG(GS) of Section 5); with the IC(0) preconditioner as the
 *                  finest-level smoother, AMG(ILU(0)) of Section 5.
 *   pcg            textbook preconditioned CG (the Krylov method the paper runs, Section 5).
 *   tpfa_gradient  -lambda^T (dA/dlog k) p, the adjoint gradient of a misfit through the assembly.
 *   mhfem_assemble the mixed-hybrid system of Section 4 in the (pressure, multiplier) form of
 *                  Section 5, Eq. alge_sys, for lowest-order Raviart-Thomas on unit bricks.
 *
 * Level numbering here is 0 = finest ... L-1 = coarsest (the paper numbers the other way).
 * Pins: tests/test_oracle_*.py.  Table 2 iteration counts: parity unpinned (the paper's
 * reservoir matrices are not available).
 *
 * Compile with -ffp-contract=off so that results do not depend on the host's FMA contraction.
 *
 * The default build is single-threaded: the OpenMP pragmas below are ignored without -fopenmp.
 * Built with -fopenmp (a second library, used only to time the oracle on all host cores), the
 * row loops of the sparse products, the vector updates and the rows of one colour of a
 * multicolour Gauss-Seidel sweep (mutually uncoupled, so the result is the same) run in parallel,
 * and the dot products reduce in a different order; the IC(0) triangular solves, the
 * natural-order Gauss-Seidel sweep and the coarsest solve stay sequential.
 */
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using std::vector;

struct Csr {
    int n = 0, m = 0;            // rows, columns
    vector<int> ptr, col;
    vector<double> val;
    int nnz() const { return (int)col.size(); }
};

// ---------------------------------------------------------------------------------------------
// Section 4, Eq. model with c = 0: cell-centred two-point flux on unit cells.
// T_ij = 2 k_i k_j / (k_i + k_j) across x/y faces, the same with k_z = kz_ratio * k across
// z faces.  A Dirichlet face (p = 0) adds the half-cell transmissibility 2 k_i (2 k_z,i).
// Row entries are in ascending column order; the diagonal sums the neighbour terms in that
// order, then the boundary terms in face order x0, x1, y0, y1, z0, z1.
// ---------------------------------------------------------------------------------------------
double harmonic(double a, double b) { return (2.0 * a * b) / (a + b); }

Csr tpfa_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask) {
    const int n = nx * ny * nz;
    vector<double> k(n), kz(n);
    for (int c = 0; c < n; ++c) { k[c] = std::exp(logk[c]); kz[c] = kzr * k[c]; }
    Csr A; A.n = A.m = n; A.ptr.assign(n + 1, 0);
    for (int kk = 0; kk < nz; ++kk)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = i + nx * (j + ny * kk);
                // neighbours in ascending index order: z-, y-, x-, x+, y+, z+
                int nb[6]; double t[6]; int cnt = 0;
                if (kk > 0)      { nb[cnt] = c - nx * ny; t[cnt++] = harmonic(kz[c], kz[c - nx * ny]); }
                if (j > 0)       { nb[cnt] = c - nx;      t[cnt++] = harmonic(k[c], k[c - nx]); }
                if (i > 0)       { nb[cnt] = c - 1;       t[cnt++] = harmonic(k[c], k[c - 1]); }
                const int nlow = cnt;
                if (i < nx - 1)  { nb[cnt] = c + 1;       t[cnt++] = harmonic(k[c], k[c + 1]); }
                if (j < ny - 1)  { nb[cnt] = c + nx;      t[cnt++] = harmonic(k[c], k[c + nx]); }
                if (kk < nz - 1) { nb[cnt] = c + nx * ny; t[cnt++] = harmonic(kz[c], kz[c + nx * ny]); }
                double d = 0.0;
                for (int q = 0; q < cnt; ++q) d += t[q];
                if ((dmask & 1) && i == 0)       d += 2.0 * k[c];
                if ((dmask & 2) && i == nx - 1)  d += 2.0 * k[c];
                if ((dmask & 4) && j == 0)       d += 2.0 * k[c];
                if ((dmask & 8) && j == ny - 1)  d += 2.0 * k[c];
                if ((dmask & 16) && kk == 0)     d += 2.0 * kz[c];
                if ((dmask & 32) && kk == nz - 1) d += 2.0 * kz[c];
                for (int q = 0; q < nlow; ++q) { A.col.push_back(nb[q]); A.val.push_back(-t[q]); }
                A.col.push_back(c); A.val.push_back(d);
                for (int q = nlow; q < cnt; ++q) { A.col.push_back(nb[q]); A.val.push_back(-t[q]); }
                A.ptr[c + 1] = (int)A.col.size();
            }
    return A;
}

// Derivative of the assembly above with respect to theta = log k, contracted with two vectors:
// g_c = -lambda^T (dA/dtheta_c) p.  A face between c and j adds T (e_c - e_j)(e_c - e_j)^T to A,
// with dT/dtheta_c = 2 k_c k_j^2 / (k_c + k_j)^2 (k_z on z faces); a Dirichlet face adds
// 2 k_c e_c e_c^T, with derivative 2 k_c.  For A p = q and A lambda = dJ/dp this is dJ/dtheta
// (the adjoint method; A is symmetric).
void tpfa_gradient(int nx, int ny, int nz, const double* logk, double kzr, int dmask, const double* lam,
                   const double* p, double* g) {
    const int n = nx * ny * nz;
    vector<double> k(n), kz(n);
    for (int c = 0; c < n; ++c) { k[c] = std::exp(logk[c]); kz[c] = kzr * k[c]; }
    auto dT = [](double a, double b) { return 2.0 * a * b * b / ((a + b) * (a + b)); };
    for (int kk = 0; kk < nz; ++kk)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = i + nx * (j + ny * kk);
                double s = 0.0;
                auto face = [&](int o, double d) { s += d * (lam[c] - lam[o]) * (p[c] - p[o]); };
                if (kk > 0)      face(c - nx * ny, dT(kz[c], kz[c - nx * ny]));
                if (j > 0)       face(c - nx, dT(k[c], k[c - nx]));
                if (i > 0)       face(c - 1, dT(k[c], k[c - 1]));
                if (i < nx - 1)  face(c + 1, dT(k[c], k[c + 1]));
                if (j < ny - 1)  face(c + nx, dT(k[c], k[c + nx]));
                if (kk < nz - 1) face(c + nx * ny, dT(kz[c], kz[c + nx * ny]));
                double b = 0.0;
                if ((dmask & 1) && i == 0)        b += 2.0 * k[c];
                if ((dmask & 2) && i == nx - 1)   b += 2.0 * k[c];
                if ((dmask & 4) && j == 0)        b += 2.0 * k[c];
                if ((dmask & 8) && j == ny - 1)   b += 2.0 * k[c];
                if ((dmask & 16) && kk == 0)      b += 2.0 * kz[c];
                if ((dmask & 32) && kk == nz - 1) b += 2.0 * kz[c];
                s += b * lam[c] * p[c];
                g[c] = -s;
            }
}

// ---------------------------------------------------------------------------------------------
// Section 4 with the linear system of Section 5 (Eq. alge_sys): mixed-hybrid finite elements,
// lowest-order Raviart-Thomas on unit bricks, fluxes eliminated, c = 0 (M = 0); unknowns are the
// cell pressures and the face multipliers.  On a unit brick the RT0 mass matrix of a^{-1} is
// block-diagonal per direction d with blocks (1/k_d) [[1/3, -1/6], [-1/6, 1/3]] (west/east,
// south/north, bottom/top), so D_K^{-1} has blocks k_d [[4, 2], [2, 4]].  With div w_F = 1 per
// face (unit outward flux) the element contributions are
//   cell-cell  B D^{-1} B^T = sum_F 6 k_F,   cell-face  B D^{-1} C^T = -6 k_F,
//   face-face  C D^{-1} C^T = 4 k_F on the diagonal and 2 k_F to the opposite face,
// with k_F = k (x, y faces) or k_z = kz_ratio k (z faces).  Faces on Dirichlet sides (p = 0)
// carry no unknown.  Unknown order: cells (i fastest), then the remaining x-faces, y-faces and
// z-faces (i fastest within each).  Rows list columns in ascending order; a face diagonal sums its
// cells in ascending cell order.  The right-hand side is the cell sources (f~1 = 0, f~2 = -f).
// ---------------------------------------------------------------------------------------------
struct MhfemIndex {
    int nx, ny, nz, n, nfx, nfy, nfz;
    vector<int> face_id;           // full face index -> unknown index (-1: Dirichlet)
    int nunk = 0;
    MhfemIndex(int nx_, int ny_, int nz_, int dmask) : nx(nx_), ny(ny_), nz(nz_) {
        n = nx * ny * nz;
        nfx = (nx + 1) * ny * nz;
        nfy = nx * (ny + 1) * nz;
        nfz = nx * ny * (nz + 1);
        face_id.assign(nfx + nfy + nfz, -1);
        int next = n;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i <= nx; ++i)
                    if (!((dmask & 1) && i == 0) && !((dmask & 2) && i == nx)) face_id[xf(i, j, k)] = next++;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i < nx; ++i)
                    if (!((dmask & 4) && j == 0) && !((dmask & 8) && j == ny)) face_id[yf(i, j, k)] = next++;
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    if (!((dmask & 16) && k == 0) && !((dmask & 32) && k == nz)) face_id[zf(i, j, k)] = next++;
        nunk = next;
    }
    int xf(int i, int j, int k) const { return (k * ny + j) * (nx + 1) + i; }
    int yf(int i, int j, int k) const { return nfx + (k * (ny + 1) + j) * nx + i; }
    int zf(int i, int j, int k) const { return nfx + nfy + (k * ny + j) * nx + i; }
};

Csr mhfem_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask) {
    MhfemIndex X(nx, ny, nz, dmask);
    const int n = X.n;
    vector<vector<std::pair<int, double>>> rows(X.nunk);
    for (int kk = 0; kk < nz; ++kk)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = i + nx * (j + ny * kk);
                const double k = std::exp(logk[c]), kz = kzr * k;
                const int f[6] = {X.face_id[X.xf(i, j, kk)], X.face_id[X.xf(i + 1, j, kk)],
                                  X.face_id[X.yf(i, j, kk)], X.face_id[X.yf(i, j + 1, kk)],
                                  X.face_id[X.zf(i, j, kk)], X.face_id[X.zf(i, j, kk + 1)]};
                const double kf[6] = {k, k, k, k, kz, kz};
                double cc = 0.0;
                for (int q = 0; q < 6; ++q) cc += 6.0 * kf[q];
                rows[c].push_back({c, cc});
                for (int q = 0; q < 6; ++q) {
                    if (f[q] < 0) continue;
                    rows[c].push_back({f[q], -6.0 * kf[q]});
                    rows[f[q]].push_back({c, -6.0 * kf[q]});
                    rows[f[q]].push_back({f[q], 4.0 * kf[q]});
                    const int o = f[q ^ 1];
                    if (o >= 0) rows[f[q]].push_back({o, 2.0 * kf[q]});
                }
            }
    Csr A;
    A.n = A.m = X.nunk;
    A.ptr.assign(X.nunk + 1, 0);
    for (int r = 0; r < X.nunk; ++r) {
        auto& e = rows[r];
        // stable sort by column keeps the cell order of the contributions to one entry
        std::stable_sort(e.begin(), e.end(), [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
            return a.first < b.first;
        });
        for (size_t q = 0; q < e.size();) {
            double v = 0.0;
            size_t t = q;
            for (; t < e.size() && e[t].first == e[q].first; ++t) v += e[t].second;
            A.col.push_back(e[q].first);
            A.val.push_back(v);
            q = t;
        }
        A.ptr[r + 1] = (int)A.col.size();
    }
    (void)n;
    return A;
}

// ---------------------------------------------------------------------------------------------
// Basic sparse helpers
// ---------------------------------------------------------------------------------------------
void spmv(const Csr& A, const double* x, double* y) {
#pragma omp parallel for schedule(static) if (A.n > 20000)
    for (int i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
        y[i] = s;
    }
}

// r = f - A u
void residual(const Csr& A, const double* f, const double* u, double* r) {
#pragma omp parallel for schedule(static) if (A.n > 20000)
    for (int i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) s += A.val[p] * u[A.col[p]];
        r[i] = f[i] - s;
    }
}

Csr transpose(const Csr& A) {
    Csr T; T.n = A.m; T.m = A.n; T.ptr.assign(T.n + 1, 0);
    for (int p = 0; p < A.nnz(); ++p) T.ptr[A.col[p] + 1]++;
    for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.nnz()); T.val.resize(A.nnz());
    vector<int> next(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n; ++i)            // ascending source row => ascending column in T
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int q = next[A.col[p]]++;
            T.col[q] = i; T.val[q] = A.val[p];
        }
    return T;
}

// C = A * B.  Each output entry sums its products in generation order: over row i of A in
// ascending column k, then over row k of B in ascending column j.  Output columns ascending.
Csr spgemm(const Csr& A, const Csr& B) {
    Csr C; C.n = A.n; C.m = B.m; C.ptr.assign(A.n + 1, 0);
    vector<double> acc(B.m, 0.0);
    vector<int> mark(B.m, -1), touched;
    for (int i = 0; i < A.n; ++i) {
        touched.clear();
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int k = A.col[p];
            for (int q = B.ptr[k]; q < B.ptr[k + 1]; ++q) {
                const int j = B.col[q];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; touched.push_back(j); }
                acc[j] += A.val[p] * B.val[q];
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int j : touched) { C.col.push_back(j); C.val.push_back(acc[j]); }
        C.ptr[i + 1] = (int)C.col.size();
    }
    return C;
}

int find_diag(const Csr& A, int i) {
    for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) if (A.col[p] == i) return p;
    return -1;
}

// Published MurmurHash3 32-bit finaliser (a bijection on 32-bit words): tie-break weights for
// the C/F splitting and the colouring.
uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
    return h;
}
const uint32_t COLOUR_SEED = 0x5bd1e995u;

// ---------------------------------------------------------------------------------------------
// Algorithm 3.1 with k = 0 (level of fill zero = the pattern of A, "Level of fill" definition).
// IKJ elimination: for each row i, for each m < i in the row (ascending), a_im := a_im / a_mm,
// then a_ij := a_ij - a_im a_mj for every j > m that is in the pattern of row i.  L (unit lower)
// and U (upper with diagonal) overwrite the values of A.  Returns the row of the first
// non-positive or non-finite pivot, or -1.  For SPD A this is IC(0) in L D L^T form (Section 3.3).
// ---------------------------------------------------------------------------------------------
int ilu0(const Csr& A, vector<double>& lu, vector<int>& diag) {
    const int n = A.n;
    lu = A.val;
    diag.assign(n, -1);
    for (int i = 0; i < n; ++i) diag[i] = find_diag(A, i);
    vector<int> pos(n, -1);
    for (int i = 0; i < n; ++i) {
        if (diag[i] < 0) return i;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) pos[A.col[p]] = p;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int m = A.col[p];
            if (m >= i) break;
            lu[p] = lu[p] / lu[diag[m]];
            for (int q = diag[m] + 1; q < A.ptr[m + 1]; ++q) {
                const int j = A.col[q];
                if (pos[j] >= 0) lu[pos[j]] -= lu[p] * lu[q];
            }
        }
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) pos[A.col[p]] = -1;
        const double u = lu[diag[i]];
        if (!(u > 0.0) || !std::isfinite(u)) return i;
    }
    return -1;
}

// w = (LU)^{-1} t : forward substitution with unit L, then backward substitution with U.
void ilu0_solve(const Csr& A, const vector<double>& lu, const vector<int>& diag,
                const double* t, double* w) {
    const int n = A.n;
    vector<double> y(n);
    for (int i = 0; i < n; ++i) {
        double s = t[i];
        for (int p = A.ptr[i]; p < diag[i]; ++p) s -= lu[p] * y[A.col[p]];
        y[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int p = diag[i] + 1; p < A.ptr[i + 1]; ++p) s -= lu[p] * w[A.col[p]];
        w[i] = s / lu[diag[i]];
    }
}

Csr permute_sym(const Csr& A, const vector<int>& order) {   // order[new] = old
    const int n = A.n;
    vector<int> inv(n);
    for (int q = 0; q < n; ++q) inv[order[q]] = q;
    Csr B; B.n = B.m = n; B.ptr.assign(n + 1, 0);
    vector<std::pair<int, double>> row;
    for (int q = 0; q < n; ++q) {
        const int i = order[q];
        row.clear();
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) row.push_back({inv[A.col[p]], A.val[p]});
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int, double>& a, const std::pair<int, double>& b) { return a.first < b.first; });
        for (auto& e : row) { B.col.push_back(e.first); B.val.push_back(e.second); }
        B.ptr[q + 1] = (int)B.col.size();
    }
    return B;
}

// ---------------------------------------------------------------------------------------------
// AMG setup (Section 3.2).  Rules shared with the CUDA path (both written from this statement):
//  strength   j strongly influences i (j in S_i) iff j != i and -a_ij >= theta * max_{k != i}(-a_ik)
//             with that maximum > 0 (the paper leaves theta open; the callers' default is 0.12);
//  PMIS       weight (|S^T_i|, fmix32(i)) compared lexicographically; points with |S^T_i| = 0 are F;
//             each round, undecided points whose weight beats every undecided point of
//             S_i u S^T_i become C, then undecided points with a C point in S_i become F;
//  direct interpolation  for F point i with strong C set C_i:
//             P_ij = -(sum_{k != i} min(a_ik,0) / sum_{j in C_i} a_ij) * a_ij / (a_ii + sum_{k != i} max(a_ik,0));
//             C point: P_{i,c(i)} = 1; coarse points numbered in ascending fine index;
//  Galerkin   A_c = R (A P) with R = P^T (explicit transpose);
//  stop       n_l <= coarse_max (callers' default 2048), max_levels reached, or no coarsening;
//             coarsest solved exactly;
//  colouring  if the pattern graph of A_l is bipartite: breadth-first parity from the smallest
//             index of each component (red-black on a structured grid); otherwise greedy
//             colouring in decreasing priority (peel round, fmix32(i ^ COLOUR_SEED)): each point
//             takes the smallest colour unused by its neighbours of higher priority.  Peel
//             rounds: while points remain, those with at most twice the smallest remaining
//             degree (off-diagonal count, reduced by the entries to earlier rounds) take the
//             round number (a smallest-last style ordering: fewer colours than random order).
// ---------------------------------------------------------------------------------------------
struct Level {
    Csr A, P, R;
    vector<int> cf;        // 1 = C, 0 = F (not set on the coarsest level)
    vector<int> colour;    // smoothing colour of each row
    int ncolours = 0;
    vector<int> order;     // colour-major order, ascending index within a colour
    vector<int> diag;      // position of a_ii
};

struct Hierarchy {
    vector<Level> lev;
    vector<double> chol;   // dense lower Cholesky factor of the coarsest A (row-major nc x nc)
    int nc = 0;
};

void strength(const Csr& A, double theta, Csr& S) {
    S.n = S.m = A.n; S.ptr.assign(A.n + 1, 0); S.col.clear(); S.val.clear();
    for (int i = 0; i < A.n; ++i) {
        double mx = 0.0;
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
            if (A.col[p] != i) mx = std::max(mx, -A.val[p]);
        if (mx > 0.0)
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
                if (A.col[p] != i && -A.val[p] >= theta * mx) { S.col.push_back(A.col[p]); S.val.push_back(1.0); }
        S.ptr[i + 1] = (int)S.col.size();
    }
}

bool heavier(const vector<int>& cnt, int a, int b) {   // weight(a) > weight(b)
    if (cnt[a] != cnt[b]) return cnt[a] > cnt[b];
    return fmix32((uint32_t)a) > fmix32((uint32_t)b);
}

void pmis(const Csr& S, const Csr& ST, vector<int>& cf) {
    const int n = S.n;
    enum { UNDEC = -1, F = 0, C = 1 };
    vector<int> cnt(n);
    for (int i = 0; i < n; ++i) cnt[i] = ST.ptr[i + 1] - ST.ptr[i];
    cf.assign(n, UNDEC);
    for (int i = 0; i < n; ++i) if (cnt[i] == 0) cf[i] = F;
    vector<int> sel;
    for (;;) {
        bool any = false;
        sel.clear();
        for (int i = 0; i < n; ++i) {
            if (cf[i] != UNDEC) continue;
            any = true;
            bool best = true;
            for (int p = S.ptr[i]; p < S.ptr[i + 1] && best; ++p) {
                const int j = S.col[p];
                if (cf[j] == UNDEC && heavier(cnt, j, i)) best = false;
            }
            for (int p = ST.ptr[i]; p < ST.ptr[i + 1] && best; ++p) {
                const int j = ST.col[p];
                if (cf[j] == UNDEC && heavier(cnt, j, i)) best = false;
            }
            if (best) sel.push_back(i);
        }
        if (!any) break;
        for (int i : sel) cf[i] = C;
        for (int i = 0; i < n; ++i) {
            if (cf[i] != UNDEC) continue;
            for (int p = S.ptr[i]; p < S.ptr[i + 1]; ++p)
                if (cf[S.col[p]] == C) { cf[i] = F; break; }
        }
    }
}

Csr direct_interpolation(const Csr& A, const Csr& S, const vector<int>& cf, int& nc) {
    const int n = A.n;
    vector<int> cidx(n, -1);
    nc = 0;
    for (int i = 0; i < n; ++i) if (cf[i] == 1) cidx[i] = nc++;
    Csr P; P.n = n; P.m = nc; P.ptr.assign(n + 1, 0);
    vector<char> strong(n, 0);
    for (int i = 0; i < n; ++i) {
        if (cf[i] == 1) {
            P.col.push_back(cidx[i]); P.val.push_back(1.0);
        } else {
            for (int p = S.ptr[i]; p < S.ptr[i + 1]; ++p) strong[S.col[p]] = 1;
            double sum_neg = 0.0, sum_pos = 0.0, c_neg = 0.0, aii = 0.0;
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                const int j = A.col[p];
                const double a = A.val[p];
                if (j == i) { aii = a; continue; }
                if (a < 0.0) sum_neg += a; else sum_pos += a;
                if (strong[j] && cf[j] == 1) c_neg += a;
            }
            if (c_neg != 0.0) {
                const double alpha = sum_neg / c_neg;
                const double d = aii + sum_pos;
                for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                    const int j = A.col[p];
                    if (j != i && strong[j] && cf[j] == 1) {
                        P.col.push_back(cidx[j]); P.val.push_back(-alpha * A.val[p] / d);
                    }
                }
            }
            for (int p = S.ptr[i]; p < S.ptr[i + 1]; ++p) strong[S.col[p]] = 0;
        }
        P.ptr[i + 1] = (int)P.col.size();
    }
    return P;
}

// Two-colouring by breadth-first parity: each connected component of the pattern graph is
// searched from its smallest index, colour = distance mod 2.  Returns false (colour undefined)
// if some edge joins two vertices of equal parity, i.e. the graph is not bipartite.
bool colour_bipartite(const Csr& A, vector<int>& colour) {
    const int n = A.n;
    colour.assign(n, -1);
    vector<int> queue;
    for (int root = 0; root < n; ++root) {
        if (colour[root] >= 0) continue;
        colour[root] = 0;
        queue.assign(1, root);
        for (size_t h = 0; h < queue.size(); ++h) {
            const int i = queue[h];
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                const int j = A.col[p];
                if (j == i) continue;
                if (colour[j] < 0) { colour[j] = colour[i] ^ 1; queue.push_back(j); }
            }
        }
    }
    for (int i = 0; i < n; ++i)
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
            if (A.col[p] != i && colour[A.col[p]] == colour[i]) return false;
    return true;
}

// Peel rounds (a smallest-last style ordering): deg_i = number of off-diagonal entries of row i;
// while points remain, every remaining point with deg_i <= 2 min_{remaining} deg takes the current
// round number, then each remaining point loses one degree per entry of its row in that round.
vector<int> peel_rounds(const Csr& A) {
    const int n = A.n;
    vector<int> deg(n, 0), rnd(n, -1);
    for (int i = 0; i < n; ++i)
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
            if (A.col[p] != i) ++deg[i];
    int left = n;
    for (int r = 0; left > 0; ++r) {
        int dmin = INT_MAX;
        for (int i = 0; i < n; ++i) if (rnd[i] < 0) dmin = std::min(dmin, deg[i]);
        for (int i = 0; i < n; ++i)
            if (rnd[i] < 0 && deg[i] <= 2 * dmin) { rnd[i] = r; --left; }
        for (int i = 0; i < n; ++i) {
            if (rnd[i] >= 0) continue;
            for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
                if (A.col[p] != i && rnd[A.col[p]] == r) --deg[i];
        }
    }
    return rnd;
}

// Smoothing colours of a level: the breadth-first 2-colouring when the graph is bipartite (the
// red-black colouring of a structured grid); otherwise greedy colouring (smallest colour unused by
// the neighbours coloured before) in decreasing priority (peel round, fmix32(i ^ COLOUR_SEED)).
void colour_jp(const Csr& A, vector<int>& colour, int& ncol, vector<int>& order) {
    const int n = A.n;
    if (colour_bipartite(A, colour)) {
        ncol = 0;
        for (int i = 0; i < n; ++i) ncol = std::max(ncol, colour[i] + 1);
        order.clear();
        for (int c = 0; c < ncol; ++c)
            for (int i = 0; i < n; ++i) if (colour[i] == c) order.push_back(i);
        return;
    }
    const vector<int> rnd = peel_rounds(A);
    vector<int> seq(n);
    for (int i = 0; i < n; ++i) seq[i] = i;
    std::sort(seq.begin(), seq.end(), [&](int a, int b) {
        if (rnd[a] != rnd[b]) return rnd[a] > rnd[b];
        return fmix32((uint32_t)a ^ COLOUR_SEED) > fmix32((uint32_t)b ^ COLOUR_SEED);
    });
    colour.assign(n, -1);
    vector<char> used;
    for (int i : seq) {
        used.assign(A.ptr[i + 1] - A.ptr[i] + 2, 0);
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int c = colour[A.col[p]];
            if (A.col[p] != i && c >= 0 && c < (int)used.size()) used[c] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        colour[i] = c;
    }
    ncol = 0;
    for (int i = 0; i < n; ++i) ncol = std::max(ncol, colour[i] + 1);
    order.clear();
    for (int c = 0; c < ncol; ++c)
        for (int i = 0; i < n; ++i) if (colour[i] == c) order.push_back(i);
}

bool dense_cholesky(const Csr& A, vector<double>& L) {
    const int n = A.n;
    L.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) L[(size_t)i * n + A.col[p]] = A.val[p];
    for (int j = 0; j < n; ++j) {
        double d = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        d = std::sqrt(d);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = L[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / d;
        }
        for (int k = j + 1; k < n; ++k) L[(size_t)j * n + k] = 0.0;
    }
    return true;
}

void dense_cholesky_solve(const vector<double>& L, int n, const double* f, double* u) {
    vector<double> y(n);
    for (int i = 0; i < n; ++i) {
        double s = f[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * u[k];
        u[i] = s / L[(size_t)i * n + i];
    }
}

const int DENSE_MAX = 4096;

// Returns 0 on success, 7 if the coarsest level is too large for the dense solve or not SPD.
int amg_setup(const Csr& A0, double theta, int coarse_max, int max_levels, Hierarchy& H) {
    H.lev.clear();
    H.lev.emplace_back();
    H.lev[0].A = A0;
    for (;;) {
        Level& L = H.lev.back();
        const int n = L.A.n;
        L.diag.resize(n);
        for (int i = 0; i < n; ++i) L.diag[i] = find_diag(L.A, i);
        bool coarsest = (n <= coarse_max) || ((int)H.lev.size() >= max_levels);
        if (!coarsest) {
            Csr S, ST;
            strength(L.A, theta, S);
            ST = transpose(S);
            pmis(S, ST, L.cf);
            int nc = 0;
            L.P = direct_interpolation(L.A, S, L.cf, nc);
            if (nc == 0 || nc == n) {
                coarsest = true;
                L.cf.clear(); L.P = Csr();
            } else {
                L.R = transpose(L.P);
                Csr AP = spgemm(L.A, L.P);
                Csr Ac = spgemm(L.R, AP);
                colour_jp(L.A, L.colour, L.ncolours, L.order);
                H.lev.emplace_back();
                H.lev.back().A = std::move(Ac);
                continue;
            }
        }
        // coarsest level
        if (n > DENSE_MAX) return 7;
        H.nc = n;
        if (!dense_cholesky(L.A, H.chol)) return 7;
        break;
    }
    return 0;
}

// Gauss-Seidel smoother of level l applied to a vector (Section 3.3, "standard GS"), in the
// colour-major order pi: S_l = (D + L_pi)^{-1} (forward, colours ascending) and
// S_l^T = (D + U_pi)^{-1} (backward, colours descending).  natural = 1 uses pi = identity.
void gs_apply(const Level& L, bool natural, bool backward, const double* r, double* d) {
    const Csr& A = L.A;
    const int n = A.n;
    vector<int> pos(n);
    vector<int> ord(n);
    if (natural) for (int i = 0; i < n; ++i) ord[i] = i;
    else ord = L.order;
    for (int q = 0; q < n; ++q) pos[ord[q]] = q;
    auto row = [&](int q) {
        const int i = ord[q];
        double acc = r[i];
        for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int j = A.col[p];
            if (j == i) continue;
            const bool solved = backward ? (pos[j] > q) : (pos[j] < q);
            if (solved) acc -= A.val[p] * d[j];
        }
        d[i] = acc / A.val[L.diag[i]];
    };
    if (natural) {
        for (int s = 0; s < n; ++s) row(backward ? n - 1 - s : s);
        return;
    }
    // colour-major order: the rows of one colour are consecutive in ord and not coupled to each
    // other, so within a colour the order of the row updates does not matter
    vector<int> seg(L.ncolours + 1, 0);
    for (int i = 0; i < n; ++i) seg[L.colour[i] + 1]++;
    for (int c = 0; c < L.ncolours; ++c) seg[c + 1] += seg[c];
    for (int cc = 0; cc < L.ncolours; ++cc) {
        const int c = backward ? L.ncolours - 1 - cc : cc;
        const int q0 = seg[c], q1 = seg[c + 1];
#pragma omp parallel for schedule(static) if (q1 - q0 > 4000)
        for (int t = q0; t < q1; ++t) row(backward ? q0 + q1 - 1 - t : t);
    }
}

struct Oracle {
    Csr A;
    Hierarchy H;
    int gs_natural = 0;
    // IC(0) of A in the chosen ordering
    int ic_colour_order = 0;
    vector<int> ic_order;          // order[new] = old (empty: natural)
    Csr Aic;                       // A in the IC ordering
    vector<double> lu;
    vector<int> lu_diag;
};

// Algorithm 3.2 (V-cycle), applied with initial guess u (in/out).  The pre-smoother is the
// forward sweep S_l (pre_bwd = false) and the post-smoother its adjoint S_l^T (post_bwd = true).
// The transpose of a cycle with pre-smoother M and post-smoother N is the cycle with
// pre-smoother N^T and post-smoother M^T (take the A-adjoint of the error propagation of
// Section 3.3 factor by factor); transpose_cycle() builds it that way.  With M = S_l and
// N = S_l^T it is the same cycle, so S^T = S.
//
// AMG(ILU(0)) of Section 5 replaces the smoother on the finest level by the IC(0) preconditioner
// B: one smoothing step is u <- u + B (f - A u) both before and after the coarse correction.  B is
// symmetric, so that cycle is its own transpose as well.
struct Cycle { bool pre_bwd = false, post_bwd = true, ilu_fine = false; };

Cycle transpose_cycle(Cycle c) {
    Cycle t;
    t.pre_bwd = !c.post_bwd;
    t.post_bwd = !c.pre_bwd;
    t.ilu_fine = c.ilu_fine;
    return t;
}

void apply_B(const struct Oracle& O, const double* r, double* z);

void vcycle(const Oracle& O, int l, const double* f, double* u, Cycle cy) {
    const Level& L = O.H.lev[l];
    const int n = L.A.n;
    if (l == (int)O.H.lev.size() - 1) {                       // step 2(b) at the coarsest level
        dense_cholesky_solve(O.H.chol, n, f, u);
        return;
    }
    const bool ilu = cy.ilu_fine && l == 0;
    vector<double> r(n), d(n);
    residual(L.A, f, u, r.data());                              // (1) pre-smoothing
    if (ilu) apply_B(O, r.data(), d.data());
    else gs_apply(L, O.gs_natural, cy.pre_bwd, r.data(), d.data());
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) u[i] += d[i];
    residual(L.A, f, u, r.data());                              // (2a) restriction
    const int nc = L.P.m;
    vector<double> fc(nc), e(nc, 0.0);
    spmv(L.R, r.data(), fc.data());
    vcycle(O, l + 1, fc.data(), e.data(), cy);                  // (2b) zero initial guess
    vector<double> pe(n);
    spmv(L.P, e.data(), pe.data());                             // (2c) prolongation
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) u[i] += pe[i];
    residual(L.A, f, u, r.data());                              // (3) post-smoothing
    if (ilu) apply_B(O, r.data(), d.data());
    else gs_apply(L, O.gs_natural, cy.post_bwd, r.data(), d.data());
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) u[i] += d[i];
}

// z = S r (transpose = false) or z = S^T r (transpose = true), zero initial guess; with ilu_fine
// the cycle of AMG(ILU(0)).
void apply_S(const Oracle& O, const double* r, double* z, bool transpose, bool ilu_fine = false) {
    const int n = O.A.n;
    for (int i = 0; i < n; ++i) z[i] = 0.0;
    Cycle cy;
    cy.ilu_fine = ilu_fine;
    vcycle(O, 0, r, z, transpose ? transpose_cycle(cy) : cy);
}

void apply_B(const Oracle& O, const double* r, double* z) {
    const int n = O.A.n;
    if (O.ic_order.empty()) { ilu0_solve(O.Aic, O.lu, O.lu_diag, r, z); return; }
    vector<double> rp(n), zp(n);
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int q = 0; q < n; ++q) rp[q] = r[O.ic_order[q]];
    ilu0_solve(O.Aic, O.lu, O.lu_diag, rp.data(), zp.data());
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int q = 0; q < n; ++q) z[O.ic_order[q]] = zp[q];
}

// Algorithm 2.1 with u^{k,0} = 0 and f = r: the action z = B_co r of Eq. barB.
void apply_bco(const Oracle& O, const double* r, double* z) {
    const int n = O.A.n;
    vector<double> u1(n), u2(n), t(n), c(n);
    apply_S(O, r, u1.data(), false);                            // (1) u1 = 0 + S (r - A 0)
    residual(O.A, r, u1.data(), t.data());                      // (2) u2 = u1 + B (r - A u1)
    apply_B(O, t.data(), c.data());
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) u2[i] = u1[i] + c[i];
    residual(O.A, r, u2.data(), t.data());                      // (3) u3 = u2 + S^T (r - A u2)
    apply_S(O, t.data(), c.data(), true);
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) z[i] = u2[i] + c[i];
}

// S~ = S + S^T - S^T A S: two cycles, I - S~A = (I - S^T A)(I - S A) (the "AMG alone" preconditioner
// AMG(GS) of Section 5; with ilu_fine, AMG(ILU(0)): the same two cycles with B as finest smoother).
void apply_stilde(const Oracle& O, const double* r, double* z, bool ilu_fine = false) {
    const int n = O.A.n;
    vector<double> u1(n), t(n), c(n);
    apply_S(O, r, u1.data(), false, ilu_fine);
    residual(O.A, r, u1.data(), t.data());
    apply_S(O, t.data(), c.data(), true, ilu_fine);
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) z[i] = u1[i] + c[i];
}

// Additive variant B^ = S~ + B (Eq. Ba with W_1 = V, Pi_1 = I, A_1^{-1} = B).
void apply_bhat(const Oracle& O, const double* r, double* z) {
    const int n = O.A.n;
    vector<double> a(n), b(n);
    apply_stilde(O, r, a.data());
    apply_B(O, r, b.data());
    for (int i = 0; i < n; ++i) z[i] = a[i] + b[i];
}

enum Op { OP_BCO = 0, OP_S = 1, OP_ST = 2, OP_B = 3, OP_STILDE = 4, OP_BHAT = 5, OP_A = 6, OP_I = 7,
          OP_S_ILU = 8, OP_AMG_ILU = 9 };

int apply_op(const Oracle& O, int op, const double* r, double* z) {
    const int n = O.A.n;
    switch (op) {
        case OP_BCO: apply_bco(O, r, z); return 0;
        case OP_S: apply_S(O, r, z, false); return 0;
        case OP_ST: apply_S(O, r, z, true); return 0;
        case OP_B: apply_B(O, r, z); return 0;
        case OP_STILDE: apply_stilde(O, r, z); return 0;
        case OP_BHAT: apply_bhat(O, r, z); return 0;
        case OP_A: spmv(O.A, r, z); return 0;
        case OP_I: for (int i = 0; i < n; ++i) z[i] = r[i]; return 0;
        case OP_S_ILU: apply_S(O, r, z, false, true); return 0;
        case OP_AMG_ILU: apply_stilde(O, r, z, true); return 0;
    }
    return 1;
}

double dot(const double* a, const double* b, int n) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s) if (n > 20000)
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

}  // namespace

// =============================================================================================
// C interface for ctypes.  Status codes: 0 ok, 1 invalid argument, 2 IC(0) breakdown,
// 3 not converged within maxit, 4 CG breakdown, 7 AMG setup failure.
// =============================================================================================
extern "C" {

// Threads the parallel loops use (1 in the default single-threaded build).
int orc_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_tpfa_nnz(int nx, int ny, int nz) {
    // 2-D/3-D structured pattern: diagonal plus two entries per interior face
    const long faces = (long)(nx - 1) * ny * nz + (long)nx * (ny - 1) * nz + (long)nx * ny * (nz - 1);
    return (int)((long)nx * ny * nz + 2 * faces);
}

int orc_tpfa(int nx, int ny, int nz, const double* logk, double kz_ratio, int dmask,
             int* rowptr, int* col, double* val) {
    if (nx < 1 || ny < 1 || nz < 1) return 1;
    Csr A = tpfa_assemble(nx, ny, nz, logk, kz_ratio, dmask);
    std::memcpy(rowptr, A.ptr.data(), sizeof(int) * (A.n + 1));
    std::memcpy(col, A.col.data(), sizeof(int) * A.nnz());
    std::memcpy(val, A.val.data(), sizeof(double) * A.nnz());
    return 0;
}

// MHFEM (p, lambda) system: sizes[0] = unknowns, sizes[1] = nonzeros.
int orc_mhfem_size(int nx, int ny, int nz, const double* logk, double kz_ratio, int dmask, int* sizes) {
    if (nx < 1 || ny < 1 || nz < 1) return 1;
    Csr A = mhfem_assemble(nx, ny, nz, logk, kz_ratio, dmask);
    sizes[0] = A.n;
    sizes[1] = A.nnz();
    return 0;
}

int orc_mhfem(int nx, int ny, int nz, const double* logk, double kz_ratio, int dmask, int* rowptr, int* col,
              double* val) {
    if (nx < 1 || ny < 1 || nz < 1) return 1;
    Csr A = mhfem_assemble(nx, ny, nz, logk, kz_ratio, dmask);
    std::memcpy(rowptr, A.ptr.data(), sizeof(int) * (A.n + 1));
    std::memcpy(col, A.col.data(), sizeof(int) * A.nnz());
    std::memcpy(val, A.val.data(), sizeof(double) * A.nnz());
    return 0;
}

int orc_tpfa_gradient(int nx, int ny, int nz, const double* logk, double kz_ratio, int dmask, const double* lam,
                      const double* p, double* g) {
    if (nx < 1 || ny < 1 || nz < 1) return 1;
    tpfa_gradient(nx, ny, nz, logk, kz_ratio, dmask, lam, p, g);
    return 0;
}

void* orc_create(int n, const int* rowptr, const int* col, const double* val, double theta,
                 int coarse_max, int max_levels, int gs_natural, int ic_colour_order, int* status) {
    *status = 1;
    if (n <= 0 || rowptr[0] != 0) return nullptr;
    Oracle* O = new Oracle();
    O->A.n = O->A.m = n;
    O->A.ptr.assign(rowptr, rowptr + n + 1);
    O->A.col.assign(col, col + rowptr[n]);
    O->A.val.assign(val, val + rowptr[n]);
    for (int i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) { delete O; return nullptr; }
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) { delete O; return nullptr; }
            if (p > rowptr[i] && col[p] <= col[p - 1]) { delete O; return nullptr; }
        }
        if (find_diag(O->A, i) < 0) { delete O; return nullptr; }
    }
    O->gs_natural = gs_natural;
    O->ic_colour_order = ic_colour_order;
    // IC(0) in natural order first, so that a breakdown is reported as such (status 2)
    O->Aic = O->A;
    if (ilu0(O->Aic, O->lu, O->lu_diag) >= 0) { *status = 2; delete O; return nullptr; }
    int st = amg_setup(O->A, theta, coarse_max, max_levels, O->H);
    if (st) { *status = st; delete O; return nullptr; }
    if (ic_colour_order && O->H.lev.size() > 1) {     // IC(0) of the colour-ordered matrix
        O->ic_order = O->H.lev[0].order;
        O->Aic = permute_sym(O->A, O->ic_order);
        if (ilu0(O->Aic, O->lu, O->lu_diag) >= 0) { *status = 2; delete O; return nullptr; }
    }
    *status = 0;
    return O;
}

void orc_destroy(void* h) { delete static_cast<Oracle*>(h); }

int orc_nlevels(void* h) { return (int)static_cast<Oracle*>(h)->H.lev.size(); }

// sizes[0..4] = n, nnz(A_l), ncolours, ncols(P_l), nnz(P_l)
int orc_level_sizes(void* h, int l, int* sizes) {
    Oracle* O = static_cast<Oracle*>(h);
    if (l < 0 || l >= (int)O->H.lev.size()) return 1;
    const Level& L = O->H.lev[l];
    sizes[0] = L.A.n; sizes[1] = L.A.nnz(); sizes[2] = L.ncolours; sizes[3] = L.P.m; sizes[4] = L.P.nnz();
    return 0;
}

int orc_level_A(void* h, int l, int* ptr, int* col, double* val) {
    Oracle* O = static_cast<Oracle*>(h);
    if (l < 0 || l >= (int)O->H.lev.size()) return 1;
    const Csr& A = O->H.lev[l].A;
    std::memcpy(ptr, A.ptr.data(), sizeof(int) * (A.n + 1));
    std::memcpy(col, A.col.data(), sizeof(int) * A.nnz());
    std::memcpy(val, A.val.data(), sizeof(double) * A.nnz());
    return 0;
}

int orc_level_P(void* h, int l, int* ptr, int* col, double* val) {
    Oracle* O = static_cast<Oracle*>(h);
    if (l < 0 || l + 1 >= (int)O->H.lev.size()) return 1;
    const Csr& P = O->H.lev[l].P;
    std::memcpy(ptr, P.ptr.data(), sizeof(int) * (P.n + 1));
    std::memcpy(col, P.col.data(), sizeof(int) * P.nnz());
    std::memcpy(val, P.val.data(), sizeof(double) * P.nnz());
    return 0;
}

int orc_level_cf_colour(void* h, int l, int* cf, int* colour) {
    Oracle* O = static_cast<Oracle*>(h);
    if (l < 0 || l + 1 >= (int)O->H.lev.size()) return 1;
    const Level& L = O->H.lev[l];
    std::memcpy(cf, L.cf.data(), sizeof(int) * L.A.n);
    std::memcpy(colour, L.colour.data(), sizeof(int) * L.A.n);
    return 0;
}

// IC(0) factor values on the pattern of A in the IC ordering (L strictly below, U on/above).
int orc_ic0_values(void* h, double* lu) {
    Oracle* O = static_cast<Oracle*>(h);
    std::memcpy(lu, O->lu.data(), sizeof(double) * O->lu.size());
    return 0;
}

// Level operators: op 0: y = A_l x; 1: y = S_l x (forward GS); 2: y = S_l^T x (backward GS);
// 3: y = A_l^{-1} x on the coarsest level; 4: y = V-cycle of level l with zero initial guess.
int orc_level_apply(void* h, int l, int op, const double* x, double* y) {
    Oracle* O = static_cast<Oracle*>(h);
    if (l < 0 || l >= (int)O->H.lev.size()) return 1;
    const Level& L = O->H.lev[l];
    const bool last = (l == (int)O->H.lev.size() - 1);
    switch (op) {
        case 0: spmv(L.A, x, y); return 0;
        case 1: if (last) return 1; gs_apply(L, O->gs_natural, false, x, y); return 0;
        case 2: if (last) return 1; gs_apply(L, O->gs_natural, true, x, y); return 0;
        case 3: if (!last) return 1; dense_cholesky_solve(O->H.chol, L.A.n, x, y); return 0;
        case 4: for (int i = 0; i < L.A.n; ++i) y[i] = 0.0; vcycle(*O, l, x, y, Cycle()); return 0;
    }
    return 1;
}

int orc_apply(void* h, int op, const double* r, double* z) {
    return apply_op(*static_cast<Oracle*>(h), op, r, z);
}

// Textbook PCG (x0 = 0), stopping when ||r_k||_2 / ||b||_2 < tol.  res_hist[k] = ||r_k||/||b||
// for k = 0..iters; alpha[k], beta[k] are the CG coefficients (for the Lanczos estimate).
// out[0] = true relative residual ||b - A x|| / ||b|| at exit.
int orc_pcg(void* h, int op, const double* b, double* x, double tol, int maxit, int* iters,
            double* res_hist, double* alpha_out, double* beta_out, int cap, double* out) {
    Oracle* O = static_cast<Oracle*>(h);
    const int n = O->A.n;
    vector<double> r(b, b + n), z(n), p(n), q(n);
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    const double bnorm = std::sqrt(dot(b, b, n));
    *iters = 0;
    if (cap > 0) res_hist[0] = bnorm > 0.0 ? 1.0 : 0.0;
    out[0] = 0.0;
    if (bnorm == 0.0) return 0;
    if (!std::isfinite(bnorm)) return 4;
    apply_op(*O, op, r.data(), z.data());
    double rz = dot(r.data(), z.data(), n);
    p = z;
    int status = 3;
    for (int k = 0; k < maxit; ++k) {
        if (!(rz > 0.0) || !std::isfinite(rz)) { status = 4; break; }
        spmv(O->A, p.data(), q.data());
        const double pq = dot(p.data(), q.data(), n);
        if (!(pq > 0.0) || !std::isfinite(pq)) { status = 4; break; }
        const double alpha = rz / pq;
#pragma omp parallel for schedule(static) if (n > 20000)
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        *iters = k + 1;
        const double res = std::sqrt(dot(r.data(), r.data(), n)) / bnorm;
        if (k < cap) alpha_out[k] = alpha;
        if (k + 1 < cap) res_hist[k + 1] = res;
        if (res < tol) { status = 0; break; }
        apply_op(*O, op, r.data(), z.data());
        const double rz_new = dot(r.data(), z.data(), n);
        const double beta = rz_new / rz;
        if (k < cap) beta_out[k] = beta;
#pragma omp parallel for schedule(static) if (n > 20000)
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
    vector<double> t(n);
    residual(O->A, b, x, t.data());
    out[0] = std::sqrt(dot(t.data(), t.data(), n)) / bnorm;
    return status;
}

}  // extern "C"
