// batched.cu -- PCG on K right-hand sides at once (independent columns in lockstep).
//
// Block vectors are row-major [n][Kp] (Kp = K rounded up to a multiple of 32), so one warp owns a
// row and its lanes own columns lane, lane + 32, ...: every matrix entry is one broadcast load
// shared by all K columns, and every gathered vector row is one coalesced load.  The matrix is read
// once per K solves instead of once per solve (SpMM).  Each column has its own alpha, beta and
// convergence flag; a converged column is frozen (alpha = 0) while the others continue, so each
// column reproduces the single-right-hand-side iteration.  Reductions are per column and finish in
// a fixed order.  The preconditioner is the handle's, applied column-wise by the same algorithms
// (Algorithm 2.1 with Algorithm 3.2 and the IC(0) solves).
#include <algorithm>
#include <type_traits>
#include <utility>

#include "device.cuh"
#include "handle.cuh"

namespace cpc {

namespace {

constexpr int BWARPS = 4;                 // rows (warps) per block
constexpr int BTPB = BWARPS * 32;
constexpr int NB_STATE = 12;              // per-column scalar slots

// column-state layout: S[slot * Kp + col]
enum { S_BNORM = 0, S_RZ, S_RZOLD, S_PQ, S_ALPHA, S_BETA, S_RES, S_ACTIVE, S_K, S_STATUS, S_TOL, S_MAXIT };

template <class MT, class DT>
struct BV {                               // SELL view for the batched kernels
    int C;
    const int* __restrict__ perm;
    const int* __restrict__ cptr;
    const int* __restrict__ col;
    const MT* __restrict__ val;
    const DT* __restrict__ diag;
};

template <class MT, class DT>
BV<MT, DT> bview(const Sell& S, const MT* val, const DT* diag) {
    return BV<MT, DT>{S.C, S.perm.p, S.cptr.p, S.col.p, val, diag};
}

template <class... KArgs, class... Args>
void blaunch(void (*k)(KArgs...), int grid, int block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)std::max(1, grid), 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CPC_CK(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
}

inline int rows_grid(int nrows) { return (nrows + BWARPS - 1) / BWARPS; }

// Calls f(std::integral_constant<int, ND>{}) with the padded diagonal count (4, 6 or 8).
template <class F>
void bwith_nd(int nd, F&& f) {
    if (nd <= 4) f(std::integral_constant<int, 4>{});
    else if (nd <= 6) f(std::integral_constant<int, 6>{});
    else f(std::integral_constant<int, 8>{});
}

// acc[j] += sum_w a_w x[col_w][lane + 32 j] over the entries of the row in slot s.  Padding entries
// (col < 0) sit at the end of a row.  Four entries are loaded before their gathers.
template <int J, class VT, class MT, class XT>
__device__ __forceinline__ void brow(const int* __restrict__ col, const MT* __restrict__ val, int C, int base,
                                     int width, int r, const XT* x, int Kp, int lane, VT (&acc)[J]) {
    int w = 0;
    for (; w + 4 <= width; w += 4) {
        int c[4];
        VT a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = col[base + (w + u) * C + r];
            a[u] = Cv<VT>::f(val[base + (w + u) * C + r]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] < 0) continue;
            const XT* xr = x + (size_t)c[u] * Kp + lane;
#pragma unroll
            for (int j = 0; j < J; ++j) acc[j] += a[u] * Cv<VT>::f(xr[32 * j]);
        }
    }
    for (; w < width; ++w) {
        const int c = col[base + w * C + r];
        if (c < 0) break;
        const VT a = Cv<VT>::f(val[base + w * C + r]);
        const XT* xr = x + (size_t)c * Kp + lane;
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] += a * Cv<VT>::f(xr[32 * j]);
    }
}

// brow with eight entries per batch (long rows): half the dependent rounds of brow.
template <int J, class VT, class MT, class XT>
__device__ __forceinline__ void brow8(const int* __restrict__ col, const MT* __restrict__ val, int C, int base,
                                      int width, int r, const XT* x, int Kp, int lane, VT (&acc)[J]) {
    int w = 0;
    for (; w + 8 <= width; w += 8) {
        int c[8];
        VT a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = col[base + (w + u) * C + r];
            a[u] = Cv<VT>::f(val[base + (w + u) * C + r]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (c[u] < 0) continue;
            const XT* xr = x + (size_t)c[u] * Kp + lane;
#pragma unroll
            for (int j = 0; j < J; ++j) acc[j] += a[u] * Cv<VT>::f(xr[32 * j]);
        }
    }
    brow<J, VT>(col, val, C, base + w * C, width - w, r, x, Kp, lane, acc);
}

// Gauss-Seidel over the slots [s0, s1) of one colour, all columns.
template <int J, class MT, class DT, class FT, class VT, bool LONG = false>
__global__ void __launch_bounds__(BTPB) kb_gs(BV<MT, DT> A, int s0, int s1, const FT* f, VT* x, int Kp) {
    const int s = s0 + blockIdx.x * BWARPS + (threadIdx.x >> 5);
    if (s >= s1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int row = A.perm[s];                   // matrix data: before the wait
    const int k = s / A.C, r = s % A.C;
    const int base = A.cptr[k];
    const int width = (A.cptr[k + 1] - base) / A.C;
    const VT dinv = Cv<VT>::f(A.diag[s]);        // the view's diagonal field holds 1 / a_ii
    pdl_wait();
    if (row < 0) return;
    VT acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = VT(0);
    if (LONG) brow8<J, VT>(A.col, A.val, A.C, base, width, r, x, Kp, lane, acc);
    else brow<J, VT>(A.col, A.val, A.C, base, width, r, x, Kp, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const size_t o = (size_t)row * Kp + lane + 32 * j;
        x[o] = (Cv<VT>::f(f[o]) - acc[j]) * dinv;
    }
}

// Gauss-Seidel for long rows in small colour groups (coarse levels): one block of BWARPS warps per
// row, warp w taking the entries w, w + BWARPS, ...; the warps' partial sums are added in warp
// order through shared memory.  A step of a few thousand rows then costs a quarter of a row's
// chain of dependent loads instead of a whole one.
template <int J, class MT, class DT, class FT, class VT>
__global__ void __launch_bounds__(BTPB) kb_gs_wide(BV<MT, DT> A, int s0, const FT* f, VT* x, int Kp) {
    __shared__ VT part[BWARPS][32 * J];
    const int s = s0 + blockIdx.x;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = A.perm[s];
    const int k = s / A.C, r = s % A.C;
    const int base = A.cptr[k];
    const int width = (A.cptr[k + 1] - base) / A.C;
    const VT dinv = Cv<VT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;                         // uniform over the block
    VT acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = VT(0);
    // entries w, w + BWARPS, ...: a strided view of the row (base + w C, step BWARPS C)
    const int mine = width > w ? (width - w + BWARPS - 1) / BWARPS : 0;
    brow<J, VT>(A.col, A.val, A.C * BWARPS, base + w * A.C, mine, r, x, Kp, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) part[w][lane + 32 * j] = acc[j];
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        VT t = part[0][lane + 32 * j];
        for (int q = 1; q < BWARPS; ++q) t += part[q][lane + 32 * j];
        const size_t o = (size_t)row * Kp + lane + 32 * j;
        x[o] = (Cv<VT>::f(f[o]) - t) * dinv;
    }
}

// out = f - A x (resid) over all slots; with DIAG the split diagonal is included.
template <int J, class MT, class DT, class FT, class XT, class RT>
__global__ void __launch_bounds__(BTPB) kb_resid(BV<MT, DT> A, int nslots, const FT* f,
                                                  const XT* x, RT* __restrict__ out, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < nslots; s += gridDim.x * BWARPS) {
        const int row = A.perm[s];
        if (row < 0) continue;
        const int k = s / A.C, r = s % A.C;
        const int base = A.cptr[k];
        RT acc[J];
        const RT d = Cv<RT>::f(A.diag[s]);
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = d * Cv<RT>::f(x[(size_t)row * Kp + lane + 32 * j]);
        brow<J, RT>(A.col, A.val, A.C, base, (A.cptr[k + 1] - base) / A.C, r, x, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            out[o] = Cv<RT>::f(f[o]) - acc[j];
        }
    }
}

// y = M x for full rows (restriction), optionally zeroing yz (the next level's initial guess).
template <int J, class MT, class VT>
__global__ void __launch_bounds__(BTPB) kb_apply(BV<MT, MT> M, int nslots, const VT* x,
                                                  VT* __restrict__ y, VT* __restrict__ yz, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < nslots; s += gridDim.x * BWARPS) {
        const int row = M.perm[s];
        if (row < 0) continue;
        const int k = s / M.C, r = s % M.C;
        const int base = M.cptr[k];
        VT acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = VT(0);
        brow<J, VT>(M.col, M.val, M.C, base, (M.cptr[k + 1] - base) / M.C, r, x, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            y[o] = acc[j];
            if (yz) yz[o] = VT(0);
        }
    }
}

// x += P e
template <int J, class MT, class VT>
__global__ void __launch_bounds__(BTPB) kb_prolong(BV<MT, MT> P, int nslots, const VT* e,
                                                    VT* __restrict__ x, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < nslots; s += gridDim.x * BWARPS) {
        const int row = P.perm[s];
        if (row < 0) continue;
        const int k = s / P.C, r = s % P.C;
        const int base = P.cptr[k];
        VT acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = VT(0);
        brow<J, VT>(P.col, P.val, P.C, base, (P.cptr[k + 1] - base) / P.C, r, e, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) x[(size_t)row * Kp + lane + 32 * j] += acc[j];
    }
}

// x = A_c^{-1} f (dense), one warp per row, lanes over columns.
template <int J, class AT, class FT, class VT>
__global__ void __launch_bounds__(BTPB) kb_coarse(int n, const AT* __restrict__ Ainv, const FT* f,
                                                   VT* __restrict__ x, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * BWARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * BWARPS) {
        VT acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = VT(0);
        for (int m = 0; m < n; ++m) {
            const VT a = Cv<VT>::f(Ainv[(size_t)i * n + m]);
#pragma unroll
            for (int j = 0; j < J; ++j) acc[j] += a * Cv<VT>::f(f[(size_t)m * Kp + lane + 32 * j]);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) x[(size_t)i * Kp + lane + 32 * j] = acc[j];
    }
}

template <class VT>
__global__ void kb_zero(int64_t n, VT* x) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = VT(0);
}

// Triangular solves of one IC(0) level, all columns: y = t - L y; w = (y - U w) / d, z += w.
template <int J, class MT, class TT, class VT>
__global__ void __launch_bounds__(BTPB) kb_lsolve(BV<MT, MT> L, int s0, int s1, const TT* t, VT* y, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int s = s0 + blockIdx.x * BWARPS + (threadIdx.x >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31;
    const int row = L.perm[s];
    if (row < 0) return;
    const int k = s / L.C, r = s % L.C;
    const int base = L.cptr[k];
    VT acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = VT(0);
    brow<J, VT>(L.col, L.val, L.C, base, (L.cptr[k + 1] - base) / L.C, r, y, Kp, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const size_t o = (size_t)row * Kp + lane + 32 * j;
        y[o] = Cv<VT>::f(t[o]) - acc[j];
    }
}

template <int J, class MT, class VT>
__global__ void __launch_bounds__(BTPB) kb_usolve(BV<MT, MT> U, int s0, int s1, const VT* y, VT* w,
                                                   VT* zadd, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int s = s0 + blockIdx.x * BWARPS + (threadIdx.x >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31;
    const int row = U.perm[s];
    if (row < 0) return;
    const int k = s / U.C, r = s % U.C;
    const int base = U.cptr[k];
    VT acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = VT(0);
    brow<J, VT>(U.col, U.val, U.C, base, (U.cptr[k + 1] - base) / U.C, r, w, Kp, lane, acc);
    const VT dinv = Cv<VT>::f(U.diag[s]);        // 1 / u_ii
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const size_t o = (size_t)row * Kp + lane + 32 * j;
        const VT v = (y[o] - acc[j]) * dinv;
        w[o] = v;
        if (zadd) zadd[o] += v;
    }
}

// ---------------------------------------------------------------------------------------------
// Diagonal form (Sell::ndiag > 0, structured fine level): the gathered rows are x[i + off_d], so a
// warp needs only its row index before it issues every gather, and the matrix values (one
// broadcast load per diagonal) and 1 / a_ii are loaded before griddepcontrol.wait.  Products are
// added in ascending column order, as in brow.
// ---------------------------------------------------------------------------------------------
template <class MT, class DT>
struct BD {
    int n, nslots;
    const int* __restrict__ perm;      // nullptr: natural order
    const MT* __restrict__ val;        // [ND][nslots]
    const DT* __restrict__ diag;
    DiaOff off;
};

template <class MT, class DT>
BD<MT, DT> bdview(const Sell& S, int n, const MT* val, const DT* diag, bool natural) {
    return BD<MT, DT>{n, S.nslots, natural ? nullptr : S.perm.p, val, diag, S.doff};
}

template <class MT, class DT>
__device__ __forceinline__ int bd_row(const BD<MT, DT>& A, int s) {
    return A.perm ? A.perm[s] : (s < A.n ? s : -1);
}

// acc[j] += sum_d v_d x[i + off_d][lane + 32 j] (all gathers issued before the products)
template <int J, int ND, class VT, class XT>
__device__ __forceinline__ void bd_dot(const VT (&v)[ND], const DiaOff& off, int row, int n, const XT* x, int Kp,
                                       int lane, VT (&acc)[J]) {
    VT xv[ND][J];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        int jr = row + off.o[d];
        jr = jr < 0 ? 0 : (jr >= n ? n - 1 : jr);
        const XT* xr = x + (size_t)jr * Kp + lane;
#pragma unroll
        for (int j = 0; j < J; ++j) xv[d][j] = Cv<VT>::f(xr[32 * j]);
    }
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] += v[d] * xv[d][j];
}

template <int J, class MT, class DT, class FT, class VT, int ND>
__global__ void __launch_bounds__(BTPB) kb_gs_dia(BD<MT, DT> A, int s0, int s1, const FT* f, VT* x, int Kp) {
    const int s = s0 + blockIdx.x * BWARPS + (threadIdx.x >> 5);
    if (s >= s1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int row = bd_row(A, s);
    VT v[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = Cv<VT>::f(A.val[(size_t)d * A.nslots + s]);
    const VT dinv = Cv<VT>::f(A.diag[s]);        // 1 / a_ii
    pdl_wait();
    if (row < 0) return;
    VT fr[J], acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        fr[j] = Cv<VT>::f(f[(size_t)row * Kp + lane + 32 * j]);
        acc[j] = VT(0);
    }
    bd_dot<J, ND>(v, A.off, row, A.n, x, Kp, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) x[(size_t)row * Kp + lane + 32 * j] = (fr[j] - acc[j]) * dinv;
}

// out = f - A x, diagonal form (grid-stride over slots).
template <int J, class MT, class DT, class FT, class XT, class RT, int ND>
__global__ void __launch_bounds__(BTPB) kb_resid_dia(BD<MT, DT> A, const FT* f, const XT* x,
                                                      RT* __restrict__ out, int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < A.nslots; s += gridDim.x * BWARPS) {
        const int row = bd_row(A, s);
        if (row < 0) continue;
        RT v[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) v[d] = Cv<RT>::f(A.val[(size_t)d * A.nslots + s]);
        const RT dg = Cv<RT>::f(A.diag[s]);
        RT acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = dg * Cv<RT>::f(x[(size_t)row * Kp + lane + 32 * j]);
        bd_dot<J, ND>(v, A.off, row, A.n, x, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            out[o] = Cv<RT>::f(f[o]) - acc[j];
        }
    }
}

// B_co step (2) with red-black IC(0), black rows only (see the single right-hand-side path):
// z_b += (r_b - (A z)_b) / u_bb on the fine colour 1, diagonal form.
template <int J, class MT, class DT, class VT, int ND>
__global__ void __launch_bounds__(BTPB) kb_bco_black_dia(BD<MT, DT> A, int s0, int s1, const double* r,
                                                          const VT* __restrict__ uinv, VT* __restrict__ z, int Kp) {
    const int s = s0 + blockIdx.x * BWARPS + (threadIdx.x >> 5);
    if (s >= s1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int row = bd_row(A, s);
    VT v[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = Cv<VT>::f(A.val[(size_t)d * A.nslots + s]);
    const VT dg = Cv<VT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const VT ui = uinv[row];
    VT zr[J], acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        zr[j] = z[(size_t)row * Kp + lane + 32 * j];
        acc[j] = dg * zr[j];
    }
    bd_dot<J, ND>(v, A.off, row, A.n, z, Kp, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const size_t o = (size_t)row * Kp + lane + 32 * j;
        z[o] = zr[j] + (Cv<VT>::f(r[o]) - acc[j]) * ui;
    }
}

// First colour step of a sweep from a zero guess fused with the zero fill: x = f / a_ii on colour 0,
// 0 elsewhere (colour-0 rows see only zeros).
template <class FT, class VT>
__global__ void kb_zero_first(int n, int Kp, const FT* f, const int* __restrict__ colour,
                              const VT* __restrict__ dnat, VT* __restrict__ x) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * Kp;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / Kp);
        x[t] = colour[i] == 0 ? Cv<VT>::f(f[t]) * dnat[i] : VT(0);
    }
}

// f_c = R r and the coarse level's first colour step from zero: x_c = f_c / a_ii on colour 0, 0 elsewhere.
template <int J, class MT, class VT>
__global__ void __launch_bounds__(BTPB) kb_restrict_first(BV<MT, MT> M, int nslots, const VT* x,
                                                           VT* __restrict__ y, VT* __restrict__ yx,
                                                           const int* __restrict__ colour, const VT* __restrict__ dnat,
                                                           int Kp) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < nslots; s += gridDim.x * BWARPS) {
        const int row = M.perm[s];
        if (row < 0) continue;
        const int k = s / M.C, r = s % M.C;
        const int base = M.cptr[k];
        const bool c0 = colour[row] == 0;
        const VT dr = dnat[row];
        VT acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = VT(0);
        brow<J, VT>(M.col, M.val, M.C, base, (M.cptr[k + 1] - base) / M.C, r, x, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            y[o] = acc[j];
            yx[o] = c0 ? acc[j] * dr : VT(0);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Per-column reductions: each block sums its rows per column (warps, then in order), writes a
// partial row; the last block sums the partial rows in block order and runs `fin` per column.
// ---------------------------------------------------------------------------------------------
template <int J, class Fin>
__device__ void col_finish(double (&v)[J], double* part, unsigned* ctr, int Kp, Fin fin) {
    __shared__ double sh[BWARPS][128];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < J; ++j) sh[w][lane + 32 * j] = v[j];
    __syncthreads();
    for (int c = threadIdx.x; c < Kp; c += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < BWARPS; ++q) t += sh[q][c];
        part[(size_t)blockIdx.x * Kp + c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int c = threadIdx.x; c < Kp; c += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&part[(size_t)b * Kp + c]);
        fin(c, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

template <int J>
__global__ void __launch_bounds__(BTPB) kb_init(int n, int Kp, const double* b, double* __restrict__ x,
                                                 double* __restrict__ r, double* part, unsigned* ctr, double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j] = 0.0;
    for (int i = blockIdx.x * BWARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * BWARPS) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)i * Kp + lane + 32 * j;
            const double bi = b[o];
            x[o] = 0.0;
            r[o] = bi;
            v[j] += bi * bi;
        }
    }
    col_finish<J>(v, part, ctr, Kp, [&](int c, double t) {
        const double bn = sqrt(t);
        S[S_BNORM * Kp + c] = bn;
        S[S_K * Kp + c] = 0.0;
        S[S_RZOLD * Kp + c] = 0.0;
        S[S_BETA * Kp + c] = 0.0;
        S[S_ALPHA * Kp + c] = 0.0;
        S[S_RES * Kp + c] = bn > 0.0 ? 1.0 : 0.0;
        const bool ok = isfinite(bn);
        S[S_STATUS * Kp + c] = ok ? (bn > 0.0 && S[S_MAXIT * Kp + c] <= 0.0 ? CPC_ENOCONV : CPC_OK) : CPC_EBREAKDOWN;
        S[S_ACTIVE * Kp + c] = (ok && bn > 0.0 && S[S_MAXIT * Kp + c] > 0.0) ? 1.0 : 0.0;
    });
}

// Any column still active?  Sets the loop condition (one thread).
__global__ void kb_any_active(int Kp, const double* S, cudaGraphConditionalHandle cond) {
    pdl_launch_dependents();
    pdl_wait();
    unsigned go = 0u;
    for (int c = 0; c < Kp; ++c) go |= S[S_ACTIVE * Kp + c] > 0.0 ? 1u : 0u;
    cudaGraphSetConditional(cond, go);
}

__global__ void kb_guard(cudaGraphConditionalHandle cond) {
    pdl_launch_dependents();
    pdl_wait();
    cudaGraphSetConditional(cond, 0u);
}

template <int J, class ZT>
__global__ void __launch_bounds__(BTPB) kb_rz(int n, int Kp, const double* r, const ZT* z,
                                               double* part, unsigned* ctr, double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j] = 0.0;
    for (int i = blockIdx.x * BWARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * BWARPS) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)i * Kp + lane + 32 * j;
            v[j] += r[o] * cvt_d(z[o]);
        }
    }
    col_finish<J>(v, part, ctr, Kp, [&](int c, double t) {
        const bool act = S[S_ACTIVE * Kp + c] > 0.0;
        if (act && (!(t > 0.0) || !isfinite(t))) {
            S[S_STATUS * Kp + c] = CPC_EBREAKDOWN;
            S[S_ACTIVE * Kp + c] = 0.0;
        }
        S[S_BETA * Kp + c] = (S[S_K * Kp + c] == 0.0 || !act) ? 0.0 : t / S[S_RZOLD * Kp + c];
        S[S_RZ * Kp + c] = t;
        S[S_RZOLD * Kp + c] = t;
    });
}

template <int J, class ZT>
__global__ void __launch_bounds__(BTPB) kb_p(int n, int Kp, const ZT* z, double* __restrict__ p,
                                              const double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double beta[J];
    bool first[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        beta[j] = S[S_BETA * Kp + lane + 32 * j];
        first[j] = S[S_K * Kp + lane + 32 * j] == 0.0;
    }
    for (int i = blockIdx.x * BWARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * BWARPS) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)i * Kp + lane + 32 * j;
            p[o] = first[j] ? cvt_d(z[o]) : cvt_d(z[o]) + beta[j] * p[o];
        }
    }
}

template <int J>
__global__ void __launch_bounds__(BTPB) kb_spmv_pq(BV<double, double> A, int nslots, int Kp, const double* p,
                                                    double* __restrict__ q, double* part, unsigned* ctr, double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j] = 0.0;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < nslots; s += gridDim.x * BWARPS) {
        const int row = A.perm[s];
        if (row < 0) continue;
        const int k = s / A.C, r = s % A.C;
        const int base = A.cptr[k];
        double acc[J];
        const double d = A.diag[s];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = d * p[(size_t)row * Kp + lane + 32 * j];
        brow<J, double>(A.col, A.val, A.C, base, (A.cptr[k + 1] - base) / A.C, r, p, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            q[o] = acc[j];
            v[j] += p[o] * acc[j];
        }
    }
    col_finish<J>(v, part, ctr, Kp, [&](int c, double t) {
        const bool act = S[S_ACTIVE * Kp + c] > 0.0;
        S[S_PQ * Kp + c] = t;
        if (act && (!(t > 0.0) || !isfinite(t))) {
            S[S_STATUS * Kp + c] = CPC_EBREAKDOWN;
            S[S_ACTIVE * Kp + c] = 0.0;
        }
        S[S_ALPHA * Kp + c] = S[S_ACTIVE * Kp + c] > 0.0 ? S[S_RZ * Kp + c] / t : 0.0;
    });
}

template <int J, int ND>
__global__ void __launch_bounds__(BTPB) kb_spmv_pq_dia(BD<double, double> A, int Kp, const double* p,
                                                        double* __restrict__ q, double* part, unsigned* ctr, double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j] = 0.0;
    for (int s = blockIdx.x * BWARPS + (threadIdx.x >> 5); s < A.nslots; s += gridDim.x * BWARPS) {
        const int row = bd_row(A, s);
        if (row < 0) continue;
        double w[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) w[d] = A.val[(size_t)d * A.nslots + s];
        const double dg = A.diag[s];
        double acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = dg * p[(size_t)row * Kp + lane + 32 * j];
        bd_dot<J, ND>(w, A.off, row, A.n, p, Kp, lane, acc);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)row * Kp + lane + 32 * j;
            q[o] = acc[j];
            v[j] += p[o] * acc[j];
        }
    }
    col_finish<J>(v, part, ctr, Kp, [&](int c, double t) {
        const bool act = S[S_ACTIVE * Kp + c] > 0.0;
        S[S_PQ * Kp + c] = t;
        if (act && (!(t > 0.0) || !isfinite(t))) {
            S[S_STATUS * Kp + c] = CPC_EBREAKDOWN;
            S[S_ACTIVE * Kp + c] = 0.0;
        }
        S[S_ALPHA * Kp + c] = S[S_ACTIVE * Kp + c] > 0.0 ? S[S_RZ * Kp + c] / t : 0.0;
    });
}

template <int J>
__global__ void __launch_bounds__(BTPB) kb_update(int n, int Kp, double* __restrict__ x, double* __restrict__ r,
                                                   const double* p, const double* q,
                                                   double* part, unsigned* ctr, double* S) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    double alpha[J], v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        alpha[j] = S[S_ALPHA * Kp + lane + 32 * j];
        v[j] = 0.0;
    }
    for (int i = blockIdx.x * BWARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * BWARPS) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const size_t o = (size_t)i * Kp + lane + 32 * j;
            x[o] += alpha[j] * p[o];
            const double ri = r[o] - alpha[j] * q[o];
            r[o] = ri;
            v[j] += ri * ri;
        }
    }
    col_finish<J>(v, part, ctr, Kp, [&](int c, double t) {
        if (S[S_ACTIVE * Kp + c] <= 0.0) return;
        const double k = S[S_K * Kp + c] + 1.0;
        S[S_K * Kp + c] = k;
        const double res = sqrt(t) / S[S_BNORM * Kp + c];
        S[S_RES * Kp + c] = res;
        if (!isfinite(res)) { S[S_STATUS * Kp + c] = CPC_EBREAKDOWN; S[S_ACTIVE * Kp + c] = 0.0; }
        else if (res < S[S_TOL * Kp + c]) { S[S_STATUS * Kp + c] = CPC_OK; S[S_ACTIVE * Kp + c] = 0.0; }
        else if (k >= S[S_MAXIT * Kp + c]) { S[S_STATUS * Kp + c] = CPC_ENOCONV; S[S_ACTIVE * Kp + c] = 0.0; }
    });
}

// [n][K] user layout <-> [n][Kp] internal layout
__global__ void kb_pack(int n, int K, int Kp, const double* in, double* __restrict__ out) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * Kp; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / Kp;
        const int c = (int)(t % Kp);
        out[t] = c < K ? in[i * K + c] : 0.0;
    }
}

__global__ void kb_unpack(int n, int K, int Kp, const double* in, double* __restrict__ out) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / K;
        const int c = (int)(t % K);
        out[t] = in[i * Kp + c];
    }
}

// Adjoint sources from the forward solutions: b[i][c] = x[i][c] where b[i][c] != 0, else 0
// (the gradient of J_c = 1/2 sum over the source cells of column c of x^2); also saves x.
__global__ void kb_adjoint_rhs(int64_t nk, double* __restrict__ b, const double* x, double* __restrict__ xsave) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nk; t += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[t];
        xsave[t] = xi;
        b[t] = b[t] != 0.0 ? xi : 0.0;
    }
}

// ---------------------------------------------------------------------------------------------
// Recording (column-wise V-cycle, IC(0), B_co)
// ---------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------------
// Block PCG (O'Leary 1980): the K columns share one block Krylov space through K x K matrices.
// Not a method of the paper; the coupled counterpart of the batched solve above.  All K x K
// arithmetic is FP64 and every sum finishes in a fixed order.
// ------------------------------------------------------------------------------------------------
constexpr int KK_TPB = 256;
constexpr int KK_ROWS = 32;               // rows staged per step of kk_gram
constexpr int KK_GRID = 152 * 2;          // blocks of kk_gram / kk_update / kk_colnorm (fixed)
enum { KM_PQ = 0, KM_GAMMA, KM_GAMMA_NEW, KM_ALPHA, KM_BETA, KM_COUNT };
enum { KV_BNORM = 0, KV_RES, KV_COUNT };
enum { KF_BAD = 0, KF_DONE, KF_COUNT };

// part[block] = U^T V over the block's rows, on the 4 x 4 tiles (ti, tj) with ti <= tj of the
// Kp x Kp result (Kp = 32 or 64); U is Z (preconditioner precision) or P, V is R or Q (FP64).
// Thread t owns the t-th upper tile in row-major order, so the T (T + 1) / 2 active threads fill
// whole warps: an FP64 warp instruction costs the same with idle lanes, and FP64 issue is the
// bound of this kernel on this part.
template <class UT>
__global__ void __launch_bounds__(KK_TPB) kk_gram(int n, int Kp, const UT* U,
                                                  const double* V, double* __restrict__ part) {
    extern __shared__ double ksm[];
    double* us = ksm;                      // [KK_ROWS][Kp]
    double* vs = ksm + KK_ROWS * Kp;       // [KK_ROWS][Kp]
    const int T = Kp / 4, t = threadIdx.x;
    int ti = 0, rem = t;
    while (ti < T && rem >= T - ti) {
        rem -= T - ti;
        ++ti;
    }
    const int tj = ti + rem;
    const bool act = ti < T;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = min(n, blockIdx.x * per), r1 = min(n, r0 + per);
    for (int base = r0; base < r1; base += KK_ROWS) {
        const int rows = min(KK_ROWS, r1 - base);
        __syncthreads();
        for (int e = t; e < KK_ROWS * Kp; e += KK_TPB) {
            const int rr = e / Kp;
            const size_t g = (size_t)base * Kp + e;
            us[e] = rr < rows ? (double)U[g] : 0.0;
            vs[e] = rr < rows ? V[g] : 0.0;
        }
        __syncthreads();
        if (act) {
            for (int rr = 0; rr < rows; ++rr) {
                double a[4], c[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = us[rr * Kp + ti * 4 + q];
                    c[q] = vs[rr * Kp + tj * 4 + q];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int w = 0; w < 4; ++w) acc[q][w] = __fma_rn(a[q], c[w], acc[q][w]);
            }
        }
    }
    if (act)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) part[((size_t)blockIdx.x * Kp + ti * 4 + q) * Kp + tj * 4 + w] = acc[q][w];
}

// out = sum over blocks of part, in block order; entry (i, j) and (j, i) both take the computed
// upper entry (min, max), so the result is exactly symmetric.
__global__ void kk_gram_sum(int G, int Kp, const double* part, double* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Kp * Kp; e += gridDim.x * blockDim.x) {
        const int i = e / Kp, j = e - (e / Kp) * Kp;
        const int a = min(i, j), b = max(i, j);
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part[((size_t)g * Kp + a) * Kp + b];
        out[e] = s;
    }
}

// Y = S^{-1} W on the leading K x K blocks by Cholesky S = L L^T (one block; S symmetric).  out is
// Kp x Kp with zeros outside K x K.  A pivot that is not finite or at most 1e-12 times its diagonal
// entry s_kk (a block column within rounding of the span of the others) sets flag[KF_BAD].
// With copy_to, W is copied there afterwards (gamma_old <- gamma_new).
__global__ void __launch_bounds__(KK_TPB) kk_solve(int K, int Kp, const double* S, const double* W,
                                                   double* __restrict__ out, double* copy_to, int* flag) {
    extern __shared__ double ksm[];
    double* L = ksm;                       // [K][K]
    double* Y = ksm + K * K;               // [K][K]
    __shared__ int bad;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) bad = 0;
    for (int e = t; e < K * K; e += nt) {
        const int i = e / K, j = e - (e / K) * K;
        L[e] = S[(size_t)i * Kp + j];
        Y[e] = W[(size_t)i * Kp + j];
    }
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        if (t == 0) {
            const double d = L[k * K + k];
            if (!(d > 1e-12 * S[(size_t)k * Kp + k]) || !isfinite(d)) bad = 1;
            L[k * K + k] = sqrt(d > 0.0 && isfinite(d) ? d : 1.0);
        }
        __syncthreads();
        const double dk = L[k * K + k];
        for (int i = k + 1 + t; i < K; i += nt) L[i * K + k] /= dk;
        __syncthreads();
        const int m = K - k - 1;
        for (int e = t; e < m * m; e += nt) {
            const int i = k + 1 + e / m, j = k + 1 + (e - (e / m) * m);
            if (j <= i) L[i * K + j] -= L[i * K + k] * L[j * K + k];
        }
        __syncthreads();
    }
    for (int c = t; c < K; c += nt) {      // one right-hand-side column per thread
        for (int i = 0; i < K; ++i) {      // L z = w
            double s = Y[i * K + c];
            for (int q = 0; q < i; ++q) s -= L[i * K + q] * Y[q * K + c];
            Y[i * K + c] = s / L[i * K + i];
        }
        for (int i = K - 1; i >= 0; --i) { // L^T y = z
            double s = Y[i * K + c];
            for (int q = i + 1; q < K; ++q) s -= L[q * K + i] * Y[q * K + c];
            Y[i * K + c] = s / L[i * K + i];
        }
    }
    __syncthreads();
    for (int e = t; e < Kp * Kp; e += nt) {
        const int i = e / Kp, j = e - (e / Kp) * Kp;
        out[e] = (i < K && j < K) ? Y[i * K + j] : 0.0;
        if (copy_to) copy_to[e] = W[e];
    }
    if (t == 0 && bad) flag[KF_BAD] = 1;
}

// Entry k of a row held across the warp (lane k mod 32 of register k / 32).
template <int J>
__device__ __forceinline__ double kk_lane(const double (&v)[J], int k) {
    if constexpr (J == 1) return __shfl_sync(0xffffffffu, v[0], k & 31);
    else return __shfl_sync(0xffffffffu, k < 32 ? v[0] : v[1], k & 31);
}

// X += P alpha and R -= Q alpha (warp per row, lanes over columns, alpha in shared memory), and
// per block the column sums of r_ij^2 in warp order into part[block][Kp].
template <int J>
__global__ void __launch_bounds__(BTPB) kk_update(int n, int Kp, int K, double* __restrict__ X, double* __restrict__ R,
                                                  const double* P, const double* Q,
                                                  const double* alpha, double* __restrict__ part,
                                                  const int* flag) {
    if (flag[KF_BAD]) return;              // a K x K solve failed: keep the last good iterate
    extern __shared__ double ksm[];
    double* al = ksm;                      // [Kp][Kp]
    double* ws = ksm + Kp * Kp;            // [BWARPS][Kp]
    for (int e = threadIdx.x; e < Kp * Kp; e += blockDim.x) al[e] = alpha[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double rr[J];
#pragma unroll
    for (int m = 0; m < J; ++m) rr[m] = 0.0;
    for (int i = blockIdx.x * BWARPS + w; i < n; i += gridDim.x * BWARPS) {
        const size_t o = (size_t)i * Kp + lane;
        double p[J], q[J], dx[J], dr[J];
#pragma unroll
        for (int m = 0; m < J; ++m) {
            p[m] = P[o + 32 * m];
            q[m] = Q[o + 32 * m];
            dx[m] = 0.0;
            dr[m] = 0.0;
        }
        for (int k = 0; k < K; ++k) {
            const double pk = kk_lane<J>(p, k), qk = kk_lane<J>(q, k);
#pragma unroll
            for (int m = 0; m < J; ++m) {
                const double a = al[k * Kp + lane + 32 * m];
                dx[m] = __fma_rn(pk, a, dx[m]);
                dr[m] = __fma_rn(qk, a, dr[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < J; ++m) {
            X[o + 32 * m] += dx[m];
            const double r = R[o + 32 * m] - dr[m];
            R[o + 32 * m] = r;
            rr[m] = __fma_rn(r, r, rr[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < J; ++m) ws[w * Kp + lane + 32 * m] = rr[m];
    __syncthreads();
    for (int c = threadIdx.x; c < Kp; c += blockDim.x) {
        double s = 0.0;
        for (int v = 0; v < BWARPS; ++v) s += ws[v * Kp + c];
        part[(size_t)blockIdx.x * Kp + c] = s;
    }
}

// P = Z + P beta, in place (a warp reads its whole row of P before writing it).
template <int J, class ZT>
__global__ void __launch_bounds__(BTPB) kk_pupdate(int n, int Kp, int K, const ZT* Z, double* __restrict__ P,
                                                   const double* beta, const int* flag) {
    if (flag[KF_BAD]) return;
    extern __shared__ double ksm[];
    for (int e = threadIdx.x; e < Kp * Kp; e += blockDim.x) ksm[e] = beta[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = blockIdx.x * BWARPS + w; i < n; i += gridDim.x * BWARPS) {
        const size_t o = (size_t)i * Kp + lane;
        double p[J], acc[J];
#pragma unroll
        for (int m = 0; m < J; ++m) {
            p[m] = P[o + 32 * m];
            acc[m] = 0.0;
        }
        for (int k = 0; k < K; ++k) {
            const double pk = kk_lane<J>(p, k);
#pragma unroll
            for (int m = 0; m < J; ++m) acc[m] = __fma_rn(pk, ksm[k * Kp + lane + 32 * m], acc[m]);
        }
#pragma unroll
        for (int m = 0; m < J; ++m) P[o + 32 * m] = (double)Z[o + 32 * m] + acc[m];
    }
}

template <class ZT>
__global__ void kk_copy(int64_t nk, const ZT* z, double* __restrict__ p) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = (double)z[e];
}

// Q = A P with A in CSR (warp per row, lanes over columns).
template <int J>
__global__ void __launch_bounds__(BTPB) kk_spmm(int n, int Kp, const int* __restrict__ ptr, const int* __restrict__ col,
                                                const double* __restrict__ val, const double* P,
                                                double* __restrict__ Q) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = blockIdx.x * BWARPS + w; i < n; i += gridDim.x * BWARPS) {
        double acc[J];
#pragma unroll
        for (int m = 0; m < J; ++m) acc[m] = 0.0;
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
            const double a = val[e];
            const size_t o = (size_t)col[e] * Kp + lane;
#pragma unroll
            for (int m = 0; m < J; ++m) acc[m] = __fma_rn(a, P[o + 32 * m], acc[m]);
        }
#pragma unroll
        for (int m = 0; m < J; ++m) Q[(size_t)i * Kp + lane + 32 * m] = acc[m];
    }
}

// Per block, the column sums of v_ij^2 in warp order into part[block][Kp].
template <int J>
__global__ void __launch_bounds__(BTPB) kk_colnorm(int n, int Kp, const double* V, double* __restrict__ part) {
    __shared__ double ws[BWARPS * 128];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double s[J];
#pragma unroll
    for (int m = 0; m < J; ++m) s[m] = 0.0;
    for (int i = blockIdx.x * BWARPS + w; i < n; i += gridDim.x * BWARPS)
#pragma unroll
        for (int m = 0; m < J; ++m) {
            const double v = V[(size_t)i * Kp + lane + 32 * m];
            s[m] = __fma_rn(v, v, s[m]);
        }
#pragma unroll
    for (int m = 0; m < J; ++m) ws[w * Kp + lane + 32 * m] = s[m];
    __syncthreads();
    for (int c = threadIdx.x; c < Kp; c += blockDim.x) {
        double t = 0.0;
        for (int v = 0; v < BWARPS; ++v) t += ws[v * Kp + c];
        part[(size_t)blockIdx.x * Kp + c] = t;
    }
}

// One block.  Column norms from the partials (block order).  init: bnorm_k = ||b_k||, a zero column
// sets KF_BAD.  Otherwise res_k = ||r_k|| / ||b_k||; KF_DONE = 1 when every column is below tol,
// and a residual that is not finite sets KF_BAD.
__global__ void kk_check(int G, int Kp, int K, const double* part, double* __restrict__ vec, double tol,
                         int init, int* flag) {
    __shared__ int all;
    if (threadIdx.x == 0) all = 1;
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part[(size_t)g * Kp + c];
        const double nrm = sqrt(s);
        if (init) {
            vec[KV_BNORM * Kp + c] = nrm;
            if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(&flag[KF_BAD], 1);
        } else {
            const double r = nrm / vec[KV_BNORM * Kp + c];
            vec[KV_RES * Kp + c] = r;
            if (!isfinite(r)) atomicOr(&flag[KF_BAD], 1);
            if (!(r < tol)) atomicAnd(&all, 0);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !init) flag[KF_DONE] = all;
}

template <class VT> VT* bx(Batched& B, int l) { return (VT*)B.lx[l].p; }
template <class VT> VT* bf(Batched& B, int l) { return (VT*)B.lf[l].p; }
template <class VT> VT* br(Batched& B, int l) { return (VT*)B.lr[l].p; }

template <int J, class FT, class VT>
void brec_gs(Level& L, int c, const FT* f, VT* x, int Kp, cudaStream_t s) {
    const int s0 = L.S.seg[c] * L.S.C, s1 = L.S.seg[c + 1] * L.S.C;
    if (s1 <= s0) return;
    const int g = rows_grid(s1 - s0);
    if (L.S.ndiag) {
        bwith_nd(L.S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                blaunch(kb_gs_dia<J, double, double, FT, VT, ND>, g, BTPB, s,
                        bdview(L.S, L.n, (const double*)L.S.dval.p, (const double*)L.S.dinv.p, false), s0, s1, f, x, Kp);
            else
                blaunch(kb_gs_dia<J, float, float, FT, VT, ND>, g, BTPB, s,
                        bdview(L.S, L.n, (const float*)L.S.dval32.p, (const float*)L.S.dinv32.p, false), s0, s1, f, x, Kp);
        });
        return;
    }
    // long rows in a small colour group: a block per row (kb_gs_wide), else a warp per row
    const bool wide = L.A.nnz >= (int64_t)16 * L.n && (s1 - s0) <= 16384;
    if (wide) {
        if constexpr (std::is_same<VT, double>::value)
            blaunch(kb_gs_wide<J, double, double, FT, VT>, s1 - s0, BTPB, s, bview(L.S, (const double*)L.S.val.p, (const double*)L.S.dinv.p), s0, f, x, Kp);
        else if (L.vt == VT_BF16)
            blaunch(kb_gs_wide<J, __nv_bfloat16, float, FT, VT>, s1 - s0, BTPB, s, bview(L.S, (const __nv_bfloat16*)L.S.val16.p, (const float*)L.S.dinv32.p), s0, f, x, Kp);
        else
            blaunch(kb_gs_wide<J, float, float, FT, VT>, s1 - s0, BTPB, s, bview(L.S, (const float*)L.S.val32.p, (const float*)L.S.dinv32.p), s0, f, x, Kp);
        return;
    }
    auto go = [&](auto longrows) {
        constexpr bool LG = decltype(longrows)::value;
        if constexpr (std::is_same<VT, double>::value)
            blaunch(kb_gs<J, double, double, FT, VT, LG>, g, BTPB, s, bview(L.S, (const double*)L.S.val.p, (const double*)L.S.dinv.p), s0, s1, f, x, Kp);
        else if (L.vt == VT_BF16)
            blaunch(kb_gs<J, __nv_bfloat16, float, FT, VT, LG>, g, BTPB, s, bview(L.S, (const __nv_bfloat16*)L.S.val16.p, (const float*)L.S.dinv32.p), s0, s1, f, x, Kp);
        else
            blaunch(kb_gs<J, float, float, FT, VT, LG>, g, BTPB, s, bview(L.S, (const float*)L.S.val32.p, (const float*)L.S.dinv32.p), s0, s1, f, x, Kp);
    };
    if (L.A.nnz >= (int64_t)16 * L.n) go(std::true_type{});   // long rows: eight entries per batch
    else go(std::false_type{});
}

template <int J, class FT, class VT>
void brec_resid(Level& L, const FT* f, const VT* x, VT* r, int Kp, cudaStream_t s) {
    const int g = std::min(rows_grid(L.S.nslots), 152 * 32);
    if (L.S.ndiag) {
        bwith_nd(L.S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                blaunch(kb_resid_dia<J, double, double, FT, VT, VT, ND>, g, BTPB, s,
                        bdview(L.S, L.n, (const double*)L.S.dval.p, (const double*)L.S.diag.p, false), f, x, r, Kp);
            else
                blaunch(kb_resid_dia<J, float, float, FT, VT, VT, ND>, g, BTPB, s,
                        bdview(L.S, L.n, (const float*)L.S.dval32.p, (const float*)L.S.diag32.p, false), f, x, r, Kp);
        });
        return;
    }
    if constexpr (std::is_same<VT, double>::value)
        blaunch(kb_resid<J, double, double, FT, VT, VT>, g, BTPB, s, bview(L.S, (const double*)L.S.val.p, (const double*)L.S.diag.p), L.S.nslots, f, x, r, Kp);
    else if (L.vt == VT_BF16)
        blaunch(kb_resid<J, __nv_bfloat16, float, FT, VT, VT>, g, BTPB, s, bview(L.S, (const __nv_bfloat16*)L.S.val16.p, (const float*)L.S.diag32.p), L.S.nslots, f, x, r, Kp);
    else
        blaunch(kb_resid<J, float, float, FT, VT, VT>, g, BTPB, s, bview(L.S, (const float*)L.S.val32.p, (const float*)L.S.diag32.p), L.S.nslots, f, x, r, Kp);
}

template <class VT>
BV<VT, VT> bfull(const Sell& S) {
    if constexpr (std::is_same<VT, double>::value) return bview(S, (const double*)S.val.p, (const double*)nullptr);
    else return bview(S, (const float*)S.val32.p, (const float*)nullptr);
}

template <class VT> const VT* bdnat(const Level& L);
template <> const double* bdnat<double>(const Level& L) { return L.dnat64.p; }
template <> const float* bdnat<float>(const Level& L) { return L.dnat32.p; }

// As rec_vcycle: with first_done the caller has applied the first colour step from the zero guess.
template <int J, class FT, class VT>
void brec_vcycle(Handle& h, int l, const FT* f, VT* x, bool zero_guess, cudaStream_t s, bool first_done = false) {
    Batched& B = h.bat;
    const int Kp = B.Kp;
    const int nl = (int)h.lev.size();
    Level& L = h.lev[l];
    if (l == nl - 1) {
        const VT* ai = std::is_same<VT, double>::value ? (const VT*)h.Ainv.p : (const VT*)h.Ainv32.p;
        blaunch(kb_coarse<J, VT, FT, VT>, rows_grid(L.n), BTPB, s, L.n, ai, f, x, Kp);
        return;
    }
    int c0 = 0;
    if (first_done) {
        c0 = 1;
    } else if (zero_guess) {
        blaunch(kb_zero_first<FT, VT>, 2048, 256, s, L.n, Kp, f, (const int*)L.colour.p, bdnat<VT>(L), x);
        c0 = 1;
    }
    for (int c = c0; c < L.ncolours; ++c) brec_gs<J>(L, c, f, x, Kp, s);
    brec_resid<J>(L, f, (const VT*)x, br<VT>(B, l), Kp, s);
    Level& C = h.lev[l + 1];
    if (l + 1 == nl - 1) {
        blaunch(kb_apply<J, VT, VT>, std::min(rows_grid(L.SR.nslots), 152 * 32), BTPB, s, bfull<VT>(L.SR), L.SR.nslots,
                (const VT*)br<VT>(B, l), bf<VT>(B, l + 1), bx<VT>(B, l + 1), Kp);
        brec_vcycle<J, VT, VT>(h, l + 1, bf<VT>(B, l + 1), bx<VT>(B, l + 1), false, s);
    } else {
        blaunch(kb_restrict_first<J, VT, VT>, std::min(rows_grid(L.SR.nslots), 152 * 32), BTPB, s, bfull<VT>(L.SR),
                L.SR.nslots, (const VT*)br<VT>(B, l), bf<VT>(B, l + 1), bx<VT>(B, l + 1), (const int*)C.colour.p,
                bdnat<VT>(C), Kp);
        brec_vcycle<J, VT, VT>(h, l + 1, bf<VT>(B, l + 1), bx<VT>(B, l + 1), true, s, true);
    }
    blaunch(kb_prolong<J, VT, VT>, std::min(rows_grid(L.SP.nslots), 152 * 32), BTPB, s, bfull<VT>(L.SP), L.SP.nslots,
            (const VT*)bx<VT>(B, l + 1), x, Kp);
    for (int c = L.ncolours - 1; c >= 0; --c) brec_gs<J>(L, c, f, x, Kp, s);
}

template <int J, class TT, class VT>
void brec_ic(Handle& h, const TT* t, VT* y, VT* w, VT* zadd, cudaStream_t s) {
    const int Kp = h.bat.Kp;
    BV<VT, VT> lv, uv;
    if constexpr (std::is_same<VT, double>::value) {
        lv = bview(h.L, (const double*)h.L.val.p, (const double*)nullptr);
        uv = bview(h.U, (const double*)h.U.val.p, (const double*)h.U.dinv.p);
    } else {
        lv = bview(h.L, (const float*)h.L.val32.p, (const float*)nullptr);
        uv = bview(h.U, (const float*)h.U.val32.p, (const float*)h.U.dinv32.p);
    }
    for (int g = 0; g + 1 < (int)h.L.seg.size(); ++g) {
        const int s0 = h.L.seg[g] * h.L.C, s1 = h.L.seg[g + 1] * h.L.C;
        blaunch(kb_lsolve<J, VT, TT, VT>, rows_grid(s1 - s0), BTPB, s, lv, s0, s1, t, y, Kp);
    }
    for (int g = 0; g + 1 < (int)h.U.seg.size(); ++g) {
        const int s0 = h.U.seg[g] * h.U.C, s1 = h.U.seg[g + 1] * h.U.C;
        blaunch(kb_usolve<J, VT, VT>, rows_grid(s1 - s0), BTPB, s, uv, s0, s1, (const VT*)y, w, zadd, Kp);
    }
}

template <int J, class VT>
void brec_precond(Handle& h, int which, const double* r, VT* z, cudaStream_t s) {
    Batched& B = h.bat;
    const int Kp = B.Kp;
    VT* t = (VT*)B.t.p;
    VT* y = (VT*)B.y.p;
    const Sell& A = h.Anat;
    auto fine_resid = [&]() {
        const int g = std::min(rows_grid(A.nslots), 152 * 32);
        if (A.ndiag) {
            bwith_nd(A.ndiag, [&](auto nd) {
                constexpr int ND = decltype(nd)::value;
                if constexpr (std::is_same<VT, double>::value)
                    blaunch(kb_resid_dia<J, double, double, double, VT, VT, ND>, g, BTPB, s,
                            bdview(A, h.n, (const double*)A.dval.p, (const double*)A.diag.p, true), r, (const VT*)z, t, Kp);
                else
                    blaunch(kb_resid_dia<J, float, float, double, VT, VT, ND>, g, BTPB, s,
                            bdview(A, h.n, (const float*)A.dval32.p, (const float*)A.diag32.p, true), r, (const VT*)z, t, Kp);
            });
            return;
        }
        if constexpr (std::is_same<VT, double>::value)
            blaunch(kb_resid<J, double, double, double, VT, VT>, g, BTPB, s, bview(A, (const double*)A.val.p, (const double*)A.diag.p), A.nslots, r, (const VT*)z, t, Kp);
        else
            blaunch(kb_resid<J, float, float, double, VT, VT>, g, BTPB, s, bview(A, (const float*)A.val32.p, (const float*)A.diag32.p), A.nslots, r, (const VT*)z, t, Kp);
    };
    switch (which) {
        case CPC_PRECOND_BCO:
            brec_vcycle<J, double, VT>(h, 0, r, z, true, s);
            if (h.ic_rb && h.lev[0].S.ndiag) {                   // step (2): black rows, one pass
                const Sell& S0 = h.lev[0].S;
                const int s0 = S0.seg[1] * S0.C, s1 = S0.seg[2] * S0.C;
                if (s1 > s0)
                    bwith_nd(S0.ndiag, [&](auto nd) {
                        constexpr int ND = decltype(nd)::value;
                        if constexpr (std::is_same<VT, double>::value)
                            blaunch(kb_bco_black_dia<J, double, double, VT, ND>, rows_grid(s1 - s0), BTPB, s,
                                    bdview(S0, h.n, (const double*)S0.dval.p, (const double*)S0.diag.p, false), s0, s1,
                                    r, (const VT*)h.ic_uinv64.p, z, Kp);
                        else
                            blaunch(kb_bco_black_dia<J, float, float, VT, ND>, rows_grid(s1 - s0), BTPB, s,
                                    bdview(S0, h.n, (const float*)S0.dval32.p, (const float*)S0.diag32.p, false), s0,
                                    s1, r, (const VT*)h.ic_uinv32.p, z, Kp);
                    });
            } else {
                fine_resid();
                brec_ic<J, VT, VT>(h, t, y, t, z, s);
            }
            brec_vcycle<J, double, VT>(h, 0, r, z, false, s);
            break;
        case CPC_PRECOND_AMG:
            brec_vcycle<J, double, VT>(h, 0, r, z, true, s);
            brec_vcycle<J, double, VT>(h, 0, r, z, false, s);
            break;
        case CPC_PRECOND_IC0:
            brec_ic<J, double, VT>(h, r, y, z, (VT*)nullptr, s);
            break;
        case CPC_PRECOND_BHAT:
            brec_vcycle<J, double, VT>(h, 0, r, z, true, s);
            brec_vcycle<J, double, VT>(h, 0, r, z, false, s);
            brec_ic<J, double, VT>(h, r, y, t, z, s);
            break;
        default:
            fail(CPC_EINVAL, "batched solve supports B_co, AMG, IC(0) and B^");
    }
}

template <int J, class VT>
void brec_loop(Handle& h, cudaGraph_t g, cudaStream_t cs, cudaGraphNode_t* dep, size_t ndep, cudaGraphNode_t* out_node) {
    Batched& B = h.bat;
    const int Kp = B.Kp;
    const int n = h.n;
    cudaGraphConditionalHandle cond;
    CPC_CK(cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CPC_CK(cudaGraphAddNode(out_node, g, dep, nullptr, ndep, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CPC_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    blaunch(kb_guard, 1, 32, cs, cond);
    VT* z = (VT*)B.z.p;
    brec_precond<J, VT>(h, h.opt.precond, B.r.p, z, cs);
    const int vg = std::min(rows_grid(n), 152 * 8);
    blaunch(kb_rz<J, VT>, vg, BTPB, cs, n, Kp, (const double*)B.r.p, (const VT*)z, B.partial.p, h.counter.p + 1, B.S.p);
    blaunch(kb_p<J, VT>, vg, BTPB, cs, n, Kp, (const VT*)z, B.p.p, (const double*)B.S.p);
    const Sell& A = h.Anat;
    if (A.ndiag)
        bwith_nd(A.ndiag, [&](auto nd) {
            blaunch(kb_spmv_pq_dia<J, decltype(nd)::value>, std::min(rows_grid(A.nslots), 152 * 8), BTPB, cs,
                    bdview(A, n, (const double*)A.dval.p, (const double*)A.diag.p, true), Kp, (const double*)B.p.p,
                    B.q.p, B.partial.p, h.counter.p + 1, B.S.p);
        });
    else
        blaunch(kb_spmv_pq<J>, std::min(rows_grid(A.nslots), 152 * 8), BTPB, cs, bview(A, (const double*)A.val.p, (const double*)A.diag.p),
                A.nslots, Kp, (const double*)B.p.p, B.q.p, B.partial.p, h.counter.p + 1, B.S.p);
    blaunch(kb_update<J>, vg, BTPB, cs, n, Kp, B.x.p, B.r.p, (const double*)B.p.p, (const double*)B.q.p, B.partial.p,
            h.counter.p + 1, B.S.p);
    blaunch(kb_any_active, 1, 32, cs, Kp, (const double*)B.S.p, cond);
    CPC_CK(cudaStreamEndCapture(cs, &body));
}

// One graph: pack B, init, while(any active) { iteration }, [adjoint: sources, init, while {...}].
template <int J, class VT>
void build_batched_graph(Handle& h, bool with_adjoint) {
    Batched& B = h.bat;
    const int Kp = B.Kp;
    const int n = h.n;
    cudaStream_t cs;
    CPC_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cs};
    cudaGraph_t g;
    CPC_CK(cudaGraphCreate(&g, 0));
    const int vg = std::min(rows_grid(n), 152 * 8);
    auto capture_into = [&](cudaGraphNode_t* deps, size_t ndeps, auto&& body) -> std::vector<cudaGraphNode_t> {
        std::vector<cudaGraphNode_t> before;
        size_t nn = 0;
        CPC_CK(cudaGraphGetNodes(g, nullptr, &nn));
        before.resize(nn);
        CPC_CK(cudaGraphGetNodes(g, before.data(), &nn));
        CPC_CK(cudaStreamBeginCaptureToGraph(cs, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
        body();
        CPC_CK(cudaStreamEndCapture(cs, &g));
        size_t nn2 = 0;
        CPC_CK(cudaGraphGetNodes(g, nullptr, &nn2));
        std::vector<cudaGraphNode_t> all(nn2);
        CPC_CK(cudaGraphGetNodes(g, all.data(), &nn2));
        std::vector<cudaGraphNode_t> added;
        for (auto nd : all) if (std::find(before.begin(), before.end(), nd) == before.end()) added.push_back(nd);
        // leaves among the added nodes
        std::vector<cudaGraphNode_t> leaves;
        for (auto nd : added) {
            size_t nout = 0;
            CPC_CK(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout));
            if (nout == 0) leaves.push_back(nd);
        }
        return leaves;
    };
    auto l1 = capture_into(nullptr, 0, [&] {
        blaunch(kb_pack, 2048, 256, cs, n, B.K, Kp, (const double*)B.user_b, B.b.p);
        blaunch(kb_init<J>, vg, BTPB, cs, n, Kp, (const double*)B.b.p, B.x.p, B.r.p, B.partial.p, h.counter.p + 1, B.S.p);
    });
    cudaGraphNode_t w1;
    brec_loop<J, VT>(h, g, cs, l1.data(), l1.size(), &w1);
    cudaGraphNode_t tail = w1;
    if (with_adjoint) {
        auto l2 = capture_into(&w1, 1, [&] {
            blaunch(kb_adjoint_rhs, 2048, 256, cs, (int64_t)n * Kp, B.b.p, (const double*)B.x.p, B.xfwd.p);
            blaunch(kb_unpack, 2048, 256, cs, n, B.K, Kp, (const double*)B.xfwd.p, B.user_x);
            CPC_CK(cudaMemcpyAsync(B.kfwd.p, B.S.p + (size_t)S_K * Kp, sizeof(double) * Kp, cudaMemcpyDeviceToDevice, cs));
            CPC_CK(cudaMemcpyAsync(B.kfwd.p + Kp, B.S.p + (size_t)S_STATUS * Kp, sizeof(double) * Kp, cudaMemcpyDeviceToDevice, cs));
            blaunch(kb_init<J>, vg, BTPB, cs, n, Kp, (const double*)B.b.p, B.x.p, B.r.p, B.partial.p, h.counter.p + 1, B.S.p);
        });
        cudaGraphNode_t w2;
        brec_loop<J, VT>(h, g, cs, l2.data(), l2.size(), &w2);
        tail = w2;
    }
    capture_into(&tail, 1, [&] {
        blaunch(kb_unpack, 2048, 256, cs, n, B.K, Kp, (const double*)B.x.p, with_adjoint ? B.user_lambda : B.user_x);
    });
    cudaGraphExec_t ge;
    CPC_CK(cudaGraphInstantiate(&ge, g, 0));
    B.graph = g;
    B.gexec = ge;
}


// Block PCG loop on the packed block vectors of h.bat (K <= Kp <= 64).  Each iteration:
//   Q = A P;  alpha = (P^T Q)^{-1} gamma;  X += P alpha, R -= Q alpha;  stop when every column
//   has ||r_k|| / ||b_k|| < tol;  Z = M R;  beta = gamma^{-1} (Z^T R);  gamma = Z^T R;  P = Z + P beta.
// The host reads two flags per iteration (one stream synchronisation).
template <int J, class VT>
int solve_block_t(Handle& h, int K, double tol, int maxit, int* iters, double* res) {
    Batched& B = h.bat;
    const int Kp = B.Kp, n = h.n;
    cudaStream_t s = h.s;
    const int64_t nk = (int64_t)n * Kp;
    auto km = [&](int i) { return B.kmat.p + (size_t)i * Kp * Kp; };
    const size_t gram_smem = 2 * (size_t)KK_ROWS * Kp * sizeof(double);
    const size_t solve_smem = 2 * (size_t)K * K * sizeof(double);
    const size_t upd_smem = ((size_t)Kp * Kp + BWARPS * Kp) * sizeof(double);
    const size_t pup_smem = (size_t)Kp * Kp * sizeof(double);
    CPC_CK(cudaFuncSetAttribute(kk_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * (int)sizeof(double)));
    const Csr& A = h.lev[0].A;
    const int rg = std::min(rows_grid(n), 152 * 8);
    VT* z = (VT*)B.z.p;
    auto gram = [&](const auto* U, const double* V, double* out) {
        kk_gram<<<KK_GRID, KK_TPB, gram_smem, s>>>(n, Kp, U, V, B.kpart.p);
        kk_gram_sum<<<16, 256, 0, s>>>(KK_GRID, Kp, B.kpart.p, out);
    };
    int flags[KF_COUNT] = {0, 0};
    auto read_flags = [&]() {
        CPC_LAUNCH_CK();
        CPC_CK(cudaMemcpyAsync(flags, B.kflag.p, sizeof(flags), cudaMemcpyDeviceToHost, s));
        CPC_CK(cudaStreamSynchronize(s));
    };
    CPC_CK(cudaMemsetAsync(B.kflag.p, 0, sizeof(int) * KF_COUNT, s));
    CPC_CK(cudaMemsetAsync(B.kmat.p, 0, sizeof(double) * KM_COUNT * Kp * Kp, s));
    kb_pack<<<2048, 256, 0, s>>>(n, K, Kp, (const double*)B.user_b, B.b.p);
    CPC_CK(cudaMemcpyAsync(B.r.p, B.b.p, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
    CPC_CK(cudaMemsetAsync(B.x.p, 0, sizeof(double) * nk, s));
    kk_colnorm<J><<<KK_GRID, BTPB, 0, s>>>(n, Kp, B.r.p, B.kpart.p);
    kk_check<<<1, 64, 0, s>>>(KK_GRID, Kp, K, B.kpart.p, B.kvec.p, tol, 1, B.kflag.p);
    read_flags();
    if (flags[KF_BAD]) fail(CPC_EINVAL, "a right-hand-side column is zero or not finite");
    brec_precond<J, VT>(h, h.opt.precond, B.r.p, z, s);              // Z = M R
    kk_copy<VT><<<2048, 256, 0, s>>>(nk, (const VT*)z, B.p.p);         // P = Z
    gram((const VT*)z, B.r.p, km(KM_GAMMA));                           // gamma = Z^T R
    int status = CPC_ENOCONV, it = 0;
    for (int k = 1; k <= maxit; ++k) {
        kk_spmm<J><<<rg, BTPB, 0, s>>>(n, Kp, A.ptr.p, A.col.p, A.val.p, (const double*)B.p.p, B.q.p);
        gram((const double*)B.p.p, B.q.p, km(KM_PQ));
        kk_solve<<<1, KK_TPB, solve_smem, s>>>(K, Kp, km(KM_PQ), km(KM_GAMMA), km(KM_ALPHA), nullptr, B.kflag.p);
        kk_update<J><<<KK_GRID, BTPB, upd_smem, s>>>(n, Kp, K, B.x.p, B.r.p, B.p.p, B.q.p, km(KM_ALPHA), B.kpart.p,
                                                    B.kflag.p);
        kk_check<<<1, 64, 0, s>>>(KK_GRID, Kp, K, B.kpart.p, B.kvec.p, tol, 0, B.kflag.p);
        read_flags();
        if (flags[KF_BAD]) {                                           // X holds iteration k - 1
            status = CPC_EBREAKDOWN;
            it = k - 1;
            break;
        }
        it = k;
        if (flags[KF_DONE]) {
            status = CPC_OK;
            break;
        }
        if (k == maxit) break;
        brec_precond<J, VT>(h, h.opt.precond, B.r.p, z, s);          // Z = M R
        gram((const VT*)z, B.r.p, km(KM_GAMMA_NEW));                   // Z^T R
        kk_solve<<<1, KK_TPB, solve_smem, s>>>(K, Kp, km(KM_GAMMA), km(KM_GAMMA_NEW), km(KM_BETA), km(KM_GAMMA),
                                               B.kflag.p);
        kk_pupdate<J, VT><<<KK_GRID, BTPB, pup_smem, s>>>(n, Kp, K, (const VT*)z, B.p.p, km(KM_BETA), B.kflag.p);
    }
    kb_unpack<<<2048, 256, 0, s>>>(n, K, Kp, (const double*)B.x.p, B.user_x);
    CPC_LAUNCH_CK();
    std::vector<double> hv((size_t)KV_COUNT * Kp);
    CPC_CK(cudaMemcpyAsync(hv.data(), B.kvec.p, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    *iters = it;
    if (res)
        for (int c = 0; c < K; ++c) res[c] = hv[(size_t)KV_RES * Kp + c];
    return status;
}

}  // namespace

void destroy_batched(Handle& h) {
    Batched& B = h.bat;
    if (B.gexec) cudaGraphExecDestroy(B.gexec);
    if (B.graph) cudaGraphDestroy(B.graph);
    B.gexec = nullptr;
    B.graph = nullptr;
}

// Allocate the block vectors for K columns (kept across calls with the same padded width).
static void ensure_batched(Handle& h, int K, bool adjoint, double* user_b, double* user_x, double* user_lambda) {
    Batched& B = h.bat;
    const int Kp = (K + 31) / 32 * 32;
    if (Kp > 128) fail(CPC_EINVAL, "at most 128 right-hand sides per batched call");
    const bool fp64 = h.opt.precision == CPC_PREC_FP64;
    const size_t vsz = fp64 ? sizeof(double) : sizeof(float);
    if (B.Kp != Kp) {
        destroy_batched(h);
        B = Batched{};
        B.Kp = Kp;
        const size_t nk = (size_t)h.n * Kp;
        B.b.alloc(nk); B.x.alloc(nk); B.r.alloc(nk); B.p.alloc(nk); B.q.alloc(nk); B.xfwd.alloc(nk);
        B.z.alloc(nk * vsz); B.t.alloc(nk * vsz); B.y.alloc(nk * vsz);
        const int nl = (int)h.lev.size();
        B.lx.resize(nl); B.lf.resize(nl); B.lr.resize(nl);
        for (int l = 0; l < nl; ++l) {
            const size_t m = (size_t)h.lev[l].n * Kp * vsz;
            B.lx[l].alloc(m); B.lf[l].alloc(m); B.lr[l].alloc(m);
        }
        B.S.alloc((size_t)NB_STATE * Kp);
        B.partial.alloc((size_t)152 * 32 * Kp);
        B.kfwd.alloc(2 * (size_t)Kp);
        if (Kp <= 64) {
            B.kmat.alloc((size_t)KM_COUNT * Kp * Kp);
            B.kpart.alloc((size_t)KK_GRID * Kp * Kp);
            B.kvec.alloc((size_t)KV_COUNT * Kp);
            B.kflag.alloc(KF_COUNT);
        }
    }
    if (B.gexec && (B.K != K || B.adjoint != adjoint || B.user_b != user_b || B.user_x != user_x ||
                    B.user_lambda != user_lambda)) destroy_batched(h);
    B.K = K;
    B.adjoint = adjoint;
    B.user_b = user_b;
    B.user_x = user_x;
    B.user_lambda = user_lambda;
}

void solve_batched(Handle& h, int K, const double* b, double* x, double* lambda, double tol, int maxit,
                   int* iters, int* status, int* iters_adj, int* status_adj) {
    ensure_batched(h, K, lambda != nullptr, (double*)b, x, lambda);
    Batched& B = h.bat;
    const int Kp = B.Kp;
    if (!B.gexec) {
        const bool fp64 = h.opt.precision == CPC_PREC_FP64;
        const int J = Kp / 32;
        const bool adj = lambda != nullptr;
        if (fp64) {
            if (J == 1) build_batched_graph<1, double>(h, adj);
            else if (J == 2) build_batched_graph<2, double>(h, adj);
            else if (J == 3) build_batched_graph<3, double>(h, adj);
            else build_batched_graph<4, double>(h, adj);
        } else {
            if (J == 1) build_batched_graph<1, float>(h, adj);
            else if (J == 2) build_batched_graph<2, float>(h, adj);
            else if (J == 3) build_batched_graph<3, float>(h, adj);
            else build_batched_graph<4, float>(h, adj);
        }
    }
    cudaStream_t s = h.s;
    std::vector<double> st((size_t)NB_STATE * Kp, 0.0);
    for (int c = 0; c < Kp; ++c) {
        st[(size_t)S_TOL * Kp + c] = tol;
        st[(size_t)S_MAXIT * Kp + c] = c < K ? (double)maxit : 0.0;
    }
    CPC_CK(cudaMemcpyAsync(B.S.p, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, s));
    CPC_CK(cudaGraphLaunch(B.gexec, s));
    CPC_CK(cudaMemcpyAsync(st.data(), B.S.p, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, s));
    std::vector<double> kf(2 * (size_t)Kp, 0.0);
    if (lambda) CPC_CK(cudaMemcpyAsync(kf.data(), B.kfwd.p, sizeof(double) * 2 * Kp, cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    for (int c = 0; c < K; ++c) {
        const int ki = (int)st[(size_t)S_K * Kp + c];
        const int si = (int)st[(size_t)S_STATUS * Kp + c];
        if (lambda) {
            iters[c] = (int)kf[c];
            if (status) status[c] = (int)kf[Kp + c];
            if (iters_adj) iters_adj[c] = ki;
            if (status_adj) status_adj[c] = si;
        } else {
            iters[c] = ki;
            if (status) status[c] = si;
        }
    }
}

int solve_block(Handle& h, int K, const double* b, double* x, double tol, int maxit, int* iters, double* res) {
    if (K < 1 || K > 64) fail(CPC_EINVAL, "block CG takes 1 to 64 right-hand sides");
    if (h.opt.precond == CPC_PRECOND_AMG_ILU) fail(CPC_EINVAL, "block CG supports B_co, AMG, IC(0) and B^");
    ensure_batched(h, K, false, (double*)b, x, nullptr);
    const bool fp64 = h.opt.precision == CPC_PREC_FP64;
    if (h.bat.Kp == 32) return fp64 ? solve_block_t<1, double>(h, K, tol, maxit, iters, res)
                                    : solve_block_t<1, float>(h, K, tol, maxit, iters, res);
    return fp64 ? solve_block_t<2, double>(h, K, tol, maxit, iters, res)
                : solve_block_t<2, float>(h, K, tol, maxit, iters, res);
}

}  // namespace cpc
