// solve.cu -- solve phase: V-cycle (Algorithm 3.2), IC(0) triangular solves, the combined
// preconditioner (Algorithm 2.1) and PCG, all as sm_103a kernels; the PCG loop is one CUDA graph
// with a device-side while node, so the host only launches it and reads back the result.
//
// Kernel layout: every matrix is SELL-C (C in {32, 16, 8, 4}): one warp per chunk of C rows with
// 32 / C lanes per row, entries column-major inside a chunk so that each load instruction of a
// warp reads 32 consecutive elements.  On a structured fine grid the diagonal form (one thread per
// row, no column indices) replaces SELL for the fine-level kernels.  Every kernel is launched with
// programmatic dependent launch and loads its matrix data before waiting for its predecessor.
// Reductions (dot products) finish in a fixed order (per-block tree, then the last block sums the
// block partials in index order), so iteration counts are reproducible run to run.
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include <utility>

#include "device.cuh"
#include "handle.cuh"

namespace cpc {

namespace {

constexpr int WPB = GS_WARPS_PER_BLOCK;  // warps (= SELL chunks) per block
constexpr int SELL_TPB = WPB * 32;
constexpr int VEC_TPB = 256;

// Launch with programmatic stream serialisation (see pdl_wait in device.cuh).
template <class... KArgs, class... Args>
void launch(void (*k)(KArgs...), int grid, int block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CPC_CK(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
}

// Calls f(std::integral_constant<int, U>{}) with the sell_dot batch width for an operator whose
// lanes hold at most `lanes` entries.
template <class F>
void with_u(int lanes, F&& f) {
    if (lanes <= 4) f(std::integral_constant<int, 4>{});
    else if (lanes <= 6) f(std::integral_constant<int, 6>{});
    else f(std::integral_constant<int, 8>{});
}

// As with_u for the Gauss-Seidel colour steps, with batches of up to 16: a colour step lasts as long
// as its widest chunk, and one batch per lane keeps it to one round of dependent gathers.  The
// products are added in the same entry order whatever the batch, so the results do not change.
template <class F>
void with_u_gs(int lanes, F&& f) {
    if (lanes <= 8) with_u(lanes, f);
    else if (lanes <= 12) f(std::integral_constant<int, 12>{});
    else f(std::integral_constant<int, 16>{});
}

// Calls f(std::integral_constant<int, ND>{}) with the padded diagonal count (4, 6 or 8).
template <class F>
void with_nd(int nd, F&& f) {
    if (nd <= 4) f(std::integral_constant<int, 4>{});
    else if (nd <= 6) f(std::integral_constant<int, 6>{});
    else f(std::integral_constant<int, 8>{});
}

inline int slot_blocks(int64_t nslots) { return (int)std::max<int64_t>(1, (nslots + SELL_TPB - 1) / SELL_TPB); }

inline int blocks_for_chunks(int nchunks) { return std::max(1, (nchunks + WPB - 1) / WPB); }
inline int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + VEC_TPB - 1) / VEC_TPB, NPART)); }

// ---------------------------------------------------------------------------------------------
// Level kernels.  A warp owns one chunk of A.C rows; lane l works on row l % C of the chunk with
// G = 32 / C lanes per row (sub-lane l / C takes entries l / C, l / C + G, ...); sub_sum() adds
// the G partial sums, after which sub-lane 0 writes the row.
// ---------------------------------------------------------------------------------------------
template <class VT>
__device__ __forceinline__ VT sub_sum(VT v, int C) {
    for (int o = C; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// Diagonal form (structured grids, Sell::ndiag > 0): one thread per slot; the matrix values of a
// slot are ND coalesced loads (no column indices, no chunk pointers), the gathers are x[i + off_d]
// with the index clamped into range (the value is 0 wherever the row has no such entry).  The
// products are added in ascending column order, as in the SELL kernels.
// ---------------------------------------------------------------------------------------------
template <class MT, class DT>
struct DV {
    int n, nslots;
    const int* __restrict__ perm;      // nullptr: natural order, row = slot
    const MT* __restrict__ val;        // [ND][nslots]
    const DT* __restrict__ diag;
    DiaOff off;
};

template <class MT, class DT>
inline DV<MT, DT> dview(const Sell& S, int n, const MT* val, const DT* diag, bool natural) {
    return DV<MT, DT>{n, S.nslots, natural ? nullptr : S.perm.p, val, diag, S.doff};
}

template <class MT, class DT>
__device__ __forceinline__ int dia_row(const DV<MT, DT>& A, int s) {
    return A.perm ? A.perm[s] : (s < A.n ? s : -1);
}

template <int ND, class VT, class MT, class DT>
__device__ __forceinline__ void dia_load(const DV<MT, DT>& A, int s, VT (&v)[ND]) {
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = Cv<VT>::f(A.val[(size_t)d * A.nslots + s]);
}

template <int ND, class VT, class XT>
__device__ __forceinline__ VT dia_dot(const VT (&v)[ND], const DiaOff& off, int row, int n, const XT* x) {
    VT xv[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        int j = row + off.o[d];
        j = j < 0 ? 0 : (j >= n ? n - 1 : j);
        xv[d] = Cv<VT>::f(x[j]);
    }
    VT acc = VT(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) acc += v[d] * xv[d];
    return acc;
}

// Gauss-Seidel on slots [s0, s1) (one colour), diagonal form; A.diag holds 1 / a_ii.
template <class MT, class DT, class FT, class VT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_gs_dia(DV<MT, DT> A, int s0, int s1, const FT* f, VT* x) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    VT v[ND];
    dia_load<ND, VT>(A, s, v);
    const VT dinv = Cv<VT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const VT fr = Cv<VT>::f(f[row]);
    const VT dot = dia_dot<ND, VT>(v, A.off, row, A.n, x);
    x[row] = (fr - dot) * dinv;
}

// Gauss-Seidel on slots [s0, s1) from the per-slot records g = -a_ij / a_ii (Sell::gval):
// x_i = f_i / a_ii + sum_d g_d x_{i + off_d}; the ND values of a slot arrive in ND / 2 two-element
// vector loads, and the update is 7 FP64 operations (one product, six fused multiply-adds).
template <class MT> struct Pair;
template <> struct Pair<double> { using T = double2; };
template <> struct Pair<float> { using T = float2; };

template <class MT, class DT, class FT, class VT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_gs_pk(DV<MT, DT> A, int s0, int s1, const FT* f, VT* x) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    using P2 = typename Pair<MT>::T;
    const P2* rec = reinterpret_cast<const P2*>(A.val + (size_t)s * ND);
    VT g[ND];
#pragma unroll
    for (int q = 0; q < ND / 2; ++q) {
        const P2 t = rec[q];
        g[2 * q] = Cv<VT>::f(t.x);
        g[2 * q + 1] = Cv<VT>::f(t.y);
    }
    const VT dinv = Cv<VT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    VT acc = Cv<VT>::f(f[row]) * dinv;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        int j = row + A.off.o[d];
        j = j < 0 ? 0 : (j >= A.n ? A.n - 1 : j);
        acc += g[d] * Cv<VT>::f(x[j]);
    }
    x[row] = acc;
}

// r = f - A x on slots [s0, s1), diagonal form.
template <class MT, class DT, class FT, class XT, class RT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_resid_dia(DV<MT, DT> A, int s0, int s1, const FT* f,
                                                         const XT* x, RT* __restrict__ r) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    RT v[ND];
    dia_load<ND, RT>(A, s, v);
    const RT dg = Cv<RT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const RT fr = Cv<RT>::f(f[row]);
    const RT dx = dg * Cv<RT>::f(x[row]);
    const RT dot = dia_dot<ND, RT>(v, A.off, row, A.n, x);
    r[row] = fr - (dx + dot);
}

// r = f - A x after a forward sweep on a two-colour level in diagonal form: slots below s1 (the
// first colour) get the full residual; the rows of the last colour were just solved from their
// current neighbours, so their residual is zero up to rounding and is written as 0 without
// loading their matrix entries.
template <class MT, class DT, class FT, class XT, class RT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_resid_dia_first(DV<MT, DT> A, int s1, const FT* f, const XT* x, RT* r) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.nslots) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    if (s >= s1) {
        pdl_wait();
        if (row >= 0) r[row] = RT(0);
        return;
    }
    RT v[ND];
    dia_load<ND, RT>(A, s, v);
    const RT dg = Cv<RT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const RT fr = Cv<RT>::f(f[row]);
    const RT dx = dg * Cv<RT>::f(x[row]);
    const RT dot = dia_dot<ND, RT>(v, A.off, row, A.n, x);
    r[row] = fr - (dx + dot);
}

// y = A x, diagonal form.
template <class MT, class DT, class XT, class YT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_spmv_dia(DV<MT, DT> A, const XT* x, YT* __restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.nslots) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    YT v[ND];
    dia_load<ND, YT>(A, s, v);
    const YT dg = Cv<YT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const YT dx = dg * Cv<YT>::f(x[row]);
    const YT dot = dia_dot<ND, YT>(v, A.off, row, A.n, x);
    y[row] = dx + dot;
}

// Gauss-Seidel over the rows of one colour (chunks [c0, c1)): x_i = (f_i - sum_{j!=i} a_ij x_j) / a_ii,
// with the view's diagonal field holding 1 / a_ii (a multiply instead of an FP64 division).
// Rows of one colour are not coupled, so they update in parallel exactly as in sequential order.
template <class MT, class DT, class FT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_gs(SV<MT, DT> A, int c0, int c1, const FT* f, VT* x) {
    const int k = c0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= c1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, C = A.C, r = lane & (C - 1), g = lane / C;
    const int s = k * C + r;
    const int row = A.perm[s];
    const bool own = g == 0 && row >= 0;
    const VT dinv = own ? Cv<VT>::f(A.diag[s]) : VT(0);
    VT fr = VT(0);
    VT dot = sell_dot<VT, true, U>(A.col, A.val, A.cptr[k] + g * C + r, A.cptr[k + 1], x,
                                   [&] { if (own) fr = Cv<VT>::f(f[row]); });
    dot = sub_sum(dot, C);
    if (own) x[row] = (fr - dot) * dinv;
}

// r = f - A x over all chunks (grid-stride over chunks).
template <class MT, class DT, class FT, class XT, class RT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_resid(SV<MT, DT> A, int nchunks, const FT* f,
                                                     const XT* x, RT* __restrict__ r) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = A.C, rr = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int s = k * C + rr;
        const int row = A.perm[s];
        const bool own = g == 0 && row >= 0;
        RT fr = RT(0), dx = RT(0);
        if (own) {
            fr = Cv<RT>::f(f[row]);
            dx = Cv<RT>::f(A.diag[s]) * Cv<RT>::f(x[row]);
        }
        RT dot = sell_dot<RT, false, U>(A.col, A.val, A.cptr[k] + g * C + rr, A.cptr[k + 1], x);
        dot = sub_sum(dot, C);
        if (own) r[row] = fr - (dx + dot);
    }
}

// y = A x (diagonal split) over all chunks.
template <class MT, class DT, class XT, class YT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_spmv(SV<MT, DT> A, int nchunks, const XT* x,
                                                    YT* __restrict__ y) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = A.C, r = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int s = k * C + r;
        const int row = A.perm[s];
        const bool own = g == 0 && row >= 0;
        const YT dx = own ? Cv<YT>::f(A.diag[s]) * Cv<YT>::f(x[row]) : YT(0);
        YT dot = sell_dot<YT, false, U>(A.col, A.val, A.cptr[k] + g * C + r, A.cptr[k + 1], x);
        dot = sub_sum(dot, C);
        if (own) y[row] = dx + dot;
    }
}

// y = M x (full rows, no split diagonal): restriction f_c = R r.
template <class MT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_apply_full(SV<MT, MT> M, int nchunks, const VT* x,
                                                          VT* __restrict__ y) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = M.C, r = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int row = M.perm[k * C + r];
        VT dot = sell_dot<VT, false, U>(M.col, M.val, M.cptr[k] + g * C + r, M.cptr[k + 1], x);
        dot = sub_sum(dot, C);
        if (g == 0 && row >= 0) y[row] = dot;
    }
}

// f_c = R r and x_c = 0 (the next level starts from a zero guess).
template <class MT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_restrict_zero(SV<MT, MT> M, int nchunks, const VT* x,
                                                             VT* __restrict__ y, VT* __restrict__ yz) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = M.C, r = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int row = M.perm[k * C + r];
        VT dot = sell_dot<VT, false, U>(M.col, M.val, M.cptr[k] + g * C + r, M.cptr[k + 1], x);
        dot = sub_sum(dot, C);
        if (g == 0 && row >= 0) { y[row] = dot; yz[row] = VT(0); }
    }
}

// f_c = R r, and the first colour step of the coarse sweep from a zero guess fused with the zero
// fill: x_c = f_c / a_ii on colour 0 (its rows see only zeros), 0 elsewhere.
template <class MT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_restrict_first(SV<MT, MT> M, int nchunks, const VT* x,
                                                              VT* __restrict__ y, VT* __restrict__ yx,
                                                              const int* __restrict__ colour,
                                                              const VT* __restrict__ dnat) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = M.C, r = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int row = M.perm[k * C + r];
        const bool own = g == 0 && row >= 0;
        int cr = 1;
        VT dr = VT(0);
        if (own) {
            cr = colour[row];
            dr = dnat[row];
        }
        VT dot = sell_dot<VT, false, U>(M.col, M.val, M.cptr[k] + g * C + r, M.cptr[k + 1], x);
        dot = sub_sum(dot, C);
        if (own) {
            y[row] = dot;
            yx[row] = cr == 0 ? dot * dr : VT(0);
        }
    }
}

// The same on the finest level (f given): x = f / a_ii on colour 0, 0 elsewhere.
template <class FT, class VT>
__global__ void k_zero_first(int64_t n, const FT* f, const int* __restrict__ colour,
                             const VT* __restrict__ dnat, VT* __restrict__ x) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = colour[i] == 0 ? Cv<VT>::f(f[i]) * dnat[i] : VT(0);
}

// x += P e (prolongation and correction).
template <class MT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_prolong(SV<MT, MT> P, int nchunks, const VT* e,
                                                       VT* __restrict__ x) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = P.C, r = lane & (C - 1), g = lane / C;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int row = P.perm[k * C + r];
        const bool own = g == 0 && row >= 0;
        const VT xr = own ? x[row] : VT(0);
        VT dot = sell_dot<VT, false, U>(P.col, P.val, P.cptr[k] + g * C + r, P.cptr[k + 1], e);
        dot = sub_sum(dot, C);
        if (own) x[row] = xr + dot;
    }
}

// x = A_c^{-1} f with the dense inverse (row-major), one warp per row.
template <class AT, class FT, class VT>
__global__ void k_coarse(int n, const AT* __restrict__ Ainv, const FT* f, VT* __restrict__ x) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += gridDim.x * (blockDim.x >> 5)) {
        VT acc = 0;
        for (int j = lane; j < n; j += 32) acc += Cv<VT>::f(Ainv[(size_t)i * n + j]) * Cv<VT>::f(f[j]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = acc;
    }
}

template <class VT>
__global__ void k_zero(int64_t n, VT* x) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0;
}

template <class A, class B>
__global__ void k_copy(int64_t n, const A* a, B* __restrict__ b) {
    pdl_launch_dependents();
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (B)a[i];
}

// Forward solve with the unit lower factor, rows of one level: y_i = t_i - sum_{j<i} l_ij y_j.
template <class MT, class TT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_lsolve(SV<MT, MT> L, int c0, int c1, const TT* t, VT* y) {
    const int k = c0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= c1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, C = L.C, r = lane & (C - 1), g = lane / C;
    const int row = L.perm[k * C + r];
    const bool own = g == 0 && row >= 0;
    VT tr = VT(0);
    VT dot = sell_dot<VT, true, U>(L.col, L.val, L.cptr[k] + g * C + r, L.cptr[k + 1], y,
                                   [&] { if (own) tr = Cv<VT>::f(t[row]); });
    dot = sub_sum(dot, C);
    if (own) y[row] = tr - dot;
}

// Backward solve with U, rows of one level: w_i = (y_i - sum_{j>i} u_ij w_j) / u_ii (the view's
// diagonal field holds 1 / u_ii); optionally z_i += w_i in the same pass.
template <class MT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_usolve(SV<MT, MT> Uf, int c0, int c1, const VT* y, VT* w,
                                                      VT* zadd) {
    const int k = c0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= c1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, C = Uf.C, r = lane & (C - 1), g = lane / C;
    const int s = k * C + r;
    const int row = Uf.perm[s];
    const bool own = g == 0 && row >= 0;
    const VT dinv = own ? Cv<VT>::f(Uf.diag[s]) : VT(0);
    VT yr = VT(0), zr = VT(0);
    VT dot = sell_dot<VT, true, U>(Uf.col, Uf.val, Uf.cptr[k] + g * C + r, Uf.cptr[k + 1], w, [&] {
        if (own) {
            yr = y[row];
            if (zadd) zr = zadd[row];
        }
    });
    dot = sub_sum(dot, C);
    if (own) {
        const VT v = (yr - dot) * dinv;
        w[row] = v;
        if (zadd) zadd[row] = zr + v;
    }
}

// B_co step (2) right after step (1) with red-black IC(0): step (1) ends with a Gauss-Seidel step on
// the red rows, which leaves their residual t_r = 0 (up to rounding), so the forward solve gives
// y_b = t_b and z_b += (r_b - (A z)_b) / u_bb on the black rows (fine colour 1, chunks [c0, c1) of
// the colour-grouped A) is the whole step; the red rows' part is overwritten by step (3).
template <class MT, class DT, class VT, int U>
__global__ void __launch_bounds__(SELL_TPB) k_bco_black(SV<MT, DT> A, int c0, int c1, const double* r,
                                                         const VT* __restrict__ uinv, VT* __restrict__ z) {
    const int k = c0 + blockIdx.x * WPB + (threadIdx.x >> 5);
    if (k >= c1) return;
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, C = A.C, rr = lane & (C - 1), g = lane / C;
    const int s = k * C + rr;
    const int row = A.perm[s];
    const bool own = g == 0 && row >= 0;
    const VT ui = own ? uinv[row] : VT(0);
    const VT dg = own ? Cv<VT>::f(A.diag[s]) : VT(0);
    VT fr = VT(0), zr = VT(0);
    VT dot = sell_dot<VT, true, U>(A.col, A.val, A.cptr[k] + g * C + rr, A.cptr[k + 1], z, [&] {
        if (own) {
            fr = Cv<VT>::f(r[row]);
            zr = z[row];
        }
    });
    dot = sub_sum(dot, C);
    if (own) z[row] = zr + (fr - (dg * zr + dot)) * ui;
}

// k_bco_black in diagonal form: slots [s0, s1) of the fine colour 1.
template <class MT, class DT, class VT, int ND>
__global__ void __launch_bounds__(SELL_TPB) k_bco_black_dia(DV<MT, DT> A, int s0, int s1, const double* r,
                                                             const VT* __restrict__ uinv, VT* __restrict__ z) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    pdl_launch_dependents();
    const int row = dia_row(A, s);
    VT v[ND];
    dia_load<ND, VT>(A, s, v);
    const VT dg = Cv<VT>::f(A.diag[s]);
    pdl_wait();
    if (row < 0) return;
    const VT ui = uinv[row];
    const VT fr = Cv<VT>::f(r[row]);
    const VT zr = z[row];
    const VT dot = dia_dot<ND, VT>(v, A.off, row, A.n, z);
    z[row] = zr + (fr - (dg * zr + dot)) * ui;
}

// ---------------------------------------------------------------------------------------------
// Deterministic reductions: block tree, then the last block to finish sums the partials in order.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (valid in thread 0).
__device__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

// Write this block's partial; returns true in every thread of the last block to arrive, which
// then holds the total (in thread 0) of all partials, summed in block-index order.
__device__ bool finish_sum(double v, double* part, unsigned* ctr, double* total) {
    __shared__ bool last;
    v = block_sum(v);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = v;
        __threadfence();
        last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double t = 0.0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x) t += __ldcg(&part[j]);
    t = block_sum(t);
    if (threadIdx.x == 0) { *total = t; *ctr = 0u; }
    return true;
}

// ---------------------------------------------------------------------------------------------
// PCG kernels (textbook PCG; the order of the oracle's loop)
// ---------------------------------------------------------------------------------------------
__global__ void k_pcg_init(int n, const double* b, double* __restrict__ x, double* __restrict__ r,
                           double* part, unsigned* ctr, PcgState* st, double* hist,
                           cudaGraphConditionalHandle cond) {
    pdl_launch_dependents();
    pdl_wait();
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        v += bi * bi;
    }
    double tot;
    if (finish_sum(v, part, ctr, &tot) && threadIdx.x == 0) {
        const double bn = sqrt(tot);
        st->bnorm = bn;
        st->k = 0;
        st->rz_old = 0.0;
        st->beta = 0.0;
        st->alpha = 0.0;
        st->res = bn > 0.0 ? 1.0 : 0.0;
        st->status = isfinite(bn) ? CPC_OK : CPC_EBREAKDOWN;
        hist[0] = st->res;
        cudaGraphSetConditional(cond, (bn > 0.0 && isfinite(bn) && st->maxit > 0) ? 1u : 0u);
        if (bn > 0.0 && isfinite(bn) && st->maxit <= 0) st->status = CPC_ENOCONV;
    }
}

// First node of every loop iteration: clear the loop condition.  Only the last block of
// k_pcg_update sets it again, so the loop cannot continue past an iteration whose final
// reduction did not complete.
__global__ void k_loop_guard(cudaGraphConditionalHandle cond) {
    pdl_launch_dependents();
    pdl_wait();
    cudaGraphSetConditional(cond, 0u);
}

template <class ZT>
__global__ void k_pcg_rz(int n, const double* r, const ZT* z, double* part, unsigned* ctr,
                         PcgState* st) {
    pdl_launch_dependents();
    pdl_wait();
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v += r[i] * cvt_d(z[i]);
    double tot;
    if (finish_sum(v, part, ctr, &tot) && threadIdx.x == 0) {
        if (!(tot > 0.0) || !isfinite(tot)) { if (st->status == CPC_OK) st->status = CPC_EBREAKDOWN; }
        st->beta = st->k == 0 ? 0.0 : tot / st->rz_old;
        st->rz = tot;
        st->rz_old = tot;
    }
}

template <class ZT>
__global__ void k_pcg_p(int n, const ZT* z, double* __restrict__ p, const PcgState* st) {
    pdl_launch_dependents();
    pdl_wait();
    const double beta = st->beta;
    const bool first = st->k == 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = first ? cvt_d(z[i]) : cvt_d(z[i]) + beta * p[i];
}

// q = A p and p.q; the last block forms alpha = (r.z) / (p.q).
template <int U>
__global__ void __launch_bounds__(SELL_TPB) k_pcg_spmv(SV<double, double> A, int nchunks, const double* p,
                                                        double* __restrict__ q, double* part, unsigned* ctr,
                                                        PcgState* st) {
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31, C = A.C, r = lane & (C - 1), g = lane / C;
    double v = 0.0;
    for (int k = blockIdx.x * WPB + (threadIdx.x >> 5); k < nchunks; k += gridDim.x * WPB) {
        const int s = k * C + r;
        const int row = A.perm[s];
        const bool own = g == 0 && row >= 0;
        const double pr = own ? p[row] : 0.0;
        const double dp = own ? A.diag[s] * pr : 0.0;
        double dot = sell_dot<double, false, U>(A.col, A.val, A.cptr[k] + g * C + r, A.cptr[k + 1], p);
        dot = sub_sum(dot, C);
        if (own) {
            const double acc = dp + dot;
            q[row] = acc;
            v += pr * acc;
        }
    }
    double tot;
    if (finish_sum(v, part, ctr, &tot) && threadIdx.x == 0) {
        st->pq = tot;
        if (!(tot > 0.0) || !isfinite(tot)) { if (st->status == CPC_OK) st->status = CPC_EBREAKDOWN; }
        st->alpha = st->status == CPC_OK ? st->rz / tot : 0.0;
    }
}

// k_pcg_spmv in diagonal form (grid-stride over the slots).
template <int ND>
__global__ void __launch_bounds__(SELL_TPB) k_pcg_spmv_dia(DV<double, double> A, const double* p,
                                                            double* __restrict__ q, double* part, unsigned* ctr,
                                                            PcgState* st) {
    pdl_launch_dependents();
    pdl_wait();
    double v = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A.nslots; s += gridDim.x * blockDim.x) {
        const int row = dia_row(A, s);
        if (row < 0) continue;
        double w[ND];
        dia_load<ND, double>(A, s, w);
        const double pr = p[row];
        const double acc = A.diag[s] * pr + dia_dot<ND, double>(w, A.off, row, A.n, p);
        q[row] = acc;
        v += pr * acc;
    }
    double tot;
    if (finish_sum(v, part, ctr, &tot) && threadIdx.x == 0) {
        st->pq = tot;
        if (!(tot > 0.0) || !isfinite(tot)) { if (st->status == CPC_OK) st->status = CPC_EBREAKDOWN; }
        st->alpha = st->status == CPC_OK ? st->rz / tot : 0.0;
    }
}

// x += alpha p, r -= alpha q, ||r||; the last block updates the iteration count, the residual
// history and the loop condition.
__global__ void k_pcg_update(int n, double* __restrict__ x, double* __restrict__ r, const double* p,
                             const double* q, double* part, unsigned* ctr, PcgState* st, double* hist,
                             int hist_cap, cudaGraphConditionalHandle cond) {
    pdl_launch_dependents();
    pdl_wait();
    const double alpha = st->alpha;
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v += ri * ri;
    }
    double tot;
    if (finish_sum(v, part, ctr, &tot) && threadIdx.x == 0) {
        unsigned go = 0u;
        if (st->status == CPC_OK) {
            const int k = st->k + 1;
            st->k = k;
            st->rr = tot;
            const double res = sqrt(tot) / st->bnorm;
            st->res = res;
            if (k < hist_cap) hist[k] = res;
            if (!isfinite(res)) st->status = CPC_EBREAKDOWN;
            else if (res < st->tol) st->status = CPC_OK;
            else if (k >= st->maxit) st->status = CPC_ENOCONV;
            else go = 1u;
        }
        cudaGraphSetConditional(cond, go);
    }
}

// ---------------------------------------------------------------------------------------------
// Recording helpers (launch sequences; captured into graphs or run directly)
// ---------------------------------------------------------------------------------------------
template <class VT> VT* lx(Level& L);
template <class VT> VT* lf(Level& L);
template <class VT> VT* lr(Level& L);
template <> double* lx<double>(Level& L) { return L.x64.p; }
template <> double* lf<double>(Level& L) { return L.f64.p; }
template <> double* lr<double>(Level& L) { return L.r64.p; }
template <> float* lx<float>(Level& L) { return L.x32.p; }
template <> float* lf<float>(Level& L) { return L.f32.p; }
template <> float* lr<float>(Level& L) { return L.r32.p; }

template <class VT> const VT* ainv(const Handle& h);
template <> const double* ainv<double>(const Handle& h) { return h.Ainv.p; }
template <> const float* ainv<float>(const Handle& h) { return h.Ainv32.p; }

// Warps per block of a colour step (or a triangular-solve level) over `chunks` SELL chunks (one
// warp each).  FP64 issue is
// about two lanes per clock per SM on this part, so a warp's row product occupies its SM's FP64
// pipe for 16 clocks per entry per lane: a colour step packed into four-warp blocks on a few SMs
// waits on their FP64 pipes, while one-warp blocks spread it over every SM.  Steps wide enough to
// give every SM four warps keep four-warp blocks (measured: one-warp blocks were slower there).
int gs_block_warps(int chunks) {
    static const int sms = [] {
        int dev = 0, n = 0;
        CPC_CK(cudaGetDevice(&dev));
        CPC_CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        return n;
    }();
    return chunks >= 4 * sms ? WPB : 1;
}

template <class FT, class VT>
void rec_gs(Level& L, int c, const FT* f, VT* x, cudaStream_t s) {
    const int c0 = L.S.seg[c], c1 = L.S.seg[c + 1];
    if (c1 <= c0) return;
    if (L.S.ndiag) {
        const int s0 = c0 * L.S.C, s1 = c1 * L.S.C;
        const bool pk = std::is_same<VT, double>::value ? L.S.gval.p != nullptr : L.S.gval32.p != nullptr;
        with_nd(L.S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value) {
                if (pk)
                    launch(k_gs_pk<double, double, FT, VT, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                           dview(L.S, L.n, (const double*)L.S.gval.p, (const double*)L.S.dinv.p, false), s0, s1, f, x);
                else
                    launch(k_gs_dia<double, double, FT, VT, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                           dview(L.S, L.n, (const double*)L.S.dval.p, (const double*)L.S.dinv.p, false), s0, s1, f, x);
            } else {
                if (pk)
                    launch(k_gs_pk<float, float, FT, VT, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                           dview(L.S, L.n, (const float*)L.S.gval32.p, (const float*)L.S.dinv32.p, false), s0, s1, f, x);
                else
                    launch(k_gs_dia<float, float, FT, VT, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                           dview(L.S, L.n, (const float*)L.S.dval32.p, (const float*)L.S.dinv32.p, false), s0, s1, f, x);
            }
        });
        return;
    }
    const int w = gs_block_warps(c1 - c0);
    const int g = (c1 - c0 + w - 1) / w, tpb = 32 * w;
    with_u_gs(L.S.lanes, [&](auto u) {
        constexpr int U = decltype(u)::value;
        if constexpr (std::is_same<VT, double>::value) {
            launch(k_gs<double, double, FT, VT, U>, g, tpb, s, view(L.S, (const double*)L.S.val.p, (const double*)L.S.dinv.p), c0, c1, f, x);
        } else {
            if (L.vt == VT_BF16)
                launch(k_gs<__nv_bfloat16, float, FT, VT, U>, g, tpb, s, view(L.S, (const __nv_bfloat16*)L.S.val16.p, (const float*)L.S.dinv32.p), c0, c1, f, x);
            else
                launch(k_gs<float, float, FT, VT, U>, g, tpb, s, view(L.S, (const float*)L.S.val32.p, (const float*)L.S.dinv32.p), c0, c1, f, x);
        }
    });
}

template <class FT, class VT>
void rec_resid_level(Level& L, const FT* f, const VT* x, VT* r, cudaStream_t s, bool after_sweep = false) {
    if (L.S.ndiag && after_sweep && L.ncolours == 2) {      // the last colour's residual is zero
        const int s1 = L.S.seg[1] * L.S.C;
        with_nd(L.S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                launch(k_resid_dia_first<double, double, FT, VT, VT, ND>, slot_blocks(L.S.nslots), SELL_TPB, s,
                       dview(L.S, L.n, (const double*)L.S.dval.p, (const double*)L.S.diag.p, false), s1, f, x, r);
            else
                launch(k_resid_dia_first<float, float, FT, VT, VT, ND>, slot_blocks(L.S.nslots), SELL_TPB, s,
                       dview(L.S, L.n, (const float*)L.S.dval32.p, (const float*)L.S.diag32.p, false), s1, f, x, r);
        });
        return;
    }
    if (L.S.ndiag) {
        with_nd(L.S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                launch(k_resid_dia<double, double, FT, VT, VT, ND>, slot_blocks(L.S.nslots), SELL_TPB, s,
                       dview(L.S, L.n, (const double*)L.S.dval.p, (const double*)L.S.diag.p, false), 0, L.S.nslots,
                       f, x, r);
            else
                launch(k_resid_dia<float, float, FT, VT, VT, ND>, slot_blocks(L.S.nslots), SELL_TPB, s,
                       dview(L.S, L.n, (const float*)L.S.dval32.p, (const float*)L.S.diag32.p, false), 0, L.S.nslots,
                       f, x, r);
        });
        return;
    }
    const int g = blocks_for_chunks(L.S.nchunks);
    with_u(L.S.lanes, [&](auto u) {
        constexpr int U = decltype(u)::value;
        if constexpr (std::is_same<VT, double>::value) {
            launch(k_resid<double, double, FT, VT, VT, U>, g, SELL_TPB, s, view(L.S, (const double*)L.S.val.p, (const double*)L.S.diag.p), L.S.nchunks, f, (const VT*)x, r);
        } else {
            if (L.vt == VT_BF16)
                launch(k_resid<__nv_bfloat16, float, FT, VT, VT, U>, g, SELL_TPB, s,
                       view(L.S, (const __nv_bfloat16*)L.S.val16.p, (const float*)L.S.diag32.p), L.S.nchunks, f, (const VT*)x, r);
            else
                launch(k_resid<float, float, FT, VT, VT, U>, g, SELL_TPB, s,
                       view(L.S, (const float*)L.S.val32.p, (const float*)L.S.diag32.p), L.S.nchunks, f, (const VT*)x, r);
        }
    });
}

template <class VT>
SV<VT, VT> full_view(const Sell& S) {
    if constexpr (std::is_same<VT, double>::value) return view(S, S.val.p, (const double*)nullptr);
    else return view(S, (const float*)S.val32.p, (const float*)nullptr);
}

template <class VT> void rec_fine_resid(Handle& h, const double* r, const VT* z, VT* t, cudaStream_t s);
template <class TT, class VT> void rec_ic_solve(Handle& h, const TT* t, VT* y, VT* w, VT* zadd, cudaStream_t s);
template <class VT> VT* ft(Handle& h);
template <class VT> VT* fy(Handle& h);

// One IC(0) smoothing step on the finest level, x <- x + B (f - A x) (AMG(ILU(0)), Section 5).
template <class VT>
void rec_ic_smooth(Handle& h, const double* f, VT* x, bool zero_guess, cudaStream_t s) {
    if (zero_guess) {
        rec_ic_solve<double, VT>(h, f, fy<VT>(h), x, (VT*)nullptr, s);      // x = B f
    } else {
        VT* t = ft<VT>(h);
        rec_fine_resid<VT>(h, f, x, t, s);
        rec_ic_solve<VT, VT>(h, t, fy<VT>(h), t, x, s);
    }
}

template <class VT> const VT* dnat(const Level& L);
template <> const double* dnat<double>(const Level& L) { return L.dnat64.p; }
template <> const float* dnat<float>(const Level& L) { return L.dnat32.p; }

// Algorithm 3.2 from level l: x <- V-cycle(f, initial guess x) (zero guess when zero_guess).  With
// ilu, the finest level is smoothed by IC(0) steps instead of Gauss-Seidel sweeps.  With
// first_done the caller has already applied the first colour step from the zero guess (and
// zeroed the other rows), so the forward sweep starts at colour 1.  A Gauss-Seidel step from
// zero on colour 0 reads only zeros, so x_i = (f_i - 0) / a_ii = f_i / a_ii exactly.
template <class FT, class VT>
void rec_vcycle(Handle& h, int l, const FT* f, VT* x, bool zero_guess, cudaStream_t s, bool ilu = false,
                bool first_done = false) {
    const int nl = (int)h.lev.size();
    Level& L = h.lev[l];
    if (l == nl - 1) {                                          // step 2(b): exact coarsest solve
        launch(k_coarse<VT, FT, VT>, std::max(1, (L.n + 7) / 8), 256, s, L.n, ainv<VT>(h), f, x);
        return;
    }
    Level& C = h.lev[l + 1];
    const bool ilu_here = ilu && l == 0;
    if constexpr (std::is_same<FT, double>::value) {
        if (ilu_here) rec_ic_smooth<VT>(h, f, x, zero_guess, s);          // (1) IC(0) step
    }
    if (!ilu_here) {
        int c0 = 0;
        if (first_done) {
            c0 = 1;
        } else if (zero_guess) {
            launch(k_zero_first<FT, VT>, vec_blocks(L.n), VEC_TPB, s, (int64_t)L.n, f, (const int*)L.colour.p,
                   dnat<VT>(L), x);
            c0 = 1;
        }
        for (int c = c0; c < L.ncolours; ++c) rec_gs(L, c, f, x, s);       // (1) S_l: colours ascending
    }
    rec_resid_level(L, f, x, lr<VT>(L), s, !ilu_here);                  // (2a) r = f - A u
    if (l + 1 >= h.tail_start) {                                         // (2a) f_c = R r, x_c = 0
        with_u(L.SR.lanes, [&](auto u) {
            launch(k_restrict_zero<VT, VT, decltype(u)::value>, blocks_for_chunks(L.SR.nchunks), SELL_TPB, s,
                   full_view<VT>(L.SR), L.SR.nchunks, (const VT*)lr<VT>(L), lf<VT>(C), lx<VT>(C));
        });
        record_tail(h, l + 1, lf<VT>(C), lx<VT>(C), s);                  // (2b) the coarser levels, one kernel
    } else if (l + 1 == nl - 1) {                                       // (2a) f_c = R r
        with_u(L.SR.lanes, [&](auto u) {
            launch(k_apply_full<VT, VT, decltype(u)::value>, blocks_for_chunks(L.SR.nchunks), SELL_TPB, s,
                   full_view<VT>(L.SR), L.SR.nchunks, (const VT*)lr<VT>(L), lf<VT>(C));
        });
        rec_vcycle<VT, VT>(h, l + 1, lf<VT>(C), lx<VT>(C), true, s);     // (2b) exact coarsest solve
    } else {                                                             // (2a) f_c = R r, first colour step
        with_u(L.SR.lanes, [&](auto u) {
            launch(k_restrict_first<VT, VT, decltype(u)::value>, blocks_for_chunks(L.SR.nchunks), SELL_TPB, s,
                   full_view<VT>(L.SR), L.SR.nchunks, (const VT*)lr<VT>(L), lf<VT>(C), lx<VT>(C),
                   (const int*)C.colour.p, dnat<VT>(C));
        });
        rec_vcycle<VT, VT>(h, l + 1, lf<VT>(C), lx<VT>(C), true, s, false, true);   // (2b) zero initial guess
    }
    with_u(L.SP.lanes, [&](auto u) {                                     // (2c)
        launch(k_prolong<VT, VT, decltype(u)::value>, blocks_for_chunks(L.SP.nchunks), SELL_TPB, s,
               full_view<VT>(L.SP), L.SP.nchunks, (const VT*)lx<VT>(C), x);
    });
    if constexpr (std::is_same<FT, double>::value) {
        if (ilu_here) {
            rec_ic_smooth<VT>(h, f, x, false, s);                          // (3) IC(0) step (B = B^T)
            return;
        }
    }
    for (int c = L.ncolours - 1; c >= 0; --c) rec_gs(L, c, f, x, s);     // (3) S_l^T: colours descending
}

// t = r - A z with the fine A in the preconditioner's precision.
template <class VT>
void rec_fine_resid(Handle& h, const double* r, const VT* z, VT* t, cudaStream_t s) {
    const Sell& A = h.Anat;
    if (A.ndiag) {
        with_nd(A.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                launch(k_resid_dia<double, double, double, VT, VT, ND>, slot_blocks(A.nslots), SELL_TPB, s,
                       dview(A, h.n, (const double*)A.dval.p, (const double*)A.diag.p, true), 0, A.nslots, r, z, t);
            else
                launch(k_resid_dia<float, float, double, VT, VT, ND>, slot_blocks(A.nslots), SELL_TPB, s,
                       dview(A, h.n, (const float*)A.dval32.p, (const float*)A.diag32.p, true), 0, A.nslots, r, z, t);
        });
        return;
    }
    const int g = blocks_for_chunks(A.nchunks);
    with_u(A.lanes, [&](auto u) {
        constexpr int U = decltype(u)::value;
        if constexpr (std::is_same<VT, double>::value)
            launch(k_resid<double, double, double, VT, VT, U>, g, SELL_TPB, s, view(A, (const double*)A.val.p, (const double*)A.diag.p), A.nchunks, r, z, t);
        else
            launch(k_resid<float, float, double, VT, VT, U>, g, SELL_TPB, s, view(A, (const float*)A.val32.p, (const float*)A.diag32.p), A.nchunks, r, z, t);
    });
}

// w = (LU)^{-1} t level by level; with zadd, z += w as well.
template <class TT, class VT>
void rec_ic_solve(Handle& h, const TT* t, VT* y, VT* w, VT* zadd, cudaStream_t s) {
    const Sell& L = h.L;
    const Sell& U = h.U;
    SV<VT, VT> lv, uv;
    if constexpr (std::is_same<VT, double>::value) {
        lv = view(L, L.val.p, (const double*)nullptr);
        uv = view(U, U.val.p, U.dinv.p);
    } else {
        lv = view(L, (const float*)L.val32.p, (const float*)nullptr);
        uv = view(U, (const float*)U.val32.p, (const float*)U.dinv32.p);
    }
    for (int g = 0; g + 1 < (int)L.seg.size(); ++g) {
        const int c0 = L.seg[g], c1 = L.seg[g + 1];
        const int w = gs_block_warps(c1 - c0);
        with_u(L.lanes, [&](auto u) {
            launch(k_lsolve<VT, TT, VT, decltype(u)::value>, (c1 - c0 + w - 1) / w, 32 * w, s, lv, c0, c1, t, y);
        });
    }
    for (int g = 0; g + 1 < (int)U.seg.size(); ++g) {
        const int c0 = U.seg[g], c1 = U.seg[g + 1];
        const int wb = gs_block_warps(c1 - c0);
        with_u(U.lanes, [&](auto u) {
            launch(k_usolve<VT, VT, decltype(u)::value>, (c1 - c0 + wb - 1) / wb, 32 * wb, s, uv, c0, c1,
                   (const VT*)y, w, zadd);
        });
    }
}

// B_co step (2) with red-black IC(0), right after step (1): black rows only (k_bco_black).
template <class VT>
void rec_bco_black(Handle& h, const double* r, VT* z, cudaStream_t s) {
    const Level& L0 = h.lev[0];
    const Sell& S = L0.S;
    const int c0 = S.seg[1], c1 = S.seg[2];
    if (c1 <= c0) return;
    if (S.ndiag) {
        const int s0 = c0 * S.C, s1 = c1 * S.C;
        with_nd(S.ndiag, [&](auto nd) {
            constexpr int ND = decltype(nd)::value;
            if constexpr (std::is_same<VT, double>::value)
                launch(k_bco_black_dia<double, double, double, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                       dview(S, L0.n, (const double*)S.dval.p, (const double*)S.diag.p, false), s0, s1, r,
                       (const double*)h.ic_uinv64.p, z);
            else
                launch(k_bco_black_dia<float, float, float, ND>, slot_blocks(s1 - s0), SELL_TPB, s,
                       dview(S, L0.n, (const float*)S.dval32.p, (const float*)S.diag32.p, false), s0, s1, r,
                       (const float*)h.ic_uinv32.p, z);
        });
        return;
    }
    with_u(S.lanes, [&](auto u) {
        if constexpr (std::is_same<VT, double>::value)
            launch(k_bco_black<double, double, double, decltype(u)::value>, blocks_for_chunks(c1 - c0), SELL_TPB, s,
                   view(S, (const double*)S.val.p, (const double*)S.diag.p), c0, c1, r, (const double*)h.ic_uinv64.p, z);
        else
            launch(k_bco_black<float, float, float, decltype(u)::value>, blocks_for_chunks(c1 - c0), SELL_TPB, s,
                   view(S, (const float*)S.val32.p, (const float*)S.diag32.p), c0, c1, r, (const float*)h.ic_uinv32.p, z);
    });
}

template <class VT> VT* ft(Handle& h);
template <> double* ft<double>(Handle& h) { return h.t.p; }
template <> float* ft<float>(Handle& h) { return h.t32.p; }
template <class VT> VT* fy(Handle& h);
template <> double* fy<double>(Handle& h) { return h.y.p; }
template <> float* fy<float>(Handle& h) { return h.y32.p; }

// z = M r for the chosen preconditioner (z in the preconditioner's vector type).
template <class VT>
void rec_precond_t(Handle& h, int which, const double* r, VT* z, cudaStream_t s) {
    VT* t = ft<VT>(h);
    VT* y = fy<VT>(h);
    switch (which) {
        case CPC_PRECOND_BCO:                         // Algorithm 2.1 with u^{k,0} = 0
            rec_vcycle<double, VT>(h, 0, r, z, true, s);        // (1) z = S r
            if (h.ic_rb) {                                      // (2) z += B (r - A z)
                rec_bco_black<VT>(h, r, z, s);
            } else {
                rec_fine_resid<VT>(h, r, z, t, s);
                rec_ic_solve<VT, VT>(h, t, y, t, z, s);
            }
            rec_vcycle<double, VT>(h, 0, r, z, false, s);       // (3) z += S^T (r - A z), S^T = S
            break;
        case CPC_PRECOND_AMG:                         // S~: two cycles
            rec_vcycle<double, VT>(h, 0, r, z, true, s);
            rec_vcycle<double, VT>(h, 0, r, z, false, s);
            break;
        case CPC_PRECOND_IC0:
            rec_ic_solve<double, VT>(h, r, y, z, (VT*)nullptr, s);
            break;
        case CPC_PRECOND_AMG_ILU:                     // two cycles with IC(0) as the finest smoother
            rec_vcycle<double, VT>(h, 0, r, z, true, s, true);
            rec_vcycle<double, VT>(h, 0, r, z, false, s, true);
            break;
        case CPC_PRECOND_BHAT:                        // S~ r + B r
            rec_vcycle<double, VT>(h, 0, r, z, true, s);
            rec_vcycle<double, VT>(h, 0, r, z, false, s);
            rec_ic_solve<double, VT>(h, r, y, t, z, s);
            break;
        default:
            launch(k_copy<double, VT>, vec_blocks(h.n), VEC_TPB, s, (int64_t)h.n, r, z);
            break;
    }
}

bool fp64(const Handle& h) { return h.opt.precision == CPC_PREC_FP64; }

void check_which(int which) {
    if (which < 0 || which >= NPRECOND) fail(CPC_EINVAL, "unknown preconditioner");
}

}  // namespace

// =============================================================================================
void record_precond(Handle& h, int which, const double* r, void* z, cudaStream_t s) {
    check_which(which);
    if (fp64(h)) rec_precond_t<double>(h, which, r, (double*)z, s);
    else rec_precond_t<float>(h, which, r, (float*)z, s);
}

void apply_precond(Handle& h, int which, const double* r, double* z) {
    check_which(which);
    cudaStream_t s = h.s;
    if (fp64(h)) {
        rec_precond_t<double>(h, which, r, z, s);
    } else {
        rec_precond_t<float>(h, which, r, h.z32.p, s);
        launch(k_copy<float, double>, vec_blocks(h.n), VEC_TPB, s, (int64_t)h.n, (const float*)h.z32.p, z);
    }
    CPC_LAUNCH_CK();
}

void spmv_fine(Handle& h, const double* x, double* y, cudaStream_t s) {
    const Sell& A = h.Anat;
    if (A.ndiag) {
        with_nd(A.ndiag, [&](auto nd) {
            launch(k_spmv_dia<double, double, double, double, decltype(nd)::value>, slot_blocks(A.nslots), SELL_TPB, s,
                   dview(A, h.n, (const double*)A.dval.p, (const double*)A.diag.p, true), x, y);
        });
        CPC_LAUNCH_CK();
        return;
    }
    with_u(A.lanes, [&](auto u) {
        launch(k_spmv<double, double, double, double, decltype(u)::value>, blocks_for_chunks(A.nchunks), SELL_TPB, s,
               view(A, (const double*)A.val.p, (const double*)A.diag.p), A.nchunks, x, y);
    });
    CPC_LAUNCH_CK();
}

float time_gs_sweep(const Sell& S, int n) {
    AllocOn plain(nullptr);                 // f and x are used on cs, not on a setup stream
    cudaStream_t cs;
    CPC_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamSynchronize(s); cudaStreamDestroy(s); } } sg{cs};
    DBuf<double> f, x;
    f.alloc(n);
    x.alloc(n);
    CPC_CK(cudaMemsetAsync(f.p, 0, sizeof(double) * n, cs));
    CPC_CK(cudaMemsetAsync(x.p, 0, sizeof(double) * n, cs));
    CPC_CK(cudaStreamSynchronize(cs));
    constexpr int SWEEPS = 4;
    cudaGraph_t g;
    CPC_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < SWEEPS; ++k)
        for (size_t c = 0; c + 1 < S.seg.size(); ++c) {
            const int c0 = S.seg[c], c1 = S.seg[c + 1];
            if (c1 <= c0) continue;
            const int w = gs_block_warps(c1 - c0);
            with_u_gs(S.lanes, [&](auto u) {         // the launch shapes of the solve's colour steps
                launch(k_gs<double, double, double, double, decltype(u)::value>, (c1 - c0 + w - 1) / w, 32 * w,
                       cs, view(S, (const double*)S.val.p, (const double*)S.dinv.p), c0, c1, (const double*)f.p, x.p);
            });
        }
    CPC_CK(cudaStreamEndCapture(cs, &g));
    cudaGraphExec_t ge;
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CPC_CK(ie);
    struct GE { cudaGraphExec_t g; ~GE() { cudaGraphExecDestroy(g); } } gg{ge};
    cudaEvent_t e0, e1;
    CPC_CK(cudaEventCreate(&e0));
    CPC_CK(cudaEventCreate(&e1));
    struct EV { cudaEvent_t a, b; ~EV() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
    CPC_CK(cudaGraphLaunch(ge, cs));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        CPC_CK(cudaEventRecord(e0, cs));
        CPC_CK(cudaGraphLaunch(ge, cs));
        CPC_CK(cudaEventRecord(e1, cs));
        CPC_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CPC_CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms / SWEEPS);
    }
    return best;
}

void level_apply(Handle& h, int l, int op, const double* x, double* y) {
    const int nl = (int)h.lev.size();
    if (l < 0 || l >= nl) fail(CPC_EINVAL, "level out of range");
    if (!fp64(h)) fail(CPC_EINVAL, "level operators are inspected in FP64 mode only");
    Level& L = h.lev[l];
    cudaStream_t s = h.s;
    const bool last = l == nl - 1;
    switch (op) {
        case 0:
            if (l == 0) spmv_fine(h, x, y, s);
            else if (last) fail(CPC_EINVAL, "coarsest level has no sparse layout");
            else with_u(L.S.lanes, [&](auto u) {
                launch(k_spmv<double, double, double, double, decltype(u)::value>, blocks_for_chunks(L.S.nchunks),
                       SELL_TPB, s, view(L.S, (const double*)L.S.val.p, (const double*)L.S.diag.p), L.S.nchunks, x, y);
            });
            break;
        case 1:
        case 2:
            if (last) fail(CPC_EINVAL, "coarsest level has no smoother");
            launch(k_zero<double>, vec_blocks(L.n), VEC_TPB, s, (int64_t)L.n, y);
            if (op == 1) for (int c = 0; c < L.ncolours; ++c) rec_gs(L, c, x, y, s);
            else for (int c = L.ncolours - 1; c >= 0; --c) rec_gs(L, c, x, y, s);
            break;
        case 3:
            if (!last) fail(CPC_EINVAL, "not the coarsest level");
            launch(k_coarse<double, double, double>, std::max(1, (L.n + 7) / 8), 256, s, L.n, (const double*)h.Ainv.p, x, y);
            break;
        case 5:                                                   // sweep from the given y (no zeroing)
            if (last) fail(CPC_EINVAL, "coarsest level has no smoother");
            for (int c = 0; c < L.ncolours; ++c) rec_gs(L, c, x, y, s);
            break;
        case 4:
            if (l >= h.tail_start) {
                launch(k_zero<double>, vec_blocks(L.n), VEC_TPB, s, (int64_t)L.n, y);
                record_tail(h, l, x, y, s);
            } else {
                rec_vcycle<double, double>(h, l, x, y, true, s);
            }
            break;
        default:
            fail(CPC_EINVAL, "unknown level operator");
    }
    CPC_LAUNCH_CK();
}

// Microseconds per forward Gauss-Seidel sweep (colours ascending) of level l in the
// preconditioner's precision on the level's own work vectors, replayed from a CUDA graph as in the
// solve: reps sweeps per replay, the best of three replays after one warm-up.
int gs_resident_blocks(int lanes) {
    int dev = 0, sms = 0, per_sm = 0;
    CPC_CK(cudaGetDevice(&dev));
    CPC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    with_u_gs(lanes, [&](auto u) {
        CPC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_gs<double, double, double, double, decltype(u)::value>, SELL_TPB, 0));
    });
    return std::max(1, sms * per_sm);
}

double sweep_time_us(Handle& h, int l, int reps) {
    const int nl = (int)h.lev.size();
    if (l < 0 || l >= nl - 1) fail(CPC_EINVAL, "level has no smoother");
    if (reps < 1 || reps > 1000) fail(CPC_EINVAL, "reps out of range");
    Level& L = h.lev[l];
    cudaStream_t cs;
    CPC_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamSynchronize(s); cudaStreamDestroy(s); } } sg{cs};
    CPC_CK(cudaStreamSynchronize(h.s));
    cudaGraph_t g;
    CPC_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < reps; ++k)
        for (int c = 0; c < L.ncolours; ++c) {
            if (fp64(h)) rec_gs<double, double>(L, c, (const double*)L.f64.p, L.x64.p, cs);
            else rec_gs<float, float>(L, c, (const float*)L.f32.p, L.x32.p, cs);
        }
    CPC_CK(cudaStreamEndCapture(cs, &g));
    cudaGraphExec_t ge;
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CPC_CK(ie);
    struct GE { cudaGraphExec_t g; ~GE() { cudaGraphExecDestroy(g); } } gg{ge};
    cudaEvent_t e0, e1;
    CPC_CK(cudaEventCreate(&e0));
    CPC_CK(cudaEventCreate(&e1));
    struct EV { cudaEvent_t a, b; ~EV() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
    CPC_CK(cudaGraphLaunch(ge, cs));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        CPC_CK(cudaEventRecord(e0, cs));
        CPC_CK(cudaGraphLaunch(ge, cs));
        CPC_CK(cudaEventRecord(e1, cs));
        CPC_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CPC_CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    return 1000.0 * best / reps;
}

void destroy_graphs(Handle& h) {
    for (int i = 0; i < NPRECOND; ++i) {
        if (h.gexec[i]) cudaGraphExecDestroy(h.gexec[i]);
        if (h.graph[i]) cudaGraphDestroy(h.graph[i]);
        h.gexec[i] = nullptr;
        h.graph[i] = nullptr;
    }
}

// The whole PCG loop as one graph: init kernel, then a while node whose body is one iteration.
static void build_solve_graph(Handle& h, int which) {
    cudaStream_t cs;
    CPC_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cs};
    cudaGraph_t g;
    CPC_CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    CPC_CK(cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
    const int n = h.n;
    // init
    CPC_CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch(k_pcg_init, vec_blocks(n), VEC_TPB, cs, n, (const double*)h.b.p, h.x.p, h.r.p, h.partial.p, h.counter.p,
           h.state.p, h.hist.p, cond);
    CPC_CK(cudaStreamEndCapture(cs, &g));
    size_t nn = 0;
    CPC_CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CPC_CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CPC_CK(cudaGraphAddNode(&wnode, g, nodes.data(), nullptr, nn, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // body: one PCG iteration
    CPC_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const Sell& A = h.Anat;
    launch(k_loop_guard, 1, 32, cs, cond);
    if (fp64(h)) {
        rec_precond_t<double>(h, which, h.r.p, h.z.p, cs);
        launch(k_pcg_rz<double>, vec_blocks(n), VEC_TPB, cs, n, (const double*)h.r.p, (const double*)h.z.p, h.partial.p, h.counter.p, h.state.p);
        launch(k_pcg_p<double>, vec_blocks(n), VEC_TPB, cs, n, (const double*)h.z.p, h.p.p, (const PcgState*)h.state.p);
    } else {
        rec_precond_t<float>(h, which, h.r.p, h.z32.p, cs);
        launch(k_pcg_rz<float>, vec_blocks(n), VEC_TPB, cs, n, (const double*)h.r.p, (const float*)h.z32.p, h.partial.p, h.counter.p, h.state.p);
        launch(k_pcg_p<float>, vec_blocks(n), VEC_TPB, cs, n, (const float*)h.z32.p, h.p.p, (const PcgState*)h.state.p);
    }
    if (A.ndiag) {
        with_nd(A.ndiag, [&](auto nd) {
            launch(k_pcg_spmv_dia<decltype(nd)::value>, std::min(slot_blocks(A.nslots), NPART), SELL_TPB, cs,
                   dview(A, h.n, (const double*)A.dval.p, (const double*)A.diag.p, true), (const double*)h.p.p,
                   h.q.p, h.partial.p, h.counter.p, h.state.p);
        });
    } else {
        with_u(A.lanes, [&](auto u) {
            launch(k_pcg_spmv<decltype(u)::value>, std::min(blocks_for_chunks(A.nchunks), NPART), SELL_TPB, cs,
                   view(A, (const double*)A.val.p, (const double*)A.diag.p), A.nchunks, (const double*)h.p.p, h.q.p,
                   h.partial.p, h.counter.p, h.state.p);
        });
    }
    launch(k_pcg_update, vec_blocks(n), VEC_TPB, cs, n, h.x.p, h.r.p, (const double*)h.p.p, (const double*)h.q.p,
           h.partial.p, h.counter.p, h.state.p, h.hist.p, (int)HIST_CAP, cond);
    CPC_CK(cudaStreamEndCapture(cs, &body));
    CPC_LAUNCH_CK();
    size_t nb = 0;
    CPC_CK(cudaGraphGetNodes(body, nullptr, &nb));
    h.body_nodes[which] = (int64_t)nb;
    cudaGraphExec_t ge;
    CPC_CK(cudaGraphInstantiate(&ge, g, 0));
    h.graph[which] = g;
    h.gexec[which] = ge;
}

void ensure_solve_graph(Handle& h, int which) {
    check_which(which);
    if (!h.gexec[which]) build_solve_graph(h, which);
}

void solve_pcg(Handle& h, const double* b, double* x, double tol, int maxit, int* iters, double* res_hist,
               int hist_cap, int* status) {
    const int which = h.opt.precond;
    check_which(which);
    if (!h.gexec[which]) build_solve_graph(h, which);
    cudaStream_t s = h.s;
    const int n = h.n;
    // parameters for this run, then the graph
    PcgState init{};
    init.tol = tol;
    init.maxit = maxit;
    CPC_CK(cudaMemcpyAsync(h.state.p, &init, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    CPC_CK(cudaMemcpyAsync(h.b.p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CPC_CK(cudaGraphLaunch(h.gexec[which], s));
    CPC_CK(cudaMemcpyAsync(x, h.x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    PcgState out{};
    CPC_CK(cudaMemcpyAsync(&out, h.state.p, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    *iters = out.k;
    *status = out.status;
    if (res_hist && hist_cap > 0) {
        const int cnt = std::min(std::min(hist_cap, out.k + 1), HIST_CAP);
        CPC_CK(cudaMemcpy(res_hist, h.hist.p, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    }
}

}  // namespace cpc
