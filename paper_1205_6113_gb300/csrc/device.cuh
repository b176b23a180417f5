// device.cuh -- device helpers shared by the solve kernels: value conversions, SELL views and the
// batched SELL row product.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace cpc {

__device__ __forceinline__ double cvt_d(double v) { return v; }
__device__ __forceinline__ double cvt_d(float v) { return (double)v; }
__device__ __forceinline__ float cvt_f(double v) { return (float)v; }
__device__ __forceinline__ float cvt_f(float v) { return v; }
__device__ __forceinline__ float cvt_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class VT> struct Cv;
template <> struct Cv<double> {
    template <class T> __device__ static __forceinline__ double f(T v) { return cvt_d(v); }
};
template <> struct Cv<float> {
    template <class T> __device__ static __forceinline__ float f(T v) { return cvt_f(v); }
};

template <class MT, class DT>
struct SV {       // SELL view passed by value
    int C;        // chunk height
    const int* __restrict__ perm;
    const int* __restrict__ cptr;
    const int* __restrict__ col;
    const MT* __restrict__ val;
    const DT* __restrict__ diag;
};

template <class MT, class DT>
inline SV<MT, DT> view(const Sell& S, const MT* val, const DT* diag) {
    return SV<MT, DT>{S.C, S.perm.p, S.cptr.p, S.col.p, val, diag};
}

// Programmatic dependent launch (sm_90+).  Kernels of the solve are launched with programmatic
// stream serialisation: each signals at its start that its successor may be scheduled, so the
// successor is resident before this kernel ends; the successor loads what does not depend on its
// predecessor (the matrix) and then waits in pdl_wait() until the predecessor grid has completed
// and its memory is visible.  Without a programmatic predecessor both are no-ops.
// A kernel of such a chain is resident while the kernels before it still write, so its reads of
// data that an earlier kernel of the chain writes (vectors, partial sums, scalars) must not take
// the non-coherent read-only path: pointers to such data are never declared const __restrict__
// (which lets the compiler use that path), only pointers to the matrices and layouts built at
// setup.  With read-only loads a kernel was seen to read values of the previous V-cycle.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One batch of exactly M entries per lane (entries o, o + 32, ... with oo < e; the others load
// nothing and add 0): loads, then (WAIT) the wait and the caller's hook, then the gathers, then the
// products in entry order.
template <int M, bool WAIT, class VT, class MT, class XT, class H>
__device__ __forceinline__ void sell_batch(const int* __restrict__ col, const MT* __restrict__ val, int o, int e,
                                           const XT* x, VT& acc, H& after_wait) {
    int c[M];
    VT v[M], xv[M];
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int oo = o + u * 32;
        c[u] = oo < e ? col[oo] : -1;
        v[u] = oo < e ? Cv<VT>::f(val[oo]) : VT(0);
    }
    if (WAIT) {
        pdl_wait();
        after_wait();           // the caller's own loads of predecessor data, in flight with the gathers
    }
#pragma unroll
    for (int u = 0; u < M; ++u) xv[u] = c[u] >= 0 ? Cv<VT>::f(x[c[u]]) : VT(0);
#pragma unroll
    for (int u = 0; u < M; ++u) acc += v[u] * xv[u];
}

template <int M, bool WAIT, int U, class VT, class MT, class XT, class H>
__device__ __forceinline__ void sell_batch_of(int m, const int* __restrict__ col, const MT* __restrict__ val, int o,
                                              int e, const XT* x, VT& acc, H& after_wait) {
    if constexpr (M <= U) {
        if (m == M) sell_batch<M, WAIT>(col, val, o, e, x, acc, after_wait);
        else sell_batch_of<M + 1, WAIT, U>(m, col, val, o, e, x, acc, after_wait);
    }
}

// sum_w val[o_w] * x[col[o_w]] over one SELL row (entries o = o0, o0+32, ... < e) of the chunk
// that the calling warp owns.  Entries are taken in batches: each lane loads a batch's column indices
// and values first, then its gathers, so it keeps the batch's loads in flight instead of a chain of
// dependent ones.  A batch holds m <= U entries per lane, m = the chunk's entries per lane left
// (the same for the whole warp, from the chunk start that lane 0 holds): a narrow chunk issues no
// loads and, above all, no FP64 products for padding, and FP64 issue is scarce on this part (FP32
// arithmetic keeps full batches of U, masked per lane: fewer registers, no dispatch).  Lanes
// with fewer entries than m load nothing for the extra ones and add 0.  Products are added in entry
// order.  U (4, 6 or 8, and 12 or 16 for the Gauss-Seidel colour steps) is at least the widest
// chunk's entries per lane (Sell::lanes), so one batch usually covers a row.  With WAIT, the first
// batch's matrix data is loaded before pdl_wait() and the vector only after it; after_wait() runs
// right after the wait, so that loads the caller issues there overlap the gathers.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <class VT, bool WAIT = false, int U = 8, class MT, class XT, class H = NoHook>
__device__ __forceinline__ VT sell_dot(const int* __restrict__ col, const MT* __restrict__ val, int o, int e,
                                       const XT* x, H&& after_wait = H{}) {
    VT acc = VT(0);
    if constexpr (!std::is_same<VT, double>::value) {
        // FP32 arithmetic is not short of issue slots: full batches of U, masked per lane (fewer
        // registers and no dispatch on the batch size)
        if (WAIT) {
            sell_batch<U, true>(col, val, o, e, x, acc, after_wait);
            o += U * 32;
        }
        for (; o < e; o += U * 32) sell_batch<U, false>(col, val, o, e, x, acc, after_wait);
        return acc;
    }
    const int cb = __shfl_sync(0xffffffffu, o, 0);            // lane 0: sub-lane 0, row 0 of the chunk
    int left = (e - cb + 31) >> 5;                              // entries per lane, warp-uniform
    if (WAIT) {
        const int m = left < U ? left : U;
        if (m == 0) {
            pdl_wait();
            after_wait();
        } else {
            sell_batch_of<1, true, U>(m, col, val, o, e, x, acc, after_wait);
        }
        o += U * 32;
        left -= U;
    }
    for (; left > 0; o += U * 32, left -= U) {
        const int m = left < U ? left : U;
        sell_batch_of<1, false, U>(m, col, val, o, e, x, acc, after_wait);
    }
    return acc;
}

}  // namespace cpc
