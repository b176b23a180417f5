// device.cuh -- device helpers shared by the solve kernels: value conversions, SELL views and the
// batched SELL row product.
#pragma once

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
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// sum_w val[o_w] * x[col[o_w]] over one SELL row (entries o = o0, o0+32, ... < e).  U column
// indices and values are loaded first, then the U gathers, so that each thread keeps U independent
// loads in flight instead of a chain of dependent ones.  Padding (col < 0) is skipped without a
// load.  Products are added in entry order.  The caller picks U >= the most entries a lane holds
// (4, 6 or 8, and 12 or 16 for the Gauss-Seidel colour steps; Sell::lanes), so one batch covers a
// row and no product is spent on padding beyond the chunk width -- FP64 issue rate is scarce on
// this part.  With WAIT, the first batch of the
// matrix row is loaded before pdl_wait() and the vector only after it; after_wait() runs right
// after the wait, so that loads the caller issues there overlap the gathers.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <class VT, bool WAIT = false, int U = 8, class MT, class XT, class H = NoHook>
__device__ __forceinline__ VT sell_dot(const int* __restrict__ col, const MT* __restrict__ val, int o, int e,
                                       const XT* x, H&& after_wait = H{}) {
    VT acc = VT(0);
    if (WAIT) {
        int c[U];
        VT v[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int oo = o + u * 32;
            c[u] = oo < e ? col[oo] : -1;
            v[u] = oo < e ? Cv<VT>::f(val[oo]) : VT(0);
        }
        pdl_wait();
        after_wait();           // the caller's own loads of predecessor data, in flight with the gathers
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? Cv<VT>::f(x[c[u]]) : VT(0);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u] * xv[u];
        o += U * 32;
    }
    for (; o < e; o += U * 32) {
        int c[U];
        VT v[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int oo = o + u * 32;
            c[u] = oo < e ? col[oo] : -1;
            v[u] = oo < e ? Cv<VT>::f(val[oo]) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? Cv<VT>::f(x[c[u]]) : VT(0);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u] * xv[u];
    }
    return acc;
}

}  // namespace cpc
