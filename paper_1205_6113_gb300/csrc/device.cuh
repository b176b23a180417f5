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

// sum_w val[o_w] * x[col[o_w]] over one SELL row (entries o = o0, o0+32, ... < e).  Eight column
// indices and values are loaded first, then the eight gathers, so that each thread keeps eight
// independent loads in flight instead of a chain of dependent ones.  Padding (col < 0) is skipped
// without a load.  Products are added in entry order.  With WAIT, the first batch of the matrix
// row is loaded before pdl_wait() and the vector only after it.
template <class VT, bool WAIT = false, class MT, class XT>
__device__ __forceinline__ VT sell_dot(const int* __restrict__ col, const MT* __restrict__ val, int o, int e,
                                       const XT* x) {
    constexpr int U = 8;
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

// As sell_dot, with the gathered vector read through L2 only (ld.global.cg): for vectors written
// earlier in the same kernel by other thread blocks of the cluster.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

template <class VT, class MT, class XT>
__device__ __forceinline__ VT sell_dot_cg(const int* __restrict__ col, const MT* __restrict__ val, int o, int e,
                                          const XT* x) {
    constexpr int U = 8;
    VT acc = VT(0);
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
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? Cv<VT>::f(ldcg(x + c[u])) : VT(0);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u] * xv[u];
    }
    return acc;
}

}  // namespace cpc
