// tail.cu -- the V-cycle below the fine level (Algorithm 3.2 on levels >= tail_start) as ONE kernel
// on one thread-block cluster.
//
// Below the fine level every step of the cycle (one Gauss-Seidel colour, a residual, a restriction,
// the coarsest solve, a prolongation) is small: a few thousand to a few hundred thousand rows.  As
// separate launches each step costs a launch gap plus a dependent-load chain, and a cycle has
// ~200 of them.  Here the whole sub-cycle runs in one cluster of up to 16 CTAs (one per SM); the
// dependent steps are separated by hardware cluster barriers (barrier.cluster arrive/wait, with
// release/acquire semantics at cluster scope) instead of kernel boundaries.  Matrices are
// read-only; the level vectors are written and read inside the kernel by different CTAs, so they
// are loaded through L2 (ld.global.cg) after each barrier.
#include <cooperative_groups.h>

#include <algorithm>

#include "device.cuh"
#include "handle.cuh"

namespace cg = cooperative_groups;

namespace cpc {

namespace {

constexpr int TAIL_TPB = 512;
constexpr int TAIL_MAXL = 32;

struct TailLevel {
    int n, ncol, nchunks;
    int ca, cp, cr;                       // chunk heights of A_l, P_l, R_l
    const int* seg;                       // colour chunk boundaries [ncol + 1]
    const int* perm;
    const int* cptr;
    const int* col;
    const void* val;                      // off-diagonals (MT)
    const void* diag;                     // diagonal per slot (DT)
    int p_nchunks, r_nchunks;             // P_l (n_l x n_{l+1}) and R_l = P_l^T, natural rows
    const int* p_perm;
    const int* p_cptr;
    const int* p_col;
    const void* p_val;
    const int* r_perm;
    const int* r_cptr;
    const int* r_col;
    const void* r_val;
    void* x;
    void* f;
    void* r;
};

struct TailDesc {
    int nl;                               // levels in the tail, the last one is the coarsest
    int nc;                               // coarsest size
    const void* ainv;                     // dense inverse of the coarsest operator (VT)
    TailLevel lev[TAIL_MAXL];
};

template <class VT>
__device__ __forceinline__ VT t_sub_sum(VT v, int C) {
    for (int o = C; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gauss-Seidel on the rows of colour c: x_i = (f_i - sum_{j != i} a_ij x_j) / a_ii.
// A warp owns a chunk of C rows, 32 / C lanes per row (as in the single-level kernels).
template <class MT, class DT, class VT>
__device__ __forceinline__ void t_gs(const TailLevel& L, int c, const VT* f, VT* x, int gw, int nw, int lane) {
    const int k1 = L.seg[c + 1];
    const int C = L.ca, r = lane & (C - 1), g = lane / C;
    const MT* val = (const MT*)L.val;
    const DT* diag = (const DT*)L.diag;
    for (int k = L.seg[c] + gw; k < k1; k += nw) {
        const int s = k * C + r;
        const int row = L.perm[s];
        VT dot = sell_dot_cg<VT>(L.col, val, L.cptr[k] + g * C + r, L.cptr[k + 1], x);
        dot = t_sub_sum(dot, C);
        if (g == 0 && row >= 0) x[row] = (ldcg(f + row) - dot) / Cv<VT>::f(diag[s]);
    }
}

// r = f - A x
template <class MT, class DT, class VT>
__device__ __forceinline__ void t_resid(const TailLevel& L, const VT* f, const VT* x, VT* r, int gw, int nw, int lane) {
    const int C = L.ca, rr = lane & (C - 1), g = lane / C;
    const MT* val = (const MT*)L.val;
    const DT* diag = (const DT*)L.diag;
    for (int k = gw; k < L.nchunks; k += nw) {
        const int s = k * C + rr;
        const int row = L.perm[s];
        VT dot = sell_dot_cg<VT>(L.col, val, L.cptr[k] + g * C + rr, L.cptr[k + 1], x);
        dot = t_sub_sum(dot, C);
        if (g == 0 && row >= 0) r[row] = ldcg(f + row) - (Cv<VT>::f(diag[s]) * ldcg(x + row) + dot);
    }
}

// f_c = R r, and x_c = 0 (the coarse level starts from a zero guess)
template <class PT, class VT>
__device__ __forceinline__ void t_restrict(const TailLevel& L, const VT* r, VT* fc, VT* xc, int gw, int nw, int lane) {
    const int C = L.cr, rr = lane & (C - 1), g = lane / C;
    const PT* val = (const PT*)L.r_val;
    for (int k = gw; k < L.r_nchunks; k += nw) {
        const int row = L.r_perm[k * C + rr];
        VT dot = sell_dot_cg<VT>(L.r_col, val, L.r_cptr[k] + g * C + rr, L.r_cptr[k + 1], r);
        dot = t_sub_sum(dot, C);
        if (g == 0 && row >= 0) { fc[row] = dot; xc[row] = VT(0); }
    }
}

// x += P e
template <class PT, class VT>
__device__ __forceinline__ void t_prolong(const TailLevel& L, const VT* e, VT* x, int gw, int nw, int lane) {
    const int C = L.cp, rr = lane & (C - 1), g = lane / C;
    const PT* val = (const PT*)L.p_val;
    for (int k = gw; k < L.p_nchunks; k += nw) {
        const int row = L.p_perm[k * C + rr];
        VT dot = sell_dot_cg<VT>(L.p_col, val, L.p_cptr[k] + g * C + rr, L.p_cptr[k + 1], e);
        dot = t_sub_sum(dot, C);
        if (g == 0 && row >= 0) x[row] = ldcg(x + row) + dot;
    }
}

// x = A_c^{-1} f, one warp per row
template <class VT>
__device__ __forceinline__ void t_coarse(const VT* ainv, int n, const VT* f, VT* x, int gw, int nw, int lane) {
    for (int i = gw; i < n; i += nw) {
        VT acc = VT(0);
        for (int j = lane; j < n; j += 32) acc += ainv[(size_t)i * n + j] * ldcg(f + j);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = acc;
    }
}

// The cycle from tail level `start` (input f0, output x0 which the caller has set to the initial
// guess -- zero for a coarse-grid correction) down to the coarsest level and back.
template <class MT, class DT, class PT, class VT>
__global__ void __launch_bounds__(TAIL_TPB) k_tail(const TailDesc* __restrict__ D, int start, const VT* f0, VT* x0) {
    cg::cluster_group cl = cg::this_cluster();
    pdl_launch_dependents();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (TAIL_TPB / 32) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (TAIL_TPB / 32);
    const int nl = D->nl;
    for (int t = start; t < nl - 1; ++t) {                 // descent
        const TailLevel& L = D->lev[t];
        const TailLevel& C = D->lev[t + 1];
        const VT* f = t == start ? f0 : (const VT*)L.f;
        VT* x = t == start ? x0 : (VT*)L.x;
        for (int c = 0; c < L.ncol; ++c) {                  // (1) S_l: colours ascending
            t_gs<MT, DT, VT>(L, c, f, x, gw, nw, lane);
            cl.sync();
        }
        t_resid<MT, DT, VT>(L, f, x, (VT*)L.r, gw, nw, lane);
        cl.sync();
        t_restrict<PT, VT>(L, (const VT*)L.r, (VT*)C.f, (VT*)C.x, gw, nw, lane);   // (2a)
        cl.sync();
    }
    {                                                        // (2b) coarsest level
        const TailLevel& L = D->lev[nl - 1];
        const VT* f = nl - 1 == start ? f0 : (const VT*)L.f;
        VT* x = nl - 1 == start ? x0 : (VT*)L.x;
        t_coarse<VT>((const VT*)D->ainv, L.n, f, x, gw, nw, lane);
        cl.sync();
    }
    for (int t = nl - 2; t >= start; --t) {                 // ascent
        const TailLevel& L = D->lev[t];
        const TailLevel& C = D->lev[t + 1];
        const VT* f = t == start ? f0 : (const VT*)L.f;
        VT* x = t == start ? x0 : (VT*)L.x;
        t_prolong<PT, VT>(L, (const VT*)C.x, x, gw, nw, lane);                    // (2c)
        cl.sync();
        for (int c = L.ncol - 1; c >= 0; --c) {             // (3) S_l^T: colours descending
            t_gs<MT, DT, VT>(L, c, f, x, gw, nw, lane);
            cl.sync();
        }
    }
}

template <class MT, class DT, class PT, class VT>
void launch_tail(const Handle& h, int start, const VT* f0, VT* x0, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h.tail_cluster, 1, 1);
    cfg.blockDim = dim3(TAIL_TPB, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = h.tail_cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    CPC_CK(cudaLaunchKernelEx(&cfg, k_tail<MT, DT, PT, VT>, (const TailDesc*)h.tail_desc.p, start, f0, x0));
}

// Largest cluster (<= 16 CTAs, one per SM) that the device can schedule for this kernel.
template <class MT, class DT, class PT, class VT>
int pick_cluster() {
    auto k = k_tail<MT, DT, PT, VT>;
    CPC_CK(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int cs : {16, 8, 4, 2, 1}) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(TAIL_TPB, 1, 1);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0) return cs;
        cudaGetLastError();
    }
    fail(CPC_ECUDA, "no cluster configuration available for the coarse-level kernel");
    return 1;
}

}  // namespace

void setup_tail(Handle& h, int64_t tail_nnz_max) {
    const int nl = (int)h.lev.size();
    h.tail_start = nl;                     // no tail for a single-level hierarchy
    if (nl < 2) return;
    int t0 = 1;
    while (t0 < nl - 1 && h.lev[t0].A.nnz > tail_nnz_max) ++t0;
    if (nl - t0 > TAIL_MAXL) t0 = nl - TAIL_MAXL;
    h.tail_start = t0;
    TailDesc d{};
    d.nl = nl - t0;
    d.nc = h.nc;
    const bool f64 = h.opt.precision == CPC_PREC_FP64;
    d.ainv = f64 ? (const void*)h.Ainv.p : (const void*)h.Ainv32.p;
    h.tail_seg.resize(d.nl);
    for (int t = 0; t < d.nl; ++t) {
        Level& L = h.lev[t0 + t];
        TailLevel& T = d.lev[t];
        T.n = L.n;
        T.x = f64 ? (void*)L.x64.p : (void*)L.x32.p;
        T.f = f64 ? (void*)L.f64.p : (void*)L.f32.p;
        T.r = f64 ? (void*)L.r64.p : (void*)L.r32.p;
        if (t == d.nl - 1) continue;      // coarsest: dense solve only
        T.ncol = L.ncolours;
        T.nchunks = L.S.nchunks;
        T.ca = L.S.C;
        T.cp = L.SP.C;
        T.cr = L.SR.C;
        h.tail_seg[t].alloc(L.S.seg.size());
        CPC_CK(cudaMemcpy(h.tail_seg[t].p, L.S.seg.data(), sizeof(int) * L.S.seg.size(), cudaMemcpyHostToDevice));
        T.seg = h.tail_seg[t].p;
        T.perm = L.S.perm.p;
        T.cptr = L.S.cptr.p;
        T.col = L.S.col.p;
        if (f64) { T.val = L.S.val.p; T.diag = L.S.diag.p; }
        else { T.val = L.vt == VT_BF16 ? (const void*)L.S.val16.p : (const void*)L.S.val32.p; T.diag = L.S.diag32.p; }
        T.p_nchunks = L.SP.nchunks;
        T.p_perm = L.SP.perm.p;
        T.p_cptr = L.SP.cptr.p;
        T.p_col = L.SP.col.p;
        T.p_val = f64 ? (const void*)L.SP.val.p : (const void*)L.SP.val32.p;
        T.r_nchunks = L.SR.nchunks;
        T.r_perm = L.SR.perm.p;
        T.r_cptr = L.SR.cptr.p;
        T.r_col = L.SR.col.p;
        T.r_val = f64 ? (const void*)L.SR.val.p : (const void*)L.SR.val32.p;
    }
    h.tail_desc.alloc(sizeof(TailDesc));
    CPC_CK(cudaMemcpy(h.tail_desc.p, &d, sizeof(TailDesc), cudaMemcpyHostToDevice));
    const bool bf16 = h.opt.precision == CPC_PREC_FP32_BF16;
    if (f64) h.tail_cluster = pick_cluster<double, double, double, double>();
    else if (bf16) h.tail_cluster = pick_cluster<__nv_bfloat16, float, float, float>();
    else h.tail_cluster = pick_cluster<float, float, float, float>();
}

void record_tail(Handle& h, int level, const void* f0, void* x0, cudaStream_t s) {
    const int start = level - h.tail_start;
    if (h.opt.precision == CPC_PREC_FP64)
        launch_tail<double, double, double, double>(h, start, (const double*)f0, (double*)x0, s);
    else if (h.opt.precision == CPC_PREC_FP32_BF16)
        launch_tail<__nv_bfloat16, float, float, float>(h, start, (const float*)f0, (float*)x0, s);
    else
        launch_tail<float, float, float, float>(h, start, (const float*)f0, (float*)x0, s);
}

}  // namespace cpc
