// tail.cu -- the coarse end of the V-cycle (Algorithm 3.2 on levels >= tail_start) as ONE kernel on
// one thread-block cluster, with the coarse operators in shared memory and the level vectors in
// distributed shared memory.
//
// Below a few thousand rows a V-cycle step (one Gauss-Seidel colour, a residual, a restriction, the
// coarsest solve, a prolongation) is a few microseconds of launch latency and dependent L2 loads
// for very little work; the coarse levels have 20-25 colours each.  Here the levels that fit are
// cut into per-CTA images at setup: chunk k of every operator belongs to CTA k mod ncta, and a CTA
// copies its image (perm, local row offsets, columns, values, diagonal) into its shared memory at
// the start of the kernel, before griddepcontrol.wait, so the copy overlaps the previous kernel.
// Vector element i of every level lives in the shared memory of CTA i mod ncta and is read and
// written through distributed shared memory (mapa).  Consecutive steps are separated by the
// hardware cluster barrier (release/acquire at cluster scope).
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "handle.cuh"

namespace cg = cooperative_groups;

namespace cpc {

namespace {

constexpr int TAIL_TPB = 512;
constexpr int TAIL_MAXL = 16;
constexpr int TAIL_MAXCTA = 16;
constexpr size_t TAIL_SMEM = 224 * 1024;      // dynamic shared memory budget per CTA (227 KB maximum)

enum { A_CPTR, A_PERM, A_COL, A_DIAG, A_DINV, A_VAL, P_CPTR, P_PERM, P_COL, P_VAL, R_CPTR, R_PERM, R_COL, R_VAL, NSEC };

struct TLev {
    int n, ncol;
    int C, nck;                               // A_l: chunk height, chunks
    int CP, nckP, CR, nckR;                   // P_l, R_l
    const int* seg;                           // colour chunk boundaries (global) [ncol + 1]
    unsigned vx, vf, vr;                      // byte offsets of the x, f, r slices in the vector region
    unsigned off[TAIL_MAXCTA][NSEC];          // byte offsets of the sections in each CTA's image
};

struct TDesc {
    int nl, nc, ncta, lg;                     // levels (last = coarsest), coarsest size, CTAs, log2(ncta)
    unsigned vec_bytes;                       // vector region (same for every CTA)
    unsigned img_off[TAIL_MAXCTA], img_bytes[TAIL_MAXCTA];
    unsigned ainv_off[TAIL_MAXCTA];           // rows i = q ncta + rank of A_c^{-1} in the image
    const unsigned char* img;                 // all images, concatenated (global)
    TLev lev[TAIL_MAXL];
};

__device__ __forceinline__ int cdiv(int a, int b) { return a <= 0 ? 0 : (a + b - 1) / b; }

// Element i of a distributed vector whose local slice starts at byte offset v of the vector region.
template <class VT>
__device__ __forceinline__ VT* delem(cg::cluster_group& cl, unsigned char* vbase, unsigned v, int i, int ncta, int lg) {
    VT* local = reinterpret_cast<VT*>(vbase + v);
    return cl.map_shared_rank(local, (unsigned)(i & (ncta - 1))) + (i >> lg);
}

template <class VT>
__device__ __forceinline__ VT t_sub_sum(VT v, int C) {
    for (int o = C; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over one row of a local chunk: entries o = o0, o0 + 32, ... < e of the local arrays,
// gathered from the distributed vector at byte offset v.
template <class VT, class MT>
__device__ __forceinline__ VT t_dot(cg::cluster_group& cl, unsigned char* vbase, unsigned v, const int* col,
                                    const MT* val, int o, int e, int ncta, int lg) {
    constexpr int U = 8;
    VT acc = VT(0);
    for (; o < e; o += U * 32) {
        int c[U];
        VT a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int oo = o + u * 32;
            c[u] = oo < e ? col[oo] : -1;
            a[u] = oo < e ? Cv<VT>::f(val[oo]) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? *delem<VT>(cl, vbase, v, c[u], ncta, lg) : VT(0);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += a[u] * xv[u];
    }
    return acc;
}

template <class MT, class DT, class PT, class VT>
__global__ void __launch_bounds__(TAIL_TPB, 1) k_tail(const TDesc* __restrict__ D, int start, const VT* f0, VT* x0) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int ncta = D->ncta, lg = D->lg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = TAIL_TPB / 32;
    unsigned char* vb = smem;
    unsigned char* img = smem + D->vec_bytes;
    pdl_launch_dependents();
    {   // this CTA's image: independent of the previous kernel, so copied before the wait
        const uint4* src = reinterpret_cast<const uint4*>(D->img + D->img_off[rank]);
        uint4* dst = reinterpret_cast<uint4*>(img);
        const int n16 = (int)(D->img_bytes[rank] / 16);
        for (int i = threadIdx.x; i < n16; i += TAIL_TPB) dst[i] = src[i];
    }
    pdl_wait();
    const int nl = D->nl;
    {   // input: f of level `start` (own elements), zero initial guess
        const TLev& L = D->lev[start];
        VT* F = reinterpret_cast<VT*>(vb + L.vf);
        VT* X = reinterpret_cast<VT*>(vb + L.vx);
        for (int q = threadIdx.x; q * ncta + rank < L.n; q += TAIL_TPB) {
            F[q] = f0[q * ncta + rank];
            X[q] = VT(0);
        }
    }
    cl.sync();
    auto gs = [&](const TLev& L, int c) {   // Gauss-Seidel on colour c
        const int C = L.C, r = lane & (C - 1), g = lane / C;
        const int* cptr = reinterpret_cast<const int*>(img + L.off[rank][A_CPTR]);
        const int* perm = reinterpret_cast<const int*>(img + L.off[rank][A_PERM]);
        const int* col = reinterpret_cast<const int*>(img + L.off[rank][A_COL]);
        const DT* dinv = reinterpret_cast<const DT*>(img + L.off[rank][A_DINV]);
        const MT* val = reinterpret_cast<const MT*>(img + L.off[rank][A_VAL]);
        const int qa = cdiv(L.seg[c] - rank, ncta), qb = cdiv(L.seg[c + 1] - rank, ncta);
        for (int q = qa + warp; q < qb; q += NW) {
            const int row = perm[q * C + r];
            VT dot = t_dot<VT>(cl, vb, L.vx, col, val, cptr[q] + g * C + r, cptr[q + 1], ncta, lg);
            dot = t_sub_sum(dot, C);
            if (g == 0 && row >= 0)
                *delem<VT>(cl, vb, L.vx, row, ncta, lg) =
                    (*delem<VT>(cl, vb, L.vf, row, ncta, lg) - dot) * Cv<VT>::f(dinv[q * C + r]);
        }
    };
    for (int t = start; t < nl - 1; ++t) {                   // descent
        const TLev& L = D->lev[t];
        const TLev& Cn = D->lev[t + 1];
        for (int c = 0; c < L.ncol; ++c) { gs(L, c); cl.sync(); }           // (1) S_l
        {                                                                     // r = f - A x
            const int C = L.C, r = lane & (C - 1), g = lane / C;
            const int* cptr = reinterpret_cast<const int*>(img + L.off[rank][A_CPTR]);
            const int* perm = reinterpret_cast<const int*>(img + L.off[rank][A_PERM]);
            const int* col = reinterpret_cast<const int*>(img + L.off[rank][A_COL]);
            const DT* diag = reinterpret_cast<const DT*>(img + L.off[rank][A_DIAG]);
            const MT* val = reinterpret_cast<const MT*>(img + L.off[rank][A_VAL]);
            const int nq = cdiv(L.nck - rank, ncta);
            for (int q = warp; q < nq; q += NW) {
                const int row = perm[q * C + r];
                VT dot = t_dot<VT>(cl, vb, L.vx, col, val, cptr[q] + g * C + r, cptr[q + 1], ncta, lg);
                dot = t_sub_sum(dot, C);
                if (g == 0 && row >= 0)
                    *delem<VT>(cl, vb, L.vr, row, ncta, lg) = *delem<VT>(cl, vb, L.vf, row, ncta, lg) -
                        (Cv<VT>::f(diag[q * C + r]) * *delem<VT>(cl, vb, L.vx, row, ncta, lg) + dot);
            }
        }
        cl.sync();
        {                                                                     // (2a) f_c = R r, x_c = 0
            const int C = L.CR, r = lane & (C - 1), g = lane / C;
            const int* cptr = reinterpret_cast<const int*>(img + L.off[rank][R_CPTR]);
            const int* perm = reinterpret_cast<const int*>(img + L.off[rank][R_PERM]);
            const int* col = reinterpret_cast<const int*>(img + L.off[rank][R_COL]);
            const PT* val = reinterpret_cast<const PT*>(img + L.off[rank][R_VAL]);
            const int nq = cdiv(L.nckR - rank, ncta);
            for (int q = warp; q < nq; q += NW) {
                const int row = perm[q * C + r];
                VT dot = t_dot<VT>(cl, vb, L.vr, col, val, cptr[q] + g * C + r, cptr[q + 1], ncta, lg);
                dot = t_sub_sum(dot, C);
                if (g == 0 && row >= 0) {
                    *delem<VT>(cl, vb, Cn.vf, row, ncta, lg) = dot;
                    *delem<VT>(cl, vb, Cn.vx, row, ncta, lg) = VT(0);
                }
            }
        }
        cl.sync();
    }
    {                                                                         // (2b) coarsest, exact
        const TLev& L = D->lev[nl - 1];
        const int n = L.n;
        const VT* ai = reinterpret_cast<const VT*>(img + D->ainv_off[rank]);
        const int nq = cdiv(n - rank, ncta);
        for (int q = warp; q < nq; q += NW) {
            VT acc = VT(0);
            for (int j = lane; j < n; j += 32) acc += ai[(size_t)q * n + j] * *delem<VT>(cl, vb, L.vf, j, ncta, lg);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) *delem<VT>(cl, vb, L.vx, q * ncta + rank, ncta, lg) = acc;
        }
        cl.sync();
    }
    for (int t = nl - 2; t >= start; --t) {                  // ascent
        const TLev& L = D->lev[t];
        const TLev& Cn = D->lev[t + 1];
        {                                                                     // (2c) x += P e
            const int C = L.CP, r = lane & (C - 1), g = lane / C;
            const int* cptr = reinterpret_cast<const int*>(img + L.off[rank][P_CPTR]);
            const int* perm = reinterpret_cast<const int*>(img + L.off[rank][P_PERM]);
            const int* col = reinterpret_cast<const int*>(img + L.off[rank][P_COL]);
            const PT* val = reinterpret_cast<const PT*>(img + L.off[rank][P_VAL]);
            const int nq = cdiv(L.nckP - rank, ncta);
            for (int q = warp; q < nq; q += NW) {
                const int row = perm[q * C + r];
                VT dot = t_dot<VT>(cl, vb, Cn.vx, col, val, cptr[q] + g * C + r, cptr[q + 1], ncta, lg);
                dot = t_sub_sum(dot, C);
                if (g == 0 && row >= 0) *delem<VT>(cl, vb, L.vx, row, ncta, lg) += dot;
            }
        }
        cl.sync();
        for (int c = L.ncol - 1; c >= 0; --c) { gs(L, c); cl.sync(); }    // (3) S_l^T
    }
    {   // output: x of level `start` (own elements)
        const TLev& L = D->lev[start];
        const VT* X = reinterpret_cast<const VT*>(vb + L.vx);
        for (int q = threadIdx.x; q * ncta + rank < L.n; q += TAIL_TPB) x0[q * ncta + rank] = X[q];
    }
    cl.sync();
}

// ---------------------------------------------------------------------------------------------
// Setup: per-CTA images
// ---------------------------------------------------------------------------------------------
inline unsigned align16(size_t b) { return (unsigned)((b + 15) / 16 * 16); }

// Copy the chunks of one SELL operator into the per-CTA sections: slot s of chunk k (rank = k mod
// ncta, local chunk q = k / ncta) goes to local slot q C + r; its entries to loc[k] + w C + r.
template <class MT, class DT>
__global__ void k_pack(const int* perm, const int* cptr, const int* col, const MT* val, const DT* diag, int nslots, int C,
                       int ncta, const int* loc, unsigned char* img, const unsigned* img_off, const unsigned* sec,
                       int s_perm, int s_col, int s_diag, int s_val) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int k = s / C, r = s % C, rank = k % ncta, q = k / ncta;
    unsigned char* base = img + img_off[rank];
    const unsigned* o = sec + rank * NSEC;
    reinterpret_cast<int*>(base + o[s_perm])[q * C + r] = perm[s];
    if (diag) reinterpret_cast<DT*>(base + o[s_diag])[q * C + r] = diag[s];
    const int w = (cptr[k + 1] - cptr[k]) / C;
    for (int e = 0; e < w; ++e) {
        reinterpret_cast<int*>(base + o[s_col])[loc[k] + e * C + r] = col[cptr[k] + e * C + r];
        reinterpret_cast<MT*>(base + o[s_val])[loc[k] + e * C + r] = val[cptr[k] + e * C + r];
    }
}

struct OpLayout {                   // one SELL operator cut into per-CTA pieces
    std::vector<int> loc;           // element offset of chunk k inside its CTA's piece
    std::vector<std::vector<int>> cptr_loc;   // per CTA: local row offsets [nown + 1]
    std::vector<int> elems;         // per CTA: entries
    std::vector<int> nown;          // per CTA: chunks
};

OpLayout cut(const Sell& S, int ncta) {
    std::vector<int> cptr(S.nchunks + 1);
    CPC_CK(cudaMemcpy(cptr.data(), S.cptr.p, sizeof(int) * (S.nchunks + 1), cudaMemcpyDeviceToHost));
    OpLayout o;
    o.loc.resize(S.nchunks);
    o.cptr_loc.assign(ncta, std::vector<int>(1, 0));
    o.elems.assign(ncta, 0);
    o.nown.assign(ncta, 0);
    for (int k = 0; k < S.nchunks; ++k) {
        const int r = k % ncta;
        o.loc[k] = o.elems[r];
        o.elems[r] += cptr[k + 1] - cptr[k];
        o.cptr_loc[r].push_back(o.elems[r]);
        o.nown[r]++;
    }
    return o;
}

template <class MT, class DT, class PT, class VT>
void build_tail_images(Handle& h, int t0, int ncta, TDesc& d, bool dry, size_t* max_img) {
    const int nl = (int)h.lev.size();
    d = TDesc{};
    d.nl = nl - t0;
    d.nc = h.nc;
    d.ncta = ncta;
    d.lg = 0;
    while ((1 << d.lg) < ncta) ++d.lg;
    // vector region
    unsigned vb = 0;
    for (int t = 0; t < d.nl; ++t) {
        const int cap = (h.lev[t0 + t].n + ncta - 1) / ncta;
        d.lev[t].n = h.lev[t0 + t].n;
        d.lev[t].vx = vb; vb += align16((size_t)cap * sizeof(VT));
        d.lev[t].vf = vb; vb += align16((size_t)cap * sizeof(VT));
        d.lev[t].vr = vb; vb += align16((size_t)cap * sizeof(VT));
    }
    d.vec_bytes = vb;
    // image sections
    std::vector<OpLayout> la(d.nl), lp(d.nl), lr(d.nl);
    std::vector<size_t> off(ncta, 0);
    for (int t = 0; t + 1 < d.nl; ++t) {
        Level& L = h.lev[t0 + t];
        la[t] = cut(L.S, ncta);
        lp[t] = cut(L.SP, ncta);
        lr[t] = cut(L.SR, ncta);
        for (int r = 0; r < ncta; ++r) {
            unsigned* o = d.lev[t].off[r];
            o[A_CPTR] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (la[t].nown[r] + 1));
            o[A_PERM] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (size_t)la[t].nown[r] * L.S.C);
            o[A_COL] = (unsigned)off[r];  off[r] += align16(sizeof(int) * (size_t)la[t].elems[r]);
            o[A_DIAG] = (unsigned)off[r]; off[r] += align16(sizeof(DT) * (size_t)la[t].nown[r] * L.S.C);
            o[A_DINV] = (unsigned)off[r]; off[r] += align16(sizeof(DT) * (size_t)la[t].nown[r] * L.S.C);
            o[A_VAL] = (unsigned)off[r];  off[r] += align16(sizeof(MT) * (size_t)la[t].elems[r]);
            o[P_CPTR] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (lp[t].nown[r] + 1));
            o[P_PERM] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (size_t)lp[t].nown[r] * L.SP.C);
            o[P_COL] = (unsigned)off[r];  off[r] += align16(sizeof(int) * (size_t)lp[t].elems[r]);
            o[P_VAL] = (unsigned)off[r];  off[r] += align16(sizeof(PT) * (size_t)lp[t].elems[r]);
            o[R_CPTR] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (lr[t].nown[r] + 1));
            o[R_PERM] = (unsigned)off[r]; off[r] += align16(sizeof(int) * (size_t)lr[t].nown[r] * L.SR.C);
            o[R_COL] = (unsigned)off[r];  off[r] += align16(sizeof(int) * (size_t)lr[t].elems[r]);
            o[R_VAL] = (unsigned)off[r];  off[r] += align16(sizeof(PT) * (size_t)lr[t].elems[r]);
        }
    }
    const int nc = h.nc;
    for (int r = 0; r < ncta; ++r) {
        d.ainv_off[r] = (unsigned)off[r];
        const int rows = nc > r ? (nc - r + ncta - 1) / ncta : 0;
        off[r] += align16(sizeof(VT) * (size_t)rows * nc);
    }
    size_t total = 0, mx = 0;
    for (int r = 0; r < ncta; ++r) {
        d.img_off[r] = (unsigned)total;
        d.img_bytes[r] = align16(off[r]);
        total += d.img_bytes[r];
        mx = std::max(mx, (size_t)d.img_bytes[r]);
    }
    *max_img = mx;
    if (dry) return;
    // fill
    h.tail_img.alloc(std::max<size_t>(total, 16));
    CPC_CK(cudaMemset(h.tail_img.p, 0, std::max<size_t>(total, 16)));
    d.img = (const unsigned char*)h.tail_img.p;
    DBuf<unsigned> doff, dsec;
    doff.alloc(ncta);
    CPC_CK(cudaMemcpy(doff.p, d.img_off, sizeof(unsigned) * ncta, cudaMemcpyHostToDevice));
    const bool f64 = std::is_same<VT, double>::value;
    for (int t = 0; t + 1 < d.nl; ++t) {
        Level& L = h.lev[t0 + t];
        std::vector<unsigned> sec((size_t)ncta * NSEC);
        for (int r = 0; r < ncta; ++r)
            for (int q = 0; q < NSEC; ++q) sec[(size_t)r * NSEC + q] = d.lev[t].off[r][q];
        dsec.alloc(sec.size());
        CPC_CK(cudaMemcpy(dsec.p, sec.data(), sizeof(unsigned) * sec.size(), cudaMemcpyHostToDevice));
        for (int r = 0; r < ncta; ++r) {
            CPC_CK(cudaMemcpy(h.tail_img.p + d.img_off[r] + d.lev[t].off[r][A_CPTR], la[t].cptr_loc[r].data(),
                              sizeof(int) * la[t].cptr_loc[r].size(), cudaMemcpyHostToDevice));
            CPC_CK(cudaMemcpy(h.tail_img.p + d.img_off[r] + d.lev[t].off[r][P_CPTR], lp[t].cptr_loc[r].data(),
                              sizeof(int) * lp[t].cptr_loc[r].size(), cudaMemcpyHostToDevice));
            CPC_CK(cudaMemcpy(h.tail_img.p + d.img_off[r] + d.lev[t].off[r][R_CPTR], lr[t].cptr_loc[r].data(),
                              sizeof(int) * lr[t].cptr_loc[r].size(), cudaMemcpyHostToDevice));
        }
        DBuf<int> loc;
        auto pack = [&](const Sell& S, const OpLayout& lo, const auto* val, const auto* diag, int sp, int sc, int sd,
                        int sv) {
            loc.alloc(lo.loc.size());
            CPC_CK(cudaMemcpy(loc.p, lo.loc.data(), sizeof(int) * lo.loc.size(), cudaMemcpyHostToDevice));
            using V = std::remove_cv_t<std::remove_pointer_t<decltype(val)>>;
            using Dg = std::remove_cv_t<std::remove_pointer_t<decltype(diag)>>;
            k_pack<V, Dg><<<(S.nslots + 255) / 256, 256>>>(S.perm.p, S.cptr.p, S.col.p, val, diag, S.nslots, S.C, ncta,
                                                          loc.p, (unsigned char*)h.tail_img.p, doff.p, dsec.p, sp, sc,
                                                          sd, sv);
            CPC_LAUNCH_CK();
            CPC_CK(cudaDeviceSynchronize());
        };
        const MT* aval = f64 ? (const MT*)L.S.val.p
                             : (L.vt == VT_BF16 ? (const MT*)L.S.val16.p : (const MT*)L.S.val32.p);
        const DT* adiag = f64 ? (const DT*)L.S.diag.p : (const DT*)L.S.diag32.p;
        const DT* adinv = f64 ? (const DT*)L.S.dinv.p : (const DT*)L.S.dinv32.p;
        pack(L.S, la[t], aval, adiag, A_PERM, A_COL, A_DIAG, A_VAL);
        pack(L.S, la[t], aval, adinv, A_PERM, A_COL, A_DINV, A_VAL);
        const PT* pval = f64 ? (const PT*)L.SP.val.p : (const PT*)L.SP.val32.p;
        pack(L.SP, lp[t], pval, (const PT*)nullptr, P_PERM, P_COL, 0, P_VAL);
        const PT* rval = f64 ? (const PT*)L.SR.val.p : (const PT*)L.SR.val32.p;
        pack(L.SR, lr[t], rval, (const PT*)nullptr, R_PERM, R_COL, 0, R_VAL);
        d.lev[t].ncol = L.ncolours;
        d.lev[t].C = L.S.C;
        d.lev[t].nck = L.S.nchunks;
        d.lev[t].CP = L.SP.C;
        d.lev[t].nckP = L.SP.nchunks;
        d.lev[t].CR = L.SR.C;
        d.lev[t].nckR = L.SR.nchunks;
        h.tail_seg[t].alloc(L.S.seg.size());
        CPC_CK(cudaMemcpy(h.tail_seg[t].p, L.S.seg.data(), sizeof(int) * L.S.seg.size(), cudaMemcpyHostToDevice));
        d.lev[t].seg = h.tail_seg[t].p;
    }
    // coarsest: rows q ncta + r of A_c^{-1}
    const VT* ainv = f64 ? (const VT*)h.Ainv.p : (const VT*)h.Ainv32.p;
    for (int r = 0; r < ncta; ++r)
        for (int i = r, q = 0; i < nc; i += ncta, ++q)
            CPC_CK(cudaMemcpy(h.tail_img.p + d.img_off[r] + d.ainv_off[r] + sizeof(VT) * (size_t)q * nc,
                              ainv + (size_t)i * nc, sizeof(VT) * nc, cudaMemcpyDeviceToDevice));
}

template <class MT, class DT, class PT, class VT>
void launch_tail(const Handle& h, int start, const VT* f0, VT* x0, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h.tail_cluster, 1, 1);
    cfg.blockDim = dim3(TAIL_TPB, 1, 1);
    cfg.dynamicSmemBytes = h.tail_smem;
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
    CPC_CK(cudaLaunchKernelEx(&cfg, k_tail<MT, DT, PT, VT>, (const TDesc*)h.tail_desc.p, start, f0, x0));
}

// Largest cluster (<= 16 CTAs, one per SM) that the device can schedule with this shared memory.
template <class MT, class DT, class PT, class VT>
int pick_cluster(size_t smem) {
    auto k = k_tail<MT, DT, PT, VT>;
    CPC_CK(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    CPC_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TAIL_SMEM));
    for (int cs : {16, 8, 4, 2, 1}) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(TAIL_TPB, 1, 1);
        cfg.dynamicSmemBytes = smem;
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
    return 0;
}

template <class MT, class DT, class PT, class VT>
void setup_tail_t(Handle& h, int64_t tail_nnz_max) {
    const int nl = (int)h.lev.size();
    // cluster size from the full budget, then the deepest-reaching start level whose images fit
    const int ncta = pick_cluster<MT, DT, PT, VT>(TAIL_SMEM);
    if (ncta < 1) return;
    int best = nl;
    TDesc d{};
    for (int t0 = nl - 1; t0 >= 1; --t0) {
        if (nl - t0 > TAIL_MAXL) break;
        if (t0 < nl - 1 && h.lev[t0].A.nnz > tail_nnz_max) break;
        size_t mx = 0;
        build_tail_images<MT, DT, PT, VT>(h, t0, ncta, d, true, &mx);
        if (mx + d.vec_bytes > TAIL_SMEM) break;
        best = t0;
    }
    if (best >= nl) return;
    h.tail_seg.clear();
    h.tail_seg.resize(nl - best);
    size_t mx = 0;
    build_tail_images<MT, DT, PT, VT>(h, best, ncta, d, false, &mx);
    h.tail_smem = mx + d.vec_bytes;
    h.tail_cluster = ncta;
    h.tail_start = best;
    h.tail_desc.alloc(sizeof(TDesc));
    CPC_CK(cudaMemcpy(h.tail_desc.p, &d, sizeof(TDesc), cudaMemcpyHostToDevice));
}

}  // namespace

void setup_tail(Handle& h, int64_t tail_nnz_max) {
    const int nl = (int)h.lev.size();
    h.tail_start = nl;                     // no tail: every level by separate launches
    if (nl < 2 || tail_nnz_max <= 0) return;
    if (h.opt.precision == CPC_PREC_FP64) setup_tail_t<double, double, double, double>(h, tail_nnz_max);
    else if (h.opt.precision == CPC_PREC_FP32_BF16) setup_tail_t<__nv_bfloat16, float, float, float>(h, tail_nnz_max);
    else setup_tail_t<float, float, float, float>(h, tail_nnz_max);
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
