// check.cu -- structural checks of a handle's device layouts, a stand-in for a memory and race
// sanitizer.  Every index a solve kernel gathers through comes from a layout built at setup, and
// every parallel step relies on a property of one, so checking the layouts checks the kernels'
// accesses and their independence:
//   [0] out of range: a slot's row, a chunk pointer or a column index outside its layout, a
//       diagonal offset of at least n, a group boundary outside the chunk range;
//   [1] coverage: a row missing from or repeated in a layout (every layout holds each of its rows
//       exactly once);
//   [2] Gauss-Seidel races: two rows coupled in A_l (a_ij != 0, i != j) in one colour group of the
//       smoother layout, whose rows one launch updates in parallel (Section 3.3);
//   [3] triangular-solve races: an entry of the IC(0) factor whose row's level is not after its
//       column's (forward levels for j < i, backward levels for j > i; Algorithm 3.1).
// Every index is bounds-checked here before it is used.
#include <vector>

#include "handle.cuh"

namespace cpc {

namespace {

constexpr int CTPB = 256;
enum { C_RANGE = 0, C_COVER, C_GS_RACE, C_TRI_RACE, C_LAYOUTS, C_COUNT };

inline int cblk(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + CTPB - 1) / CTPB, 152 * 64)); }

// Group of chunk k: the g with seg[g] <= k < seg[g + 1] (seg ascending), or -1.
__device__ int group_of(const int* seg, int ng, int k) {
    if (ng < 1 || k < seg[0] || k >= seg[ng]) return -1;
    int lo = 0, hi = ng;                       // seg[lo] <= k < seg[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (seg[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Slots: row in range (or -1 padding), counted in seen; grp[row] = the slot's group when grp.
__global__ void k_chk_slots(int nslots, int C, int nrows, const int* perm, const int* seg, int ng, int* seen,
                            int* grp, unsigned long long* cnt) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
        const int p = perm ? perm[s] : (s < nrows ? s : -1);
        if (p < -1 || p >= nrows) { atomicAdd(&cnt[C_RANGE], 1ull); continue; }
        if (p < 0) continue;
        atomicAdd(&seen[p], 1);
        if (grp) {
            const int g = group_of(seg, ng, s / C);
            if (g < 0) atomicAdd(&cnt[C_RANGE], 1ull);
            else grp[p] = g;
        }
    }
}

// Chunk pointers ascending within [0, nelem] with widths a multiple of C; columns in [-1, ncols).
__global__ void k_chk_entries(int nchunks, int C, int64_t nelem, int ncols, const int* cptr, const int* col,
                              unsigned long long* cnt) {
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = t0; k < nchunks; k += st) {
        const int a = cptr[k], b = cptr[k + 1];
        if (a < 0 || a > b || b > nelem || (b - a) % C != 0) atomicAdd(&cnt[C_RANGE], 1ull);
    }
    if (col)
        for (int64_t e = t0; e < nelem; e += st) {
            const int c = col[e];
            if (c < -1 || c >= ncols) atomicAdd(&cnt[C_RANGE], 1ull);
        }
}

__global__ void k_chk_seen(int n, const int* seen, int exact, unsigned long long* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (exact ? seen[i] != 1 : seen[i] > 1) atomicAdd(&cnt[C_COVER], 1ull);
}

// tri = 0: coupled rows i != j of one group gl.  tri = 1 (the factor, on the pattern of the matrix
// in IC order, whose row q is row imap[q] of the layouts): an entry whose row is not in a later
// group than its column, in the forward groups gl for q' < q and the backward groups gu for q' > q.
__global__ void k_chk_pairs(int n, const int* ptr, const int* col, const int* gl, const int* gu, int tri,
                            const int* imap, unsigned long long* cnt) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = imap ? imap[q] : q;
        if (i < 0 || i >= n) { atomicAdd(&cnt[C_RANGE], 1ull); continue; }
        for (int e = ptr[q]; e < ptr[q + 1]; ++e) {
            const int qc = col[e];
            if (qc < 0 || qc >= n) { atomicAdd(&cnt[C_RANGE], 1ull); continue; }
            if (qc == q) continue;
            const int j = imap ? imap[qc] : qc;
            if (j < 0 || j >= n) { atomicAdd(&cnt[C_RANGE], 1ull); continue; }
            if (!tri) {
                if (gl[i] >= 0 && gl[i] == gl[j]) atomicAdd(&cnt[C_GS_RACE], 1ull);
            } else {
                const int* g = qc < q ? gl : gu;
                if (g[i] < 0 || g[j] < 0 || g[j] >= g[i]) atomicAdd(&cnt[C_TRI_RACE], 1ull);
            }
        }
    }
}

struct Checker {
    Handle& h;
    cudaStream_t s;
    DBuf<unsigned long long> cnt;
    explicit Checker(Handle& hh) : h(hh), s(hh.s) {
        cnt.alloc(C_COUNT);
        CPC_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * C_COUNT, s));
    }
    // One SELL layout with nrows rows and ncols columns; grp (n-vector) receives each row's group.
    void sell(const Sell& S, int nrows, int ncols, bool exact, int* grp = nullptr) {
        if (S.nslots == 0 && S.nchunks == 0) return;
        Tmp<int> seen(nrows, s), dseg(std::max<size_t>(1, S.seg.size()), s);
        CPC_CK(cudaMemsetAsync(seen.get(), 0, sizeof(int) * nrows, s));
        int ng = 0;
        if (grp) {
            std::vector<int> seg = S.seg;
            ng = (int)seg.size() - 1;
            bool ok = ng >= 1 && seg.front() == 0 && seg.back() == S.nchunks;
            for (int g = 0; g + 1 < (int)seg.size(); ++g) ok = ok && seg[g] <= seg[g + 1];
            if (!ok) bump(C_RANGE);
            CPC_CK(cudaMemcpyAsync(dseg.get(), seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice, s));
            CPC_CK(cudaMemsetAsync(grp, 0xff, sizeof(int) * nrows, s));
            CPC_CK(cudaStreamSynchronize(s));             // seg goes out of scope
        }
        k_chk_slots<<<cblk(S.nslots), CTPB, 0, s>>>(S.nslots, S.C, nrows, S.perm.p, dseg.get(), ng, seen.get(), grp, cnt.p);
        if (S.cptr.p)
            k_chk_entries<<<cblk(std::max<int64_t>(S.nchunks, S.nelem)), CTPB, 0, s>>>(S.nchunks, S.C, S.nelem, ncols,
                                                                                     S.cptr.p, S.col.p, cnt.p);
        k_chk_seen<<<cblk(nrows), CTPB, 0, s>>>(nrows, seen.get(), exact ? 1 : 0, cnt.p);
        for (int d = 0; d < S.ndiag; ++d)
            if (S.doff.o[d] <= -nrows || S.doff.o[d] >= nrows) bump(C_RANGE);
        CPC_LAUNCH_CK();
        CPC_CK(cudaStreamSynchronize(s));
        bump(C_LAYOUTS);
    }
    void bump(int k) {
        unsigned long long v = 0;
        CPC_CK(cudaMemcpyAsync(&v, cnt.p + k, sizeof(v), cudaMemcpyDeviceToHost, s));
        CPC_CK(cudaStreamSynchronize(s));
        ++v;
        CPC_CK(cudaMemcpyAsync(cnt.p + k, &v, sizeof(v), cudaMemcpyHostToDevice, s));
        CPC_CK(cudaStreamSynchronize(s));
    }
};

}  // namespace

void check_layouts(Handle& h, int64_t* counts) {
    Checker ck(h);
    cudaStream_t s = h.s;
    CPC_CK(cudaStreamSynchronize(s));
    const int nl = (int)h.lev.size();
    for (int l = 0; l + 1 < nl; ++l) {
        Level& L = h.lev[l];
        const int nc = h.lev[l + 1].n;
        Tmp<int> grp(L.n, s);
        ck.sell(L.S, L.n, L.n, true, grp.get());
        k_chk_pairs<<<cblk(L.n), CTPB, 0, s>>>(L.n, L.A.ptr.p, L.A.col.p, grp.get(), grp.get(), 0, nullptr, ck.cnt.p);
        CPC_LAUNCH_CK();
        CPC_CK(cudaStreamSynchronize(s));
        ck.sell(L.SP, L.n, nc, true);
        ck.sell(L.SR, nc, L.n, true);
    }
    ck.sell(h.Anat, h.n, h.n, true);
    if (h.Aic.n == h.n && h.L.nslots > 0) {
        Tmp<int> gl(h.n, s), gu(h.n, s);
        ck.sell(h.L, h.n, h.n, true, gl.get());
        ck.sell(h.U, h.n, h.n, true, gu.get());
        k_chk_pairs<<<cblk(h.n), CTPB, 0, s>>>(h.n, h.Aic.ptr.p, h.Aic.col.p, gl.get(), gu.get(), 1, h.ic_order.p,
                                               ck.cnt.p);
        CPC_LAUNCH_CK();
    }
    unsigned long long c[C_COUNT];
    CPC_CK(cudaMemcpyAsync(c, ck.cnt.p, sizeof(c), cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    for (int k = 0; k < C_COUNT; ++k) counts[k] = (int64_t)c[k];
}

}  // namespace cpc
