// setup.cu -- GPU setup: TPFA assembly, IC(0) factorisation, AMG hierarchy, SELL-C layouts.
//
// Everything here runs on the device; the host only sequences launches and reads back a few
// counters (round loops of PMIS, colouring and level scheduling).  The rules are those of
// Section 3 of the paper with the readings listed in the library docs:
//   IC(0)   Algorithm 3.1 with k = 0 in IKJ form, rows factored level by level of the lower DAG;
//   AMG     strength theta, PMIS splitting with weight (|S^T_i|, fmix32(i)), direct
//           interpolation, R = P^T, Galerkin A_c = R (A P) (Section 3.2);
//   colour  breadth-first parity 2-colouring when the level graph is bipartite (red-black on a
//           structured grid), else Jones-Plassmann with priority (peel round, fmix32(i ^
//           0x5bd1e995)) and the smallest free colour; peel rounds are a smallest-last style
//           ordering that needs fewer colours than a random one; with natural-order
//           Gauss-Seidel, the wavefronts of the lower-triangular graph of A_l instead.
// Sums that define matrix entries are accumulated in a fixed order (the order the products are
// generated in), so results do not depend on thread scheduling.
#include <cub/cub.cuh>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>

#include "handle.cuh"
#include "tpfa_cell.cuh"

namespace cpc {

namespace {

constexpr uint32_t COLOUR_SEED = 0x5bd1e995u;
constexpr int TPB = 256;

// Published MurmurHash3 32-bit finaliser (a bijection): tie-break weights.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
    return h;
}

inline int nblk(int64_t n, int t = TPB) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

template <class T>
T d2h(const T* p, cudaStream_t s) {
    T v;
    CPC_CK(cudaMemcpyAsync(&v, p, sizeof(T), cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    return v;
}

template <class T>
void h2d(T* dst, const T* src, size_t n, cudaStream_t s) {
    CPC_CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
}

// out[0..n) = exclusive prefix sum of in[0..n)
template <class T>
void exclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s) {
    size_t tmp = 0;
    CPC_CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
    Tmp<char> t(tmp, s);
    CPC_CK(cub::DeviceScan::ExclusiveSum(t.get(), tmp, in, out, n, s));
}

template <class T>
void inclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s) {
    size_t tmp = 0;
    CPC_CK(cub::DeviceScan::InclusiveSum(nullptr, tmp, in, out, n, s));
    Tmp<char> t(tmp, s);
    CPC_CK(cub::DeviceScan::InclusiveSum(t.get(), tmp, in, out, n, s));
}

// Stable radix sort of (key, value) pairs over the low `bits` bits of the key.
template <class K, class V>
void sort_pairs(const K* kin, K* kout, const V* vin, V* vout, int64_t n, int bits, cudaStream_t s) {
    size_t tmp = 0;
    CPC_CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp, kin, kout, vin, vout, n, 0, bits, s));
    Tmp<char> t(tmp, s);
    CPC_CK(cub::DeviceRadixSort::SortPairs(t.get(), tmp, kin, kout, vin, vout, n, 0, bits, s));
}

int bits_for(uint64_t maxval) {
    int b = 1;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

__global__ void k_iota(int* a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

__global__ void k_fill_int(int* a, int64_t n, int v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// ============================================================================================
// a0: two-point-flux assembly (Section 4, Eq. model with c = 0), unit cells; the row of a cell
// (entry order, harmonic means, Dirichlet terms) is tpfa_fill_row in tpfa_cell.cuh.
// ============================================================================================
__global__ void k_tpfa_rowlen(int nx, int ny, int nz, int* len) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int n = nx * ny * nz;
    if (c >= n) return;
    len[c] = tpfa_row_len(c, nx, ny, nz);
}

__global__ void k_tpfa_fill(int nx, int ny, int nz, const double* logk, double kzr, int dmask,
                            const int* rowptr, int* col, double* val) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int n = nx * ny * nz;
    if (c >= n) return;
    tpfa_fill_row(c, nx, ny, nz, logk, kzr, dmask, rowptr[c], col, val);
}

// ============================================================================================
// CSR validation and helpers
// ============================================================================================
// flags: [0] bad row pointer, [1] bad column / order, [2] missing diagonal
__global__ void k_validate(int n, const int* ptr, const int* col, int nnz, int* bad, int* diag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = ptr[i], b = ptr[i + 1];
    if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) {
        atomicOr(bad, 1);
        diag[i] = -1;
        return;
    }
    int d = -1;
    for (int p = a; p < b; ++p) {
        int j = col[p];
        if (j < 0 || j >= n || (p > a && j <= col[p - 1])) { atomicOr(bad, 2); diag[i] = -1; return; }
        if (j == i) d = p;
    }
    if (d < 0) atomicOr(bad, 4);
    diag[i] = d;
}

// Row index of every entry.
__global__ void k_entry_rows(int n, const int* ptr, int* rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) rows[p] = i;
}

// tpos[p] = position of (j, i) for entry p = (i, j); flags structural asymmetry.
__global__ void k_transpose_pos(int n, const int* ptr, const int* col, int* tpos, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        int j = col[p];
        int lo = ptr[j], hi = ptr[j + 1] - 1, found = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int c = col[mid];
            if (c == i) { found = mid; break; }
            if (c < i) lo = mid + 1; else hi = mid - 1;
        }
        tpos[p] = found;
        if (found < 0) atomicOr(bad, 8);
    }
}

// ============================================================================================
// Transpose and sparse products (ESC: expand, stable sort, sum each key in generation order)
// ============================================================================================
__global__ void k_col_count(int64_t nnz, const int* col, int* cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_gather_transpose(int64_t nnz, const int* idx, const int* rows, const double* val,
                                   int* tcol, double* tval) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    int p = idx[k];
    tcol[k] = rows[p];
    tval[k] = val[p];
}

void transpose(const Csr& A, Csr& T, cudaStream_t s) {
    T.n = A.m; T.m = A.n; T.nnz = A.nnz;
    T.ptr.alloc(T.n + 1);
    T.col.alloc(A.nnz);
    T.val.alloc(A.nnz);
    Tmp<int> rows(A.nnz, s), idx(A.nnz, s), sk(A.nnz, s), sv(A.nnz, s), cnt(T.n + 1, s);
    k_entry_rows<<<nblk(A.n), TPB, 0, s>>>(A.n, A.ptr.p, rows.get());
    k_iota<<<nblk(A.nnz), TPB, 0, s>>>(idx.get(), (int)A.nnz);
    sort_pairs(A.col.p, sk.get(), idx.get(), sv.get(), A.nnz, bits_for((uint64_t)std::max(1, A.m)), s);
    CPC_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int) * (T.n + 1), s));
    k_col_count<<<nblk(A.nnz), TPB, 0, s>>>(A.nnz, A.col.p, cnt.get());
    exclusive_scan(cnt.get(), T.ptr.p, T.n + 1, s);
    k_gather_transpose<<<nblk(A.nnz), TPB, 0, s>>>(A.nnz, sv.get(), rows.get(), A.val.p, T.col.p, T.val.p);
    CPC_LAUNCH_CK();
}

__global__ void k_prod_count(int n, const int* aptr, const int* acol, const int* bptr, int64_t* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) { cnt[n] = 0; return; }
    int64_t c = 0;
    for (int p = aptr[i]; p < aptr[i + 1]; ++p) { int k = acol[p]; c += bptr[k + 1] - bptr[k]; }
    cnt[i] = c;
}

__global__ void k_prod_expand(int n, const int* aptr, const int* acol, const double* aval,
                              const int* bptr, const int* bcol, const double* bval, int64_t m,
                              const int64_t* off, uint64_t* key, double* val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = off[i];
    for (int p = aptr[i]; p < aptr[i + 1]; ++p) {
        const int k = acol[p];
        const double a = aval[p];
        for (int q = bptr[k]; q < bptr[k + 1]; ++q) {
            key[o] = (uint64_t)i * (uint64_t)m + (uint64_t)bcol[q];
            val[o] = a * bval[q];
            ++o;
        }
    }
}

__global__ void k_seg_head(int64_t N, const uint64_t* key, int* head) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) head[t] = (t == 0 || key[t] != key[t - 1]) ? 1 : 0;
}

__global__ void k_seg_start(int64_t N, const int* head, const int* segid, int64_t* start) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N && head[t]) start[segid[t] - 1] = t;
}

__global__ void k_seg_sum(int nseg, int64_t N, const int64_t* start, const uint64_t* key, const double* val,
                          int64_t m, int* ccol, double* cval, int* rowcnt) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg) return;
    const int64_t a = start[g];
    const int64_t b = (g + 1 < nseg) ? start[g + 1] : N;
    double s = val[a];
    for (int64_t t = a + 1; t < b; ++t) s += val[t];
    const uint64_t kk = key[a];
    ccol[g] = (int)(kk % (uint64_t)m);
    cval[g] = s;
    atomicAdd(&rowcnt[(int)(kk / (uint64_t)m)], 1);
}

__global__ void k_max_int(const int* a, int n, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, a[i]);
}

__global__ void k_max_i64(const int64_t* a, int n, int64_t* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax((unsigned long long*)out, (unsigned long long)a[i]);
}

// ---------------------------------------------------------------------------------------------
// Hash sparse product C = A B, one warp per row i of C.  The row's entries live in a hash table in
// shared memory (open addressing, linear probing).  Row i of A is taken in order of its entries
// (ascending k); for each k the products a_ik b_kj of row k of B enter the table together, one per
// lane: the j of one row of B are distinct, so no two lanes touch one entry in the same step, and
// entry (i, j) receives its products in ascending k, each product rounded and then added: the
// sums of the sort-based product below, bit for bit.  Before the steps, the products of the rows
// of B for up to HS_STAGE of them are formed and staged in shared memory, all loads in flight.  A symbolic pass
// counts each row's entries; the numeric pass compacts the table, sorts it by column (bitonic, in
// registers) and writes the row.  A row with more than half a table of entries, or a row of B
// longer than the stage, is not taken: the caller falls back to the sort-based product.
// ---------------------------------------------------------------------------------------------
constexpr int HS_WARPS = 4;                 // warps per CTA
constexpr int HS_STAGE = 512;               // staged products per warp
constexpr int HS_SYM = 1024;                // table slots per warp in the symbolic pass
constexpr int HS_SORT = 128;                // most entries of a row sorted in registers
constexpr unsigned FULLW = 0xffffffffu;

__device__ __forceinline__ int hs_slot(int j, int lg) { return (int)(((uint32_t)j * 0x9E3779B1u) >> (32 - lg)); }

// Per-warp shared memory: staged columns / values, the table, the group's entries of A.
struct HsEntry {
    int k, b0, len, off;
    double a;
};

// Row i: the steps k of row i of A in order; insert(j, prod) is called by the lanes of a step.
// Returns false (warp-uniform) if a row of B is longer than the stage.
template <bool NUMERIC, class Ins>
__device__ bool hs_row(int i, const int* aptr, const int* acol, const double* aval, const int* bptr, const int* bcol,
                       const double* bval, int* sc, double* sv, HsEntry* ent, int lane, Ins&& insert) {
    const int p0 = aptr[i], p1 = aptr[i + 1];
    for (int c0 = p0; c0 < p1; c0 += 32) {
        const int cn = min(32, p1 - c0);
        int k = -1, b0 = 0, len = 0;
        double a = 0.0;
        if (lane < cn) {
            k = acol[c0 + lane];
            if (NUMERIC) a = aval[c0 + lane];
        }
        if (lane < cn) {
            b0 = bptr[k];
            len = bptr[k + 1] - b0;
        }
        if (__any_sync(FULLW, len > HS_STAGE)) return false;
        for (int e0 = 0; e0 < cn;) {
            // entries [e0, e1) whose products fit the stage
            const int my = lane >= e0 && lane < cn ? len : 0;
            int inc = my;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULLW, inc, o);
                if (lane >= o) inc += t;
            }
            const unsigned fm = __ballot_sync(FULLW, lane >= e0 && lane < cn && inc <= HS_STAGE);
            const int e1 = 32 - __clz(fm);                      // one past the last entry that fits
            const int tot = __shfl_sync(FULLW, inc, e1 - 1);
            __syncwarp();
            if (lane >= e0 && lane < e1) ent[lane] = HsEntry{k, b0, len, inc - my, a};
            __syncwarp();
            // stage: flattened product f of the group -> its entry by binary search on the offsets
            for (int f0 = 0; f0 < tot; f0 += 8 * 32) {
                int cj[8];
                double cv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int f = f0 + u * 32 + lane;
                    cj[u] = -1;
                    cv[u] = 0.0;
                    if (f < tot) {
                        int lo = e0, hi = e1 - 1;                   // last entry with off <= f
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (ent[mid].off <= f) lo = mid; else hi = mid - 1;
                        }
                        const int q = ent[lo].b0 + (f - ent[lo].off);
                        cj[u] = bcol[q];
                        if (NUMERIC) cv[u] = __dmul_rn(ent[lo].a, bval[q]);      // the product, rounded
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int f = f0 + u * 32 + lane;
                    if (f < tot) {
                        sc[f] = cj[u];
                        if (NUMERIC) sv[f] = cv[u];
                    }
                }
            }
            __syncwarp();
            for (int e = e0; e < e1; ++e) {                     // steps in ascending k
                const HsEntry en = ent[e];
                for (int q = lane; q < en.len; q += 32) insert(sc[en.off + q], NUMERIC ? sv[en.off + q] : 0.0);
                __syncwarp();
            }
            e0 = e1;
        }
    }
    return true;
}

// Claims or finds j's slot; returns the slot, or -1 if the table is full.  *fresh: claimed now.
__device__ __forceinline__ int hs_find(int* key, int lg, int j, bool* fresh) {
    const int ts = 1 << lg;
    int sl = hs_slot(j, lg);
    for (int t = 0; t < ts; ++t) {
        const int cur = key[sl];
        if (cur == j) { *fresh = false; return sl; }
        if (cur == -1) {
            const int prev = atomicCAS(&key[sl], -1, j);
            if (prev == -1) { *fresh = true; return sl; }
            if (prev == j) { *fresh = false; return sl; }
        }
        sl = (sl + 1) & (ts - 1);
    }
    return -1;
}

// Sorts the cnt (<= 32 E) entries sk[], svv[] of a row by column, bitonic over 32 E elements held
// E per lane (element g = e * 32 + lane), and writes them to col[], val[].
template <int E>
__device__ void hs_sort_write(const int* sk, const double* svv, int cnt, int lane, int* col, double* val) {
    constexpr int M = 32 * E;
    int kr[E];
    double vr[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = e * 32 + lane;
        kr[e] = g < cnt ? sk[g] : INT_MAX;
        vr[e] = g < cnt ? svv[g] : 0.0;
    }
#pragma unroll
    for (int kk = 2; kk <= M; kk <<= 1) {
#pragma unroll
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            if (jj >= 32) {
                const int de = jj >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int e2 = e ^ de;
                    if (e2 > e) {
                        const bool asc = ((e * 32 + lane) & kk) == 0;
                        if ((kr[e] > kr[e2]) == asc) {
                            const int tk = kr[e]; kr[e] = kr[e2]; kr[e2] = tk;
                            const double tv = vr[e]; vr[e] = vr[e2]; vr[e2] = tv;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int g = e * 32 + lane;
                    const int ok2 = __shfl_xor_sync(FULLW, kr[e], jj);
                    const double ov = __shfl_xor_sync(FULLW, vr[e], jj);
                    const bool asc = (g & kk) == 0;
                    const bool lower = (g & jj) == 0;               // g < partner
                    if (lower == asc ? ok2 < kr[e] : ok2 > kr[e]) {
                        kr[e] = ok2;
                        vr[e] = ov;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = e * 32 + lane;
        if (g < cnt) {
            col[g] = kr[e];
            val[g] = vr[e];
        }
    }
}

// Symbolic pass: cnt[i] = entries of row i of C; *over = 1 if a row cannot be taken.
__global__ void __launch_bounds__(HS_WARPS * 32) k_hs_count(int n, const int* aptr, const int* acol, const int* bptr,
                                                             const int* bcol, int* cnt, int* over) {
    __shared__ int s_key[HS_WARPS][HS_SYM];
    __shared__ int s_col[HS_WARPS][HS_STAGE];
    __shared__ HsEntry s_ent[HS_WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* key = s_key[w];
    constexpr int LG = 10;
    static_assert((1 << LG) == HS_SYM, "table size");
    for (int t = lane; t < HS_SYM; t += 32) key[t] = -1;
    __syncwarp();
    for (int i = blockIdx.x * HS_WARPS + w; i < n; i += gridDim.x * HS_WARPS) {
        int claimed = 0;
        bool full = false;
        const bool ok = hs_row<false>(i, aptr, acol, nullptr, bptr, bcol, nullptr, s_col[w], nullptr, s_ent[w], lane,
                                      [&](int j, double) {
                                          bool fresh;
                                          if (hs_find(key, LG, j, &fresh) < 0) full = true;
                                          else if (fresh) ++claimed;
                                      });
        for (int o = 16; o > 0; o >>= 1) claimed += __shfl_xor_sync(FULLW, claimed, o);
        const bool bad = !ok || __any_sync(FULLW, full) || claimed > HS_SYM / 2;
        if (lane == 0) {
            cnt[i] = claimed;
            if (bad) atomicOr(over, 1);
        }
        __syncwarp();
        for (int t = lane; t < HS_SYM; t += 32) key[t] = -1;
        __syncwarp();
    }
}

// Numeric pass: row i of C into col[cptr[i] ..], val[..], sorted by column.  LG: log2 table slots.
template <int LG, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_hs_fill(int n, const int* aptr, const int* acol, const double* aval,
                                                         const int* bptr, const int* bcol, const double* bval,
                                                         const int* cptr, int* ccol, double* cval, int* over) {
    constexpr int TS = 1 << LG;
    __shared__ int s_key[WARPS][TS];
    __shared__ double s_val[WARPS][TS];
    __shared__ int s_col[WARPS][HS_STAGE];
    __shared__ double s_sv[WARPS][HS_STAGE];
    __shared__ HsEntry s_ent[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* key = s_key[w];
    double* val = s_val[w];
    for (int t = lane; t < TS; t += 32) key[t] = -1;
    __syncwarp();
    for (int i = blockIdx.x * WARPS + w; i < n; i += gridDim.x * WARPS) {
        bool full = false;
        const bool ok = hs_row<true>(i, aptr, acol, aval, bptr, bcol, bval, s_col[w], s_sv[w], s_ent[w], lane,
                                     [&](int j, double prod) {
                                         bool fresh;
                                         const int sl = hs_find(key, LG, j, &fresh);
                                         if (sl < 0) full = true;
                                         else val[sl] = fresh ? prod : __dadd_rn(val[sl], prod);
                                     });
        const int c0 = cptr[i], cnt = cptr[i + 1] - c0;
        if (!ok || __any_sync(FULLW, full) || cnt > HS_STAGE) {
            if (lane == 0) atomicOr(over, 1);
        } else {
            // compact the table into the stage (cnt entries), then sort by column
            int* sk = s_col[w];
            double* svv = s_sv[w];
            int base = 0;
            for (int t0 = 0; t0 < TS; t0 += 32) {
                const int kk = key[t0 + lane];
                const unsigned um = __ballot_sync(FULLW, kk != -1);
                if (kk != -1) {
                    const int r = base + __popc(um & ((1u << lane) - 1u));
                    if (r < HS_STAGE) {
                        sk[r] = kk;
                        svv[r] = val[t0 + lane];
                    }
                }
                base += __popc(um);
            }
            __syncwarp();
            if (base != cnt) {
                if (lane == 0) atomicOr(over, 1);
            } else if (cnt <= 32) {
                hs_sort_write<1>(sk, svv, cnt, lane, ccol + c0, cval + c0);
            } else if (cnt <= 64) {
                hs_sort_write<2>(sk, svv, cnt, lane, ccol + c0, cval + c0);
            } else if (cnt <= HS_SORT) {
                hs_sort_write<4>(sk, svv, cnt, lane, ccol + c0, cval + c0);
            } else {
                // long row: rank of each entry among the row's columns (distinct)
                for (int g = lane; g < cnt; g += 32) {
                    const int kg = sk[g];
                    int r = 0;
                    for (int h = 0; h < cnt; ++h) r += sk[h] < kg;
                    ccol[c0 + r] = kg;
                    cval[c0 + r] = svv[g];
                }
            }
        }
        __syncwarp();
        for (int t = lane; t < TS; t += 32) key[t] = -1;
        __syncwarp();
    }
}

// Short rows: one thread per row of C, the row's entries kept sorted by column in the thread's
// slice of shared memory (entry e of thread t at [e][t]: no bank conflicts), at most RP_CAP of
// them.  Products are taken in ascending k and each is rounded, then added to its entry (or starts
// it): the same sums as the other products.  The row goes to tmp at off[i] (its product count is a
// bound on its entries); cnt[i] = its entries; *over = 1 if a row has more than RP_CAP.
constexpr int RP_TPB = 64;
constexpr int RP_CAP = 64;

__global__ void __launch_bounds__(RP_TPB) k_rowprod(int n, const int* aptr, const int* acol, const double* aval,
                                                     const int* bptr, const int* bcol, const double* bval,
                                                     const int64_t* off, int* tcol, double* tval, int* cnt, int* over) {
    __shared__ int sc[RP_CAP][RP_TPB];
    __shared__ double sv[RP_CAP][RP_TPB];
    const int t = threadIdx.x;
    const int i = blockIdx.x * RP_TPB + t;
    if (i >= n) return;
    int m = 0;
    bool full = false;
    for (int p = aptr[i]; p < aptr[i + 1] && !full; ++p) {
        const int k = acol[p];
        const double a = aval[p];
        for (int q = bptr[k]; q < bptr[k + 1]; ++q) {
            const int j = bcol[q];
            const double prod = __dmul_rn(a, bval[q]);
            int lo = 0, hi = m;                                 // first entry with column >= j
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sc[mid][t] < j) lo = mid + 1; else hi = mid;
            }
            if (lo < m && sc[lo][t] == j) {
                sv[lo][t] = __dadd_rn(sv[lo][t], prod);
            } else {
                if (m == RP_CAP) { full = true; break; }
                for (int e = m; e > lo; --e) {
                    sc[e][t] = sc[e - 1][t];
                    sv[e][t] = sv[e - 1][t];
                }
                sc[lo][t] = j;
                sv[lo][t] = prod;
                ++m;
            }
        }
    }
    if (full) {
        atomicOr(over, 1);
        return;
    }
    const int64_t o = off[i];
    for (int e = 0; e < m; ++e) {
        tcol[o + e] = sc[e][t];
        tval[o + e] = sv[e][t];
    }
    cnt[i] = m;
}

__global__ void k_rowprod_compact(int n, const int64_t* off, const int* tcol, const double* tval, const int* cptr,
                                  int* ccol, double* cval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = off[i];
    const int c0 = cptr[i], m = cptr[i + 1] - c0;
    for (int e = 0; e < m; ++e) {
        ccol[c0 + e] = tcol[o + e];
        cval[c0 + e] = tval[o + e];
    }
}

// Product of short rows (thread per row); false (C untouched) if a row has more than RP_CAP entries.
bool spgemm_rows(const Csr& A, const Csr& B, Csr& C, const int64_t* off, int64_t N, cudaStream_t s) {
    const int n = A.n;
    Tmp<int> tcol(std::max<int64_t>(1, N), s), cnt(n + 1, s), over(1, s);
    Tmp<double> tval(std::max<int64_t>(1, N), s);
    CPC_CK(cudaMemsetAsync(over.get(), 0, sizeof(int), s));
    CPC_CK(cudaMemsetAsync(cnt.get() + n, 0, sizeof(int), s));
    k_rowprod<<<nblk(n, RP_TPB), RP_TPB, 0, s>>>(n, A.ptr.p, A.col.p, A.val.p, B.ptr.p, B.col.p, B.val.p, off,
                                                 tcol.get(), tval.get(), cnt.get(), over.get());
    CPC_LAUNCH_CK();
    if (d2h(over.get(), s)) return false;
    C.n = n;
    C.m = B.m;
    C.ptr.alloc(n + 1);
    exclusive_scan(cnt.get(), C.ptr.p, n + 1, s);
    C.nnz = d2h(C.ptr.p + n, s);
    C.col.alloc(std::max<int64_t>(1, C.nnz));
    C.val.alloc(std::max<int64_t>(1, C.nnz));
    k_rowprod_compact<<<nblk(n), TPB, 0, s>>>(n, off, tcol.get(), tval.get(), C.ptr.p, C.col.p, C.val.p);
    CPC_LAUNCH_CK();
    return true;
}

// Hash product; false (C untouched) if a row cannot be taken.
bool spgemm_hash(const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
    const int n = A.n;
    Tmp<int> cnt(n + 1, s), over(1, s), mx(1, s);
    CPC_CK(cudaMemsetAsync(over.get(), 0, sizeof(int), s));
    CPC_CK(cudaMemsetAsync(cnt.get() + n, 0, sizeof(int), s));
    int dev = 0, sms = 0;
    CPC_CK(cudaGetDevice(&dev));
    CPC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int g = std::max(1, std::min(nblk(n, HS_WARPS), sms * 16));
    k_hs_count<<<g, HS_WARPS * 32, 0, s>>>(n, A.ptr.p, A.col.p, B.ptr.p, B.col.p, cnt.get(), over.get());
    CPC_CK(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
    k_max_int<<<nblk(n), TPB, 0, s>>>(cnt.get(), n, mx.get());
    CPC_LAUNCH_CK();
    if (d2h(over.get(), s)) return false;
    const int most = d2h(mx.get(), s);
    C.n = n;
    C.m = B.m;
    C.ptr.alloc(n + 1);
    exclusive_scan(cnt.get(), C.ptr.p, n + 1, s);
    const int64_t nnz = d2h(C.ptr.p + n, s);
    C.nnz = nnz;
    C.col.alloc(std::max<int64_t>(1, nnz));
    C.val.alloc(std::max<int64_t>(1, nnz));
    int lg = 6;
    while ((1 << lg) < 2 * most) ++lg;
    auto run = [&](auto lgc) {                                 // two warps per CTA for the larger tables
        constexpr int L = decltype(lgc)::value;
        constexpr int W = L <= 8 ? HS_WARPS : 2;
        const int gf = std::max(1, std::min(nblk(n, W), sms * 32));
        k_hs_fill<L, W><<<gf, W * 32, 0, s>>>(n, A.ptr.p, A.col.p, A.val.p, B.ptr.p, B.col.p, B.val.p, C.ptr.p,
                                              C.col.p, C.val.p, over.get());
    };
    if (lg <= 6) run(std::integral_constant<int, 6>{});
    else if (lg == 7) run(std::integral_constant<int, 7>{});
    else if (lg == 8) run(std::integral_constant<int, 8>{});
    else if (lg == 9) run(std::integral_constant<int, 9>{});
    else run(std::integral_constant<int, 10>{});
    CPC_LAUNCH_CK();
    return d2h(over.get(), s) == 0;
}

// C = A * B; every entry sums its products in generation order (row of A ascending, then row of B).
void spgemm_sort(const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
    const int n = A.n;
    C.n = n; C.m = B.m;
    Tmp<int64_t> cnt(n + 1, s), off(n + 1, s);
    k_prod_count<<<nblk(n + 1), TPB, 0, s>>>(n, A.ptr.p, A.col.p, B.ptr.p, cnt.get());
    exclusive_scan(cnt.get(), off.get(), n + 1, s);
    const int64_t N = d2h(off.get() + n, s);
    C.ptr.alloc(n + 1);
    if (N == 0) {
        CPC_CK(cudaMemsetAsync(C.ptr.p, 0, sizeof(int) * (n + 1), s));
        C.nnz = 0; C.col.alloc(1); C.val.alloc(1);
        return;
    }
    if (N > (int64_t)INT_MAX) fail(CPC_ESETUP, "sparse product too large");
    Tmp<uint64_t> key(N, s), key2(N, s);
    Tmp<double> val(N, s), val2(N, s);
    k_prod_expand<<<nblk(n), TPB, 0, s>>>(n, A.ptr.p, A.col.p, A.val.p, B.ptr.p, B.col.p, B.val.p,
                                          (int64_t)B.m, off.get(), key.get(), val.get());
    CPC_LAUNCH_CK();
    sort_pairs(key.get(), key2.get(), val.get(), val2.get(), N,
               bits_for((uint64_t)n * (uint64_t)B.m), s);
    Tmp<int> head(N, s), segid(N, s);
    k_seg_head<<<nblk(N), TPB, 0, s>>>(N, key2.get(), head.get());
    inclusive_scan(head.get(), segid.get(), N, s);
    const int nseg = d2h(segid.get() + N - 1, s);
    Tmp<int64_t> start(nseg, s);
    Tmp<int> rowcnt(n + 1, s);
    CPC_CK(cudaMemsetAsync(rowcnt.get(), 0, sizeof(int) * (n + 1), s));
    k_seg_start<<<nblk(N), TPB, 0, s>>>(N, head.get(), segid.get(), start.get());
    C.nnz = nseg;
    C.col.alloc(nseg);
    C.val.alloc(nseg);
    k_seg_sum<<<nblk(nseg), TPB, 0, s>>>(nseg, N, start.get(), key2.get(), val2.get(), (int64_t)B.m,
                                         C.col.p, C.val.p, rowcnt.get());
    exclusive_scan(rowcnt.get(), C.ptr.p, n + 1, s);
    CPC_LAUNCH_CK();
}

// C = A * B: the hash product, or the sort-based one for rows the hash product cannot take (same
// sums, bit for bit).
void spgemm(const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
    // products per row: short rows (at most twice RP_CAP products) a thread each, else a warp each
    const int n = A.n;
    Tmp<int64_t> cnt(n + 1, s), off(n + 1, s), mx(1, s);
    k_prod_count<<<nblk(n + 1), TPB, 0, s>>>(n, A.ptr.p, A.col.p, B.ptr.p, cnt.get());
    CPC_CK(cudaMemsetAsync(mx.get(), 0, sizeof(int64_t), s));
    k_max_i64<<<nblk(n), TPB, 0, s>>>(cnt.get(), n, mx.get());
    exclusive_scan(cnt.get(), off.get(), n + 1, s);
    CPC_LAUNCH_CK();
    const int64_t most = d2h(mx.get(), s);
    const int64_t N = d2h(off.get() + n, s);
    if (most <= 2 * RP_CAP && spgemm_rows(A, B, C, off.get(), N, s)) return;
    C = Csr{};
    if (spgemm_hash(A, B, C, s)) return;
    C = Csr{};
    spgemm_sort(A, B, C, s);
}

// ============================================================================================
// AMG: strength, PMIS, direct interpolation (Section 3.2 with the stated readings)
// ============================================================================================
__global__ void k_strength(int n, const int* ptr, const int* col, const double* val, double theta,
                           uint8_t* strong) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double mx = 0.0;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p)
        if (col[p] != i) mx = fmax(mx, -val[p]);
    for (int p = ptr[i]; p < ptr[i + 1]; ++p)
        strong[p] = (col[p] != i && mx > 0.0 && -val[p] >= theta * mx) ? 1 : 0;
}

// |S^T_i| = number of rows j with i in S_j
__global__ void k_st_count(int n, const int* ptr, const int* tpos, const uint8_t* strong, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) c += strong[tpos[p]];
    cnt[i] = c;
}

enum : int8_t { ST_UNDEC = -1, ST_F = 0, ST_C = 1 };

__device__ __forceinline__ bool heavier(const int* cnt, int a, int b) {
    if (cnt[a] != cnt[b]) return cnt[a] > cnt[b];
    return fmix32((uint32_t)a) > fmix32((uint32_t)b);
}

__global__ void k_pmis_init(int n, const int* cnt, int8_t* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) st[i] = cnt[i] == 0 ? ST_F : ST_UNDEC;
}

__global__ void k_pmis_select(int n, const int* ptr, const int* col, const int* tpos, const uint8_t* strong,
                              const int* cnt, const int8_t* st, uint8_t* sel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t best = 0;
    if (st[i] == ST_UNDEC) {
        best = 1;
        for (int p = ptr[i]; p < ptr[i + 1] && best; ++p) {
            const int j = col[p];
            if (j == i) continue;
            if ((strong[p] || strong[tpos[p]]) && st[j] == ST_UNDEC && heavier(cnt, j, i)) best = 0;
        }
    }
    sel[i] = best;
}

__global__ void k_pmis_setc(int n, const uint8_t* sel, int8_t* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && sel[i]) st[i] = ST_C;
}

__global__ void k_pmis_setf(int n, const int* ptr, const int* col, const uint8_t* strong, int8_t* st, int* undec) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || st[i] != ST_UNDEC) return;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p)
        if (strong[p] && st[col[p]] == ST_C) { st[i] = ST_F; return; }
    atomicAdd(undec, 1);
}

__global__ void k_cf_flags(int n, const int8_t* st, int* cf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cf[i] = st[i] == ST_C ? 1 : 0;
}

__global__ void k_interp_count(int n, const int* ptr, const int* col, const uint8_t* strong, const int* cf,
                               int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) { cnt[n] = 0; return; }
    if (cf[i]) { cnt[i] = 1; return; }
    int c = 0;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) c += (strong[p] && cf[col[p]]) ? 1 : 0;
    cnt[i] = c;
}

// Direct interpolation:
//   P_ij = -(sum_{k!=i} min(a_ik,0) / sum_{j in C_i} a_ij) a_ij / (a_ii + sum_{k!=i} max(a_ik,0))
__global__ void k_interp_fill(int n, const int* ptr, const int* col, const double* val, const uint8_t* strong,
                              const int* cf, const int* cidx, const int* pptr, int* pcol, double* pval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = pptr[i];
    if (cf[i]) { pcol[o] = cidx[i]; pval[o] = 1.0; return; }
    double sum_neg = 0.0, sum_pos = 0.0, c_neg = 0.0, aii = 0.0;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int j = col[p];
        const double a = val[p];
        if (j == i) { aii = a; continue; }
        if (a < 0.0) sum_neg += a; else sum_pos += a;
        if (strong[p] && cf[j]) c_neg += a;
    }
    if (c_neg == 0.0) return;
    const double alpha = sum_neg / c_neg;
    const double d = aii + sum_pos;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int j = col[p];
        if (j != i && strong[p] && cf[j]) { pcol[o] = cidx[j]; pval[o] = -alpha * val[p] / d; ++o; }
    }
}

// ============================================================================================
// Colouring priority: peel rounds (a smallest-last style ordering).  deg_i = off-diagonal count of
// row i; in round r every remaining point with deg_i <= 2 min_{remaining} deg takes round r, then
// each remaining point loses one degree per entry of its row taken in round r.
// ============================================================================================
// ============================================================================================
// Jones-Plassmann colouring with priority (peel round, fmix32(i ^ COLOUR_SEED)): a point whose
// neighbours of higher priority are all coloured takes the smallest colour they leave free.  Its
// neighbours of lower priority cannot be coloured before it, so the result is the greedy colouring
// in decreasing priority.  Colours written during a round by other threads may or may not be seen
// (volatile reads): seeing one only lets a point finish in an earlier round, with the same colour.
// ============================================================================================
__device__ __forceinline__ bool jp_beats(int rj, int j, int ri, uint32_t hi) {
    return rj > ri || (rj == ri && fmix32((uint32_t)j ^ COLOUR_SEED) > hi);
}

// Grid-wide barrier of a cooperative launch (every CTA resident).  Arrivals count up on *ctr (zero
// before the launch); barrier number e completes when it reaches e * gridDim.x.  The wait gives up
// after GBAR_NS or as soon as another CTA has given up (*err != 0), setting *err = 1; then every
// thread of the CTA gets false and the kernel returns.
constexpr unsigned long long GBAR_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_bar(unsigned long long* ctr, unsigned long long& epoch, int* err) {
    __shared__ int ok;
    ++epoch;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
        const unsigned long long target = epoch * gridDim.x;
        const unsigned long long t0 = gtime_ns();
        int good = 1;
        for (;;) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (*(volatile int*)err != 0 || gtime_ns() - t0 > GBAR_NS) {
                atomicCAS(err, 0, 1);
                good = 0;
                break;
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

constexpr int COL_TPB = 256;
constexpr int COL_G = 16;                                       // lanes per point in k_colour
constexpr int COL_K = 4;                                        // points per lane whose loads overlap

template <class Op>
__device__ int block_reduce(int v, Op op, int identity) {
    __shared__ int part[COL_TPB / 32];
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < COL_TPB / 32 ? part[threadIdx.x] : identity;
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;                                                   // valid in thread 0
}

// blk[i]: the uncoloured neighbour of higher priority that stopped point i last time (-1: none
// yet).  While that neighbour stays uncoloured the point is skipped.  Once it
// is coloured, the point's row is examined again by a group of COL_G lanes (gl = lane in the
// group, gm = the group's lane mask, gs = its first lane in the warp), COL_U entries per lane per
// pass, with all loads of a pass in flight together: the first uncoloured neighbour of higher
// priority in row order is recorded and false returned; if there is none, the point takes the
// smallest colour left free by its neighbours of higher priority (from the colours just loaded
// when the row fits one pass) and true is returned (group-uniform).  Entries before the old
// blocking one are examined again although they cannot block (lower priority, or coloured for
// good): with the loads in flight together that costs nothing, and their colours are needed.
constexpr int COL_U = 4;

// The lowest 32 / COL_G set bits of a warp-uniform mask go to the groups of the warp, one each in
// order: returns group g's bit (-1: none left for it) and clears them all.
__device__ __forceinline__ int take_group_bit(unsigned& bits, int g) {
    int mine = -1;
#pragma unroll
    for (int q = 0; q < 32 / COL_G; ++q) {
        const int b = bits ? __ffs(bits) - 1 : -1;
        if (q == g) mine = b;
        if (bits) bits &= bits - 1;
    }
    return mine;
}

__device__ bool jp_group(int i, int p0, int p1, int ri, const int* col, const int* rnd, volatile int* vc, int* blk,
                         int gl, unsigned gm, int gs) {
    const uint32_t hi = fmix32((uint32_t)i ^ COLOUR_SEED);
    constexpr int W = COL_U * COL_G;                             // entries per pass
    int cj[COL_U];
    bool up[COL_U];                                             // neighbour of higher priority
    for (int base = p0; base < p1; base += W) {
        int j[COL_U];
#pragma unroll
        for (int u = 0; u < COL_U; ++u) {
            const int p = base + u * COL_G + gl;
            j[u] = p < p1 ? col[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < COL_U; ++u) {
            const bool e = j[u] >= 0 && j[u] != i;
            const int rj = e ? rnd[j[u]] : 0;                   // both loads in flight together
            cj[u] = e ? vc[j[u]] : 0;
            up[u] = e && jp_beats(rj, j[u], ri, hi);
        }
#pragma unroll
        for (int u = 0; u < COL_U; ++u) {
            const unsigned bits = (__ballot_sync(gm, up[u] && cj[u] < 0) >> gs) & ((1u << COL_G) - 1u);
            if (bits) {
                const int q = __ffs(bits) - 1;                  // first blocking entry of this batch
                const int jq = __shfl_sync(gm, j[u], gs + q);
                if (gl == 0) blk[i] = jq;
                return false;
            }
        }
    }
    const bool one = p1 - p0 <= W;                              // colours of the only pass still at hand
    for (int cb = 0;; cb += 64) {
        unsigned long long used = 0ull;
        if (one) {
#pragma unroll
            for (int u = 0; u < COL_U; ++u)
                if (up[u] && cj[u] >= cb && cj[u] < cb + 64) used |= 1ull << (cj[u] - cb);
        } else {
            for (int p = p0 + gl; p < p1; p += COL_G) {
                const int j = col[p];
                if (j == i || !jp_beats(rnd[j], j, ri, hi)) continue;
                const int c = vc[j];
                if (c >= cb && c < cb + 64) used |= 1ull << (c - cb);
            }
        }
        for (int o = COL_G / 2; o > 0; o >>= 1) used |= __shfl_xor_sync(gm, used, o);
        if (used != ~0ull) {
            if (gl == 0) vc[i] = cb + __ffsll((long long)~used) - 1;
            return true;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// All levels are coloured by one cooperative launch of k_colour.  Each level runs its own state
// machine, and all advance one step per grid barrier, so that the setup waits for the longest
// chain of rounds, not their sum:
//   init       degrees, round -1, colour -1, blocking entry -1, parity word, triangle probe
//   parity     the breadth-first parity 2-colouring (only if no triangle was found): colour =
//              distance parity from the smallest index of the component.  A union-find over the
//              entries, each word (parent, parity relative to it), joins the two ends of every
//              entry with opposite parities, always hooking the larger root under the smaller:
//              the smallest index stays the root of its component, and for a bipartite graph the
//              parity of a point relative to it is its distance parity (all paths agree)
//   check      any entry joining two points of equal parity: not bipartite, colours reset, go to
//              peel rounds
//   peel       round r, step 1: points with deg <= 2 dmin take round r and count a decrement on
//              each neighbour in dec[]; step 2: the remaining points apply their decrements and
//              the next dmin is their minimum (decrements counted on points taken in the same
//              round are never read)
//   colour     Jones-Plassmann rounds (jp_group)
// The CTAs of a step are shared among the levels with work in that step, in proportion to their
// points (at least one each); a CTA works on one level.
// ---------------------------------------------------------------------------------------------
constexpr int COL_MAXL = CPC_MAX_LEVELS - 1;     // every level but the coarsest is coloured

struct ColLev {
    int n;
    const int* ptr;
    const int* col;
    int* colour;
    int *deg, *dec, *rnd, *blk;
    unsigned* w;                              // union-find words
    int* scal;                                // COL_NS counters, see below
};

// scal of a level: [0], [1] dmin of even / odd peel rounds; [2..4] points coloured in colour
// round t (slot t % 3: a slot is cleared one round before it is added to and read one barrier
// after); [5] triangle found; [6] not bipartite; [7] peel rounds; [8] colour rounds.
enum { CS_DMIN = 0, CS_JP = 2, CS_TRI = 5, CS_BAD = 6, CS_PEEL_ROUNDS = 7, CS_JP_ROUNDS = 8, COL_NS = 12 };
enum { CP_INIT, CP_UNION, CP_FIND, CP_CHECK, CP_RESET, CP_MARK, CP_MIN, CP_JP, CP_DONE };

// Union-find words: parent << 1 | parity relative to the parent (a root: itself, parity 0).
// Returns the root of x and x's parity relative to it, halving the path on the way (a point is
// re-pointed to its grandparent with the composed parity, only if its word is still the one read).
__device__ int uf_find(unsigned* uf, int x, int& par) {
    volatile unsigned* v = uf;
    int cur = x;
    unsigned w = v[cur];
    par = 0;
    while ((int)(w >> 1) != cur) {
        const int p = (int)(w >> 1);
        const unsigned wp = v[p];
        if ((int)(wp >> 1) == p) {                              // p is the root
            par ^= (int)(w & 1u);
            return p;
        }
        const unsigned nw = (wp & ~1u) | ((w ^ wp) & 1u);       // grandparent, composed parity
        atomicCAS(&uf[cur], w, nw);
        par ^= (int)((w ^ wp) & 1u);
        cur = (int)(wp >> 1);
        w = v[cur];
    }
    return cur;
}

// Joins a and b with opposite parities (the larger root is hooked under the smaller); false if
// it has not succeeded within a bound of attempts (other joins keep winning the race).
__device__ bool uf_join(unsigned* uf, int a, int b) {
    for (int attempt = 0; attempt < (1 << 20); ++attempt) {
        int pa, pb;
        int ra = uf_find(uf, a, pa), rb = uf_find(uf, b, pb);
        if (ra == rb) return true;
        if (ra > rb) {
            const int t = ra; ra = rb; rb = t;
            const int u = pa; pa = pb; pb = u;
        }
        const unsigned x = (unsigned)(pa ^ pb ^ 1) & 1u;
        if (atomicCAS(&uf[rb], (unsigned)rb << 1, ((unsigned)ra << 1) | x) == ((unsigned)rb << 1)) return true;
    }
    return false;
}

// A triangle at point i (adjacent neighbours j, k among its first 8 entries) proves that the
// graph is not bipartite; finding none proves nothing.
__device__ bool tri_probe(int i, const int* ptr, const int* col) {
    const int p0 = ptr[i], p1 = min(ptr[i + 1], ptr[i] + 8);
    for (int a = p0; a < p1; ++a) {
        const int j = col[a];
        if (j == i) continue;
        for (int b = a + 1; b < p1; ++b) {
            const int k = col[b];
            if (k == i) continue;
            int lo = ptr[j], hi = ptr[j + 1] - 1;              // columns ascending: binary search for k
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int c = col[mid];
                if (c == k) return true;
                if (c < k) lo = mid + 1; else hi = mid - 1;
            }
        }
    }
    return false;
}

// The work of one step of one level on the threads [t0, t0 + T) of its CTAs (t = t0 + local
// index; whole CTAs, so that the block reductions see every thread of the CTA).
__device__ void col_step(const ColLev& V, int phase, int rnd_no, int dm, int t, int T) {
    auto imin = [](int a, int b) { return a < b ? a : b; };
    auto iadd = [](int a, int b) { return a + b; };
    const int n = V.n;
    const int* ptr = V.ptr;
    const int* col = V.col;
    const int lane = threadIdx.x & 31, gl = lane % COL_G, gs = lane - gl;
    const unsigned gm = ((1u << COL_G) - 1u) << gs;
    if (phase == CP_INIT) {
        int m = INT_MAX, tri = 0;
        for (int i = t; i < n; i += T) {
            int d = 0;
            for (int p = ptr[i]; p < ptr[i + 1]; ++p) d += col[p] != i;
            V.deg[i] = d;
            V.dec[i] = 0;
            V.rnd[i] = -1;
            V.colour[i] = -1;
            V.blk[i] = -1;
            V.w[i] = (unsigned)i << 1;
            m = imin(m, d);
            if (!tri) tri = tri_probe(i, ptr, col);
        }
        m = block_reduce(m, imin, INT_MAX);
        tri = block_reduce(tri, iadd, 0);
        if (threadIdx.x == 0) {
            if (m != INT_MAX) atomicMin(&V.scal[CS_DMIN], m);
            if (tri) atomicOr(&V.scal[CS_TRI], 1);
        }
    } else if (phase == CP_UNION) {
        int fail = 0;
        for (int i = t; i < n; i += T)
            for (int p = ptr[i]; p < ptr[i + 1]; ++p)
                if (col[p] > i && !uf_join(V.w, i, col[p])) fail = 1;
        fail = block_reduce(fail, iadd, 0);
        if (threadIdx.x == 0 && fail) atomicOr(&V.scal[CS_BAD], 2);
    } else if (phase == CP_FIND) {
        for (int i = t; i < n; i += T) {
            int par;
            uf_find(V.w, i, par);
            V.colour[i] = par;
        }
    } else if (phase == CP_CHECK) {
        int bad = 0;
        for (int i = t; i < n && !bad; i += T) {
            const int ci = __ldcg(&V.colour[i]);
            for (int p = ptr[i]; p < ptr[i + 1]; ++p)
                if (col[p] != i && __ldcg(&V.colour[col[p]]) == ci) { bad = 1; break; }
        }
        bad = block_reduce(bad, iadd, 0);
        if (threadIdx.x == 0 && bad) atomicOr(&V.scal[CS_BAD], 1);
    } else if (phase == CP_RESET) {
        for (int i = t; i < n; i += T) V.colour[i] = -1;
    } else if (phase == CP_MARK) {
        for (int b0 = t - lane; b0 < n; b0 += COL_K * T) {     // warp-uniform trip count
            bool take[COL_K];
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {                   // loads of COL_K points in flight
                const int i = b0 + k * T + lane;
                take[k] = i < n && __ldcg(&V.rnd[i]) < 0 && __ldcg(&V.deg[i]) <= 2 * dm;
            }
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {
                const int base = b0 + k * T;
                if (take[k]) V.rnd[base + lane] = rnd_no;
                unsigned bits = __ballot_sync(0xffffffffu, take[k]);
                while (bits) {                                  // a taken point per group at a time
                    const int mine = take_group_bit(bits, gs / COL_G);
                    if (mine >= 0) {
                        const int ip = base + mine;
                        for (int p = ptr[ip] + gl; p < ptr[ip + 1]; p += COL_G)
                            if (col[p] != ip) atomicSub(&V.dec[col[p]], 1);
                    }
                }
            }
        }
    } else if (phase == CP_MIN) {
        int m = INT_MAX;
        for (int i0 = t; i0 < n; i0 += COL_K * T) {
            int rv[COL_K], dv[COL_K], ev[COL_K];
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {                   // loads of COL_K points in flight
                const int i = i0 + k * T;
                rv[k] = i < n ? __ldcg(&V.rnd[i]) : 0;
                dv[k] = i < n ? __ldcg(&V.deg[i]) : 0;
                ev[k] = i < n ? __ldcg(&V.dec[i]) : 0;
            }
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {
                const int i = i0 + k * T;
                if (i >= n || rv[k] >= 0) continue;
                const int d = dv[k] + ev[k];
                V.deg[i] = d;
                V.dec[i] = 0;
                m = imin(m, d);
            }
        }
        m = block_reduce(m, imin, INT_MAX);
        if (threadIdx.x == 0 && m != INT_MAX) atomicMin(&V.scal[CS_DMIN + ((rnd_no + 1) & 1)], m);
    } else if (phase == CP_JP) {
        volatile int* vc = V.colour;
        int cnt = 0;
        for (int b0 = t - lane; b0 < n; b0 += COL_K * T) {     // warp-uniform trip count
            int cv[COL_K], bv[COL_K], vb[COL_K];
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {                   // loads of COL_K points in flight
                const int i = b0 + k * T + lane;
                cv[k] = i < n ? vc[i] : 0;
                bv[k] = i < n ? V.blk[i] : -1;
            }
#pragma unroll
            for (int k = 0; k < COL_K; ++k) vb[k] = cv[k] < 0 && bv[k] >= 0 ? vc[bv[k]] : -1;
#pragma unroll
            for (int k = 0; k < COL_K; ++k) {
                const int base = b0 + k * T;
                // uncoloured, and either never examined or its blocker has been coloured since
                const bool ready = cv[k] < 0 && (bv[k] < 0 || vb[k] >= 0);
                int q0 = 0, q1 = 0, qr = 0;                     // row bounds and round of a ready point
                if (ready) {
                    q0 = ptr[base + lane];
                    q1 = ptr[base + lane + 1];
                    qr = V.rnd[base + lane];
                }
                unsigned bits = __ballot_sync(0xffffffffu, ready);
                while (bits) {                                  // a ready point per group at a time
                    const int mine = take_group_bit(bits, gs / COL_G);
                    const int src = mine < 0 ? 0 : mine;
                    const int m0 = __shfl_sync(0xffffffffu, q0, src), m1 = __shfl_sync(0xffffffffu, q1, src);
                    const int mr = __shfl_sync(0xffffffffu, qr, src);
                    if (mine >= 0 && jp_group(base + mine, m0, m1, mr, col, V.rnd, vc, V.blk, gl, gm, gs) && gl == 0) ++cnt;
                }
            }
        }
        cnt = block_reduce(cnt, iadd, 0);
        if (threadIdx.x == 0 && cnt) atomicAdd(&V.scal[CS_JP + rnd_no % 3], cnt);
    }
}

// *err: 1 a barrier gave up, 2 peel rounds or 3 colour rounds beyond their bound, 4 a union-find
// join kept losing its race.
// Each CTA keeps the level descriptors and the levels' phases in shared memory; at each step its
// threads load every level's counters at once (they change only before a barrier), thread 0 takes
// the phase decisions (the same in every CTA) and picks the CTA's level, and the CTA works on it.
__global__ void __launch_bounds__(COL_TPB) k_colour(const ColLev* levs, int nlev, unsigned long long* bar, int* err) {
    __shared__ ColLev lv[COL_MAXL];
    __shared__ int sc[COL_MAXL * COL_NS];
    __shared__ int ph[COL_MAXL], rr[COL_MAXL], work[COL_MAXL], dmv[COL_MAXL];
    __shared__ long long done[COL_MAXL];
    __shared__ int mine, c0s, cns, quit;
    unsigned long long epoch = 0;
    const bool lead = threadIdx.x == 0, first = lead && blockIdx.x == 0;
    for (int l = threadIdx.x; l < nlev; l += blockDim.x) {
        lv[l] = levs[l];
        ph[l] = CP_INIT;
        rr[l] = 0;
        done[l] = 0;
    }
    __syncthreads();
    for (int step = 0;; ++step) {
        for (int q = threadIdx.x; q < nlev * COL_NS; q += blockDim.x) sc[q] = __ldcg(&lv[q / COL_NS].scal[q % COL_NS]);
        __syncthreads();
        if (lead) {
            // transitions: every CTA reads the same counters and takes the same decisions
            int active = 0;
            long long wsum = 0;
            quit = 0;
            for (int l = 0; l < nlev && !quit; ++l) {
                const int* c = sc + l * COL_NS;
                int* g = lv[l].scal;
                const int n = lv[l].n;
                work[l] = -1;
                for (;;) {                                      // a phase change may act at once
                    const int p = ph[l];
                    if (p == CP_INIT) {
                        if (step == 0) { work[l] = CP_INIT; break; }
                        ph[l] = c[CS_TRI] ? CP_MARK : CP_UNION;
                        rr[l] = 0;
                        if (ph[l] == CP_UNION) { work[l] = CP_UNION; break; }
                    } else if (p == CP_UNION) {
                        if (c[CS_BAD] & 2) { if (first) atomicCAS(err, 0, 4); quit = 1; break; }
                        ph[l] = CP_FIND;
                        work[l] = CP_FIND;
                        break;
                    } else if (p == CP_FIND) {
                        ph[l] = CP_CHECK;
                        work[l] = CP_CHECK;
                        break;
                    } else if (p == CP_CHECK) {
                        if (c[CS_BAD]) {
                            ph[l] = CP_RESET;
                            work[l] = CP_RESET;
                        } else {
                            ph[l] = CP_DONE;
                        }
                        break;
                    } else if (p == CP_RESET) {
                        ph[l] = CP_MARK;
                        rr[l] = 0;
                    } else if (p == CP_MARK) {
                        dmv[l] = c[CS_DMIN + (rr[l] & 1)];
                        if (dmv[l] == INT_MAX) {
                            if (first) g[CS_PEEL_ROUNDS] = rr[l];
                            ph[l] = CP_JP;
                            rr[l] = 0;
                            continue;
                        }
                        if (rr[l] > n + 16) { if (first) atomicCAS(err, 0, 2); quit = 1; break; }
                        if (first) g[CS_DMIN + ((rr[l] + 1) & 1)] = INT_MAX;
                        work[l] = CP_MARK;
                        break;
                    } else if (p == CP_MIN) {
                        work[l] = CP_MIN;
                        break;
                    } else if (p == CP_JP) {
                        if (rr[l] > 0) {
                            done[l] += c[CS_JP + (rr[l] - 1) % 3];
                            if (done[l] >= n) {
                                if (first) g[CS_JP_ROUNDS] = rr[l];
                                ph[l] = CP_DONE;
                                break;
                            }
                        }
                        if (rr[l] > n + 32) { if (first) atomicCAS(err, 0, 3); quit = 1; break; }
                        if (first) g[CS_JP + (rr[l] + 1) % 3] = 0;
                        work[l] = CP_JP;
                        break;
                    } else {
                        break;                                  // done
                    }
                }
                if (work[l] >= 0) {
                    ++active;
                    wsum += n;
                }
            }
            mine = -1;
            if (!quit && active == 0) {
                bool all = true;
                for (int l = 0; l < nlev; ++l) all = all && ph[l] == CP_DONE;
                quit = all ? 2 : 3;                             // 3: transitions only, no work, no barrier
            }
            if (!quit) {
                // one CTA per level with work, the others in proportion to points
                const int G = gridDim.x, spare = G - active;
                int c0 = 0, cs = 0;
                long long wacc = 0;
                for (int l = 0; l < nlev && mine < 0; ++l) {
                    if (work[l] < 0) continue;
                    wacc += lv[l].n;
                    const int c1 = (int)(((long long)spare * wacc) / wsum) + (++cs);
                    if ((int)blockIdx.x >= c0 && (int)blockIdx.x < c1) {
                        mine = l;
                        c0s = c0;
                        cns = c1 - c0;
                    } else {
                        c0 = c1;
                    }
                }
            }
        }
        __syncthreads();
        if (quit == 1 || quit == 2) return;
        if (quit == 3) continue;
        if (mine >= 0) {
            const int l = mine;
            col_step(lv[l], work[l], rr[l], work[l] == CP_MARK ? dmv[l] : 0, ((int)blockIdx.x - c0s) * COL_TPB + threadIdx.x,
                     cns * COL_TPB);
        }
        __syncthreads();
        if (lead) {                                             // advance the phases worked in this step
            for (int l = 0; l < nlev; ++l) {
                if (work[l] == CP_JP) ++rr[l];
                else if (work[l] == CP_MARK) ph[l] = CP_MIN;
                else if (work[l] == CP_MIN) {
                    ph[l] = CP_MARK;
                    ++rr[l];
                }
            }
        }
        if (!grid_bar(bar, epoch, err)) return;
    }
}

// ============================================================================================
// IC(0): level scheduling and factorisation (Algorithm 3.1, k = 0)
// ============================================================================================
// One round: rows whose dependencies (lower: j < i, upper: j > i) all have levels < round get
// level = round.
__global__ void k_dag_round(int n, const int* ptr, const int* col, int* lvl, int round, int upper, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || lvl[i] >= 0) return;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int j = col[p];
        if (upper ? j > i : j < i) {
            const int lj = lvl[j];
            if (lj < 0 || lj >= round) return;
        }
    }
    lvl[i] = round;
    atomicAdd(cnt, 1);
}

// IKJ elimination of the rows of one level: for m < i in the row (ascending), l_im = a_im / u_mm,
// then a_ij -= l_im u_mj for j > m in both rows.  Products and differences are rounded
// separately (no fused multiply-add), in the same order as the plain sequential algorithm.
__global__ void k_ic0_level(const int* rows, int cnt, const int* ptr, const int* col, const int* diag,
                            double* lu, int* fail, int min_len) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = rows[t];
    if (ptr[i + 1] - ptr[i] < min_len) return;               // a warp of k_ic0_level_warp has it
    const int di = diag[i];
    const int end_i = ptr[i + 1];
    for (int p = ptr[i]; p < di; ++p) {
        const int m = col[p];
        const double l = lu[p] / lu[diag[m]];
        lu[p] = l;
        int pi = p + 1;
        for (int q = diag[m] + 1; q < ptr[m + 1]; ++q) {
            const int j = col[q];
            while (pi < end_i && col[pi] < j) ++pi;
            if (pi >= end_i) break;
            if (col[pi] == j) lu[pi] = __dsub_rn(lu[pi], __dmul_rn(l, lu[q]));
        }
    }
    const double u = lu[di];
    if (!(u > 0.0) || !isfinite(u)) atomicMin(fail, i);
}

__global__ void k_max_rowlen(int n, const int* ptr, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, ptr[i + 1] - ptr[i]);
}

// The same elimination with a warp per row, for long rows: row i (columns and values) is staged in
// shared memory; for each m (ascending) one lane forms l_im, then the lanes take the entries j > m
// of row m, find j in row i by binary search and apply a_ij -= l_im u_mj, each product and
// difference rounded separately.  Every entry of row i receives its updates in ascending m, as in
// k_ic0_level, so the factor is the same to the bit.  Rows longer than IC_WROW are left to
// k_ic0_level (min_len = IC_WROW + 1 there: each kernel takes its own rows).
constexpr int IC_WROW = 2048;
constexpr int IC_WARPS = 2;

__global__ void __launch_bounds__(IC_WARPS * 32) k_ic0_level_warp(const int* rows, int cnt, const int* ptr,
                                                                   const int* col, const int* diag, double* lu,
                                                                   int* fail) {
    __shared__ int s_col[IC_WARPS][IC_WROW];
    __shared__ double s_val[IC_WARPS][IC_WROW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * IC_WARPS + w;
    if (t >= cnt) return;
    const int i = rows[t];
    const int p0 = ptr[i], len = ptr[i + 1] - p0;
    if (len > IC_WROW) return;
    int* sc = s_col[w];
    double* sv = s_val[w];
    for (int e = lane; e < len; e += 32) {
        sc[e] = col[p0 + e];
        sv[e] = lu[p0 + e];
    }
    __syncwarp();
    const int dl = diag[i] - p0;                              // the diagonal's position in row i
    for (int e = 0; e < dl; ++e) {                            // m = col of entry e, ascending
        const int m = sc[e];
        const int dm = diag[m];
        const double l = sv[e] / lu[dm];                      // every lane forms the same quotient
        __syncwarp();
        if (lane == 0) sv[e] = l;
        const int q1 = ptr[m + 1];
        for (int q = dm + 1 + lane; q < q1; q += 32) {
            const int j = col[q];
            int lo = e + 1, hi = len - 1;                     // j > m: after entry e
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sc[mid] < j) lo = mid + 1; else hi = mid;
            }
            if (lo < len && sc[lo] == j) sv[lo] = __dsub_rn(sv[lo], __dmul_rn(l, lu[q]));
        }
        __syncwarp();
    }
    for (int e = lane; e < len; e += 32) lu[p0 + e] = sv[e];
    if (lane == 0) {
        const double u = sv[dl];
        if (!(u > 0.0) || !isfinite(u)) atomicMin(fail, i);
    }
}

// Symmetric permutation B = Q^T A Q: new row q is old row order[q], columns renumbered by inv.
__global__ void k_perm_rowlen(int n, const int* ptr, const int* order, int* len) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > n) return;
    if (q == n) { len[n] = 0; return; }
    const int i = order[q];
    len[q] = ptr[i + 1] - ptr[i];
}

__global__ void k_perm_fill(int n, const int* ptr, const int* col, const double* val, const int* order,
                            const int* inv, const int* bptr, int* bcol, double* bval) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = order[q];
    const int o = bptr[q];
    const int len = ptr[i + 1] - ptr[i];
    for (int e = 0; e < len; ++e) {            // insertion sort by new column
        const int c = inv[col[ptr[i] + e]];
        const double v = val[ptr[i] + e];
        int w = e;
        while (w > 0 && bcol[o + w - 1] > c) { bcol[o + w] = bcol[o + w - 1]; bval[o + w] = bval[o + w - 1]; --w; }
        bcol[o + w] = c;
        bval[o + w] = v;
    }
}

__global__ void k_inverse_perm(int n, const int* order, int* inv) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) inv[order[q]] = q;
}

// ============================================================================================
// SELL-C construction
// ============================================================================================
enum SellMode { SELL_OFFDIAG = 0, SELL_LOWER = 1, SELL_UPPER = 2, SELL_ALL = 3 };

__device__ __forceinline__ bool sell_keep(int mode, int j, int i) {
    switch (mode) {
        case SELL_OFFDIAG: return j != i;
        case SELL_LOWER: return j < i;
        case SELL_UPPER: return j > i;
        default: return true;
    }
}

__global__ void k_sell_width(const int* perm, int nchunks, int C, const int* ptr, const int* col, int mode,
                             int* width) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nchunks) return;
    if (k == nchunks) { width[k] = 0; return; }
    int w = 0;
    for (int l = 0; l < C; ++l) {
        const int i = perm[k * C + l];
        if (i < 0) continue;
        int c = 0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) c += sell_keep(mode, col[p], i) ? 1 : 0;
        w = max(w, c);
    }
    width[k] = w * C;
}

template <class T>
__global__ void k_slot_to_nat(int nslots, const int* perm, const T* v, T* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nslots && perm[s] >= 0) out[perm[s]] = v[s];
}


// Slots refer to rows of the CSR; imap (optional) renames rows and columns on output
// (IC factor stored in its own ordering but applied to naturally ordered vectors).
__global__ void k_sell_fill(const int* perm, int nslots, int C, const int* ptr, const int* col, const double* val,
                            int mode, const int* cptr, const int* imap, int* perm_out, int* scol, double* sval,
                            double* sdiag) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int k = s / C, lane = s % C;
    const int base = cptr[k];
    const int w = (cptr[k + 1] - base) / C;
    const int i = perm[s];
    const int out_row = i < 0 ? -1 : (imap ? imap[i] : i);
    perm_out[s] = out_row;
    int e = 0;
    double d = 1.0;
    if (i >= 0) {
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int j = col[p];
            if (j == i) d = val[p];
            if (sell_keep(mode, j, i)) {
                scol[base + e * C + lane] = imap ? imap[j] : j;
                sval[base + e * C + lane] = val[p];
                ++e;
            }
        }
    }
    for (; e < w; ++e) {                       // padding: column -1, skipped by every kernel
        scol[base + e * C + lane] = -1;
        sval[base + e * C + lane] = 0.0;
    }
    if (sdiag) sdiag[s] = d;
}

// Slot order from a per-row group key (colour or level): rows sorted by (key, row), each group
// padded to a multiple of the chunk height C.  Returns the chunk boundaries of the groups in seg.
__global__ void k_group_count(int n, const int* key, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key[i]], 1);
}

__global__ void k_group_scatter(int n, const int* skey, const int* srow, const int* gstart, const int* sstart,
                                int* perm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int g = skey[t];
    perm[sstart[g] + (t - gstart[g])] = srow[t];
}

// Build perm (device, nslots) from a group key per row; ngroups known.
void grouped_slots(int n, const int* key, int ngroups, int C, cudaStream_t s, DBuf<int>& perm, int& nslots,
                   std::vector<int>& seg, DBuf<int>* sorted_rows = nullptr) {
    Tmp<int> rows(n, s), skey(n, s), srow(n, s), cnt(ngroups, s);
    k_iota<<<nblk(n), TPB, 0, s>>>(rows.get(), n);
    sort_pairs(key, skey.get(), rows.get(), srow.get(), n, bits_for((uint64_t)std::max(1, ngroups)), s);
    CPC_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int) * ngroups, s));
    k_group_count<<<nblk(n), TPB, 0, s>>>(n, key, cnt.get());
    std::vector<int> hc(ngroups);
    CPC_CK(cudaMemcpyAsync(hc.data(), cnt.get(), sizeof(int) * ngroups, cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    std::vector<int> gstart(ngroups), sstart(ngroups);
    seg.assign(ngroups + 1, 0);
    int g0 = 0, s0 = 0;
    for (int g = 0; g < ngroups; ++g) {
        gstart[g] = g0;
        sstart[g] = s0;
        seg[g] = s0 / C;
        g0 += hc[g];
        s0 += (hc[g] + C - 1) / C * C;
    }
    seg[ngroups] = s0 / C;
    nslots = s0;
    perm.alloc_async(nslots, s);                                // a temporary slot order
    k_fill_int<<<nblk(nslots), TPB, 0, s>>>(perm.p, nslots, -1);
    Tmp<int> dg(ngroups, s), ds(ngroups, s);
    h2d(dg.get(), gstart.data(), ngroups, s);
    h2d(ds.get(), sstart.data(), ngroups, s);
    k_group_scatter<<<nblk(n), TPB, 0, s>>>(n, skey.get(), srow.get(), dg.get(), ds.get(), perm.p);
    if (sorted_rows) {
        sorted_rows->alloc(n);
        CPC_CK(cudaMemcpyAsync(sorted_rows->p, srow.get(), sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    CPC_CK(cudaStreamSynchronize(s));      // host vectors above go out of scope
    CPC_LAUNCH_CK();
}

void natural_slots(int n, int C, cudaStream_t s, DBuf<int>& perm, int& nslots, std::vector<int>& seg) {
    nslots = (n + C - 1) / C * C;
    perm.alloc_async(nslots, s);                                // a temporary slot order
    k_fill_int<<<nblk(nslots), TPB, 0, s>>>(perm.p, nslots, -1);
    k_iota<<<nblk(n), TPB, 0, s>>>(perm.p, n);
    seg = {0, nslots / C};
    CPC_LAUNCH_CK();
}

__global__ void k_recip(int n, const double* d, double* r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = 1.0 / d[i];
}

// Chunk height for rows of average length avg: 32 / G rows per warp with G lanes sharing a row,
// G the largest power of two <= avg / 4 (1..8), so that a row costs one round of loads.
int choose_chunk(double avg) {
    int G = 1;
    while (G < 8 && 2 * G <= avg / 4.0) G *= 2;
    return 32 / G;
}

// Fill a Sell of chunk height C from CSR rows in the slot order `slots` (device, nslots entries).
void build_sell(const int* ptr, const int* col, const double* val, const DBuf<int>& slots, int nslots,
                const std::vector<int>& seg, int C, int mode, bool split_diag, const int* imap, Sell& S,
                cudaStream_t s) {
    S.nslots = nslots;
    S.C = C;
    S.nchunks = nslots / C;
    S.seg = seg;
    Tmp<int> width(S.nchunks + 1, s);
    k_sell_width<<<nblk(S.nchunks + 1), TPB, 0, s>>>(slots.p, S.nchunks, C, ptr, col, mode, width.get());
    {
        Tmp<int> wmax(1, s);
        CPC_CK(cudaMemsetAsync(wmax.get(), 0, sizeof(int), s));
        k_max_int<<<nblk(S.nchunks + 1), TPB, 0, s>>>(width.get(), S.nchunks + 1, wmax.get());
        S.lanes = (d2h(wmax.get(), s) + 31) / 32;
    }
    S.cptr.alloc(S.nchunks + 1);
    exclusive_scan(width.get(), S.cptr.p, S.nchunks + 1, s);
    S.nelem = d2h(S.cptr.p + S.nchunks, s);
    S.perm.alloc(nslots);
    S.col.alloc(S.nelem);
    S.val.alloc(S.nelem);
    if (split_diag) S.diag.alloc(nslots);
    k_sell_fill<<<nblk(nslots), TPB, 0, s>>>(slots.p, nslots, C, ptr, col, val, mode, S.cptr.p, imap, S.perm.p,
                                             S.col.p, S.val.p, split_diag ? S.diag.p : nullptr);
    if (split_diag) {       // reciprocal diagonal: the sweeps multiply instead of dividing
        S.dinv.alloc(nslots);
        k_recip<<<nblk(nslots), TPB, 0, s>>>(nslots, S.diag.p, S.dinv.p);
    }
    CPC_LAUNCH_CK();
}

// Distinct off-diagonal offsets col - row of the rows, into a table of 8 (EMPTY = INT_MIN: no offset
// can be INT_MIN); *over = 1 when there are more than 8.
__global__ void k_dia_offsets(int n, const int* ptr, const int* col, int* table, int* over) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    volatile int* vt = table;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        const int j = col[p];
        if (j == i) continue;
        const int off = j - i;
        bool found = false;
        for (int t = 0; t < 8 && !found; ++t) {
            int cur = vt[t];
            if (cur == INT_MIN) cur = atomicCAS(table + t, INT_MIN, off);
            found = cur == INT_MIN || cur == off;
        }
        if (!found) *over = 1;
    }
}

// dval[d * nslots + s] = a_{i, i + off_d} for slot s = row i (0 where absent or padding).
__global__ void k_dia_fill(int nslots, const int* perm, const int* ptr, const int* col, const double* val, int nd,
                           DiaOff off, double* dval) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int i = perm[s];
    for (int d = 0; d < nd; ++d) {
        double v = 0.0;
        if (i >= 0 && off.o[d] != 0)
            for (int p = ptr[i]; p < ptr[i + 1]; ++p)
                if (col[p] == i + off.o[d]) v = val[p];
        dval[(size_t)d * nslots + s] = v;
    }
}

// gval[s * nd + d] = -dval[d * nslots + s] / a_ii (times the stored reciprocal).
__global__ void k_gval(int nslots, int nd, const double* dval, const double* dinv, double* gval) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    for (int d = 0; d < nd; ++d) gval[(size_t)s * nd + d] = -(dval[(size_t)d * nslots + s] * dinv[s]);
}

// Adds the diagonal form to S (built from the same CSR rows, diagonal split) when the off-diagonal
// entries lie on at most 8 offsets; ndiag is rounded up to 4, 6 or 8 with zero diagonals.
void build_dia(int n, const int* ptr, const int* col, const double* val, Sell& S, cudaStream_t s, bool gs = false) {
    Tmp<int> table(8, s), over(1, s);
    k_fill_int<<<1, 32, 0, s>>>(table.get(), 8, INT_MIN);
    CPC_CK(cudaMemsetAsync(over.get(), 0, sizeof(int), s));
    k_dia_offsets<<<nblk(n), TPB, 0, s>>>(n, ptr, col, table.get(), over.get());
    CPC_LAUNCH_CK();
    int t[8];
    CPC_CK(cudaMemcpyAsync(t, table.get(), sizeof(t), cudaMemcpyDeviceToHost, s));
    const int ov = d2h(over.get(), s);
    if (ov) return;
    std::vector<int> offs;
    for (int q = 0; q < 8; ++q) if (t[q] != INT_MIN) offs.push_back(t[q]);
    if (offs.empty()) return;
    std::sort(offs.begin(), offs.end());
    const int nd = offs.size() <= 4 ? 4 : (offs.size() <= 6 ? 6 : 8);
    DiaOff o{};
    for (int q = 0; q < nd; ++q) o.o[q] = q < (int)offs.size() ? offs[q] : 0;
    // padding diagonals (offset 0, value 0) go last; the real ones stay in ascending column order
    S.dval.alloc((size_t)nd * S.nslots);
    k_dia_fill<<<nblk(S.nslots), TPB, 0, s>>>(S.nslots, S.perm.p, ptr, col, val, nd, o, S.dval.p);
    CPC_LAUNCH_CK();
    S.ndiag = nd;
    S.doff = o;
    if (gs && S.dinv.p) {
        S.gval.alloc((size_t)nd * S.nslots);
        k_gval<<<nblk(S.nslots), TPB, 0, s>>>(S.nslots, nd, S.dval.p, S.dinv.p, S.gval.p);
        CPC_LAUNCH_CK();
    }
}

__global__ void k_to_f32(int64_t n, const double* a, float* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_bf16(int64_t n, const double* a, __nv_bfloat16* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2bfloat16(a[i]);
}

void sell_lowp(Sell& S, VType vt, cudaStream_t s) {
    if (vt == VT_F64) return;
    if (S.ndiag) {
        const int64_t m = (int64_t)S.ndiag * S.nslots;
        S.dval32.alloc(m);
        k_to_f32<<<nblk(m), TPB, 0, s>>>(m, S.dval.p, S.dval32.p);
        if (S.gval.p) {
            S.gval32.alloc(m);
            k_to_f32<<<nblk(m), TPB, 0, s>>>(m, S.gval.p, S.gval32.p);
        }
    }
    S.val32.alloc(S.nelem);
    k_to_f32<<<nblk(S.nelem), TPB, 0, s>>>(S.nelem, S.val.p, S.val32.p);
    if (S.diag.p) {
        S.diag32.alloc(S.nslots);
        k_to_f32<<<nblk(S.nslots), TPB, 0, s>>>(S.nslots, S.diag.p, S.diag32.p);
        S.dinv32.alloc(S.nslots);
        k_to_f32<<<nblk(S.nslots), TPB, 0, s>>>(S.nslots, S.dinv.p, S.dinv32.p);
    }
    if (vt == VT_BF16) {
        S.val16.alloc(S.nelem);
        k_to_bf16<<<nblk(S.nelem), TPB, 0, s>>>(S.nelem, S.val.p, S.val16.p);
    }
    CPC_LAUNCH_CK();
}

// ============================================================================================
// Coarsest level: the explicit inverse X = A_c^{-1} (Algorithm 3.2, step 2(b)).
// Dense Cholesky A_c = L L^T, blocked right-looking with panels of NB = 32 columns:
//   k_chol_diag   factor the 32 x 32 diagonal block and invert it (k_chol_diag_warp in FP32),
//   chol_trsm     L21 = A21 L11^{-T} as a tile product with that inverse,
//   chol_syrk     A22 -= L21 L21^T on the lower triangle, 64 x 64 tiles;
// with W = L^{-1} by row panels in the same launches (trinv_panel, trinv_update: k_panel_rows and
// k_panel_update), then A_c^{-1} = W^T W (k_lauum_part, k_lauum_sum).  L is left in the lower triangle of M.  The kernels are templated on the element
// type: the inverse is first formed in FP32 (FP64 issue is scarce on this part) and then refined
// to FP64 accuracy by Newton-Schulz steps (refined_inverse); the FP64 instantiation is the
// fallback when that does not converge.
// ============================================================================================
constexpr int CHOL_NB = 32;

template <class T>
__global__ void k_csr_to_dense(int n, const int* ptr, const int* col, const double* val, T* M) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = ptr[i]; p < ptr[i + 1]; ++p) M[(size_t)i * n + col[p]] = T(val[p]);
}

// Factor the nb x nb diagonal block (nb <= 32) in shared memory with CHOL_DT threads, write L11
// back, and write Li = L11^{-1} (lower triangular, 32 x 32 with zeros beyond nb) for the tile
// products of the panel.  Each elimination step spreads its trailing update over all threads (four
// warps: on this part one warp alone issues FP64 at a quarter of the SM's rate); the inverse is
// formed right-looking on [L11 | I]: row j of X scaled by 1 / l_jj, then subtracted from the rows
// below, so every step is a short parallel update.
constexpr int CHOL_DT = 128;

template <class T>
__global__ void __launch_bounds__(CHOL_DT) k_chol_diag(int n, int jb, T* M, T* Li, int* fail) {
    __shared__ T D[CHOL_NB][CHOL_NB + 1];
    __shared__ T X[CHOL_NB][CHOL_NB + 1];
    const int tid = threadIdx.x;
    const int nb = min(CHOL_NB, n - jb);
    if (*(volatile int*)fail) return;
    for (int t = tid; t < CHOL_NB * CHOL_NB; t += CHOL_DT) {
        const int r = t / CHOL_NB, c = t % CHOL_NB;
        D[r][c] = (r < nb && c <= r) ? M[(size_t)(jb + r) * n + jb + c] : T(0);
        X[r][c] = (r == c && r < nb) ? T(1) : T(0);
    }
    __syncthreads();
    __shared__ T piv_inv;
    __shared__ int piv_bad;
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {                                       // one thread takes the pivot's root
            const T d = D[j][j];
            piv_bad = !(d > T(0)) || !isfinite(d);
            if (!piv_bad) {
                const T sj = sqrt(d);
                D[j][j] = sj;
                piv_inv = T(1) / sj;
            }
        }
        __syncthreads();
        if (piv_bad) {                                        // the same for every thread
            if (tid == 0) *fail = 1;
            return;
        }
        const T inv = piv_inv;
        for (int r = j + 1 + tid; r < nb; r += CHOL_DT) D[r][j] *= inv;
        __syncthreads();
        const int m = nb - j - 1;
        for (int e = tid; e < m * m; e += CHOL_DT) {
            const int r = j + 1 + e / m, c = j + 1 + e % m;
            if (c <= r) D[r][c] -= D[r][j] * D[c][j];
        }
        __syncthreads();
    }
    for (int t = tid; t < CHOL_NB * CHOL_NB; t += CHOL_DT) {
        const int r = t / CHOL_NB, c = t % CHOL_NB;
        if (r < nb && c <= r) M[(size_t)(jb + r) * n + jb + c] = D[r][c];
    }
    __shared__ T rdiag[CHOL_NB];
    if (tid < nb) rdiag[tid] = T(1) / D[tid][tid];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const T rj = rdiag[j];
        for (int c = tid; c <= j; c += CHOL_DT) X[j][c] *= rj;
        __syncthreads();
        const int m = nb - j - 1;
        for (int e = tid; e < m * (j + 1); e += CHOL_DT) {
            const int r = j + 1 + e / (j + 1), c = e % (j + 1);
            X[r][c] -= D[r][j] * X[j][c];
        }
        __syncthreads();
    }
    for (int t = tid; t < CHOL_NB * CHOL_NB; t += CHOL_DT) Li[t] = X[t / CHOL_NB][t % CHOL_NB];
}

// The FP32 diagonal block on one warp, with no block barrier: lane r keeps row r of the block in
// registers (rows beyond nb are identity rows, which factor trivially).  Column j's pivot a_jj is
// broadcast from lane j by a shuffle and each later column c receives l_cj from lane c the same
// way; then Li = L11^{-1} right-looking in the same form (lane r keeps row r of X).  Shared memory
// only stages the coalesced loads and stores.
__global__ void __launch_bounds__(32) k_chol_diag_warp(int n, int jb, float* M, float* Li, int* fail) {
    __shared__ float T[CHOL_NB][CHOL_NB + 1];
    if (*(volatile int*)fail) return;
    const unsigned FULL = 0xffffffffu;
    const int r = threadIdx.x;
    const int nb = min(CHOL_NB, n - jb);
    {
        float v[CHOL_NB];                                       // all 32 loads in flight
#pragma unroll
        for (int q = 0; q < CHOL_NB; ++q) v[q] = (q < nb && r <= q) ? M[(size_t)(jb + q) * n + jb + r] : 0.f;
#pragma unroll
        for (int q = 0; q < CHOL_NB; ++q) T[q][r] = v[q];       // coalesced: row q, column r
    }
    __syncwarp();
    float a[CHOL_NB];
#pragma unroll
    for (int c = 0; c < CHOL_NB; ++c) a[c] = r < nb ? (c <= r ? T[r][c] : 0.f) : (c == r ? 1.f : 0.f);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < CHOL_NB; ++j) {
        const float d = __shfl_sync(FULL, a[j], j);            // a_jj, the same in every lane
        bad = bad || !(d > 0.f) || !isfinite(d);
        const float ljj = sqrtf(d);
        if (r == j) a[j] = ljj;
        if (r > j) a[j] *= 1.f / ljj;                          // l_rj
#pragma unroll
        for (int c = j + 1; c < CHOL_NB; ++c) {
            const float lcj = __shfl_sync(FULL, a[j], c);
            if (r >= c) a[c] -= a[j] * lcj;
        }
    }
    if (bad) {                                                  // the same in every lane
        if (r == 0) *fail = 1;
        return;
    }
    float x[CHOL_NB];
#pragma unroll
    for (int c = 0; c < CHOL_NB; ++c) x[c] = c == r ? 1.f : 0.f;
#pragma unroll
    for (int j = 0; j < CHOL_NB; ++j) {
        const float rj = 1.f / __shfl_sync(FULL, a[j], j);     // 1 / l_jj
        if (r == j)
#pragma unroll
            for (int c = 0; c <= j; ++c) x[c] *= rj;
#pragma unroll
        for (int c = 0; c <= j; ++c) {
            const float xjc = __shfl_sync(FULL, x[c], j);
            if (r > j) x[c] -= a[j] * xjc;
        }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < CHOL_NB; ++c) T[r][c] = (r < nb && c <= r) ? a[c] : 0.f;
    __syncwarp();
    for (int q = 0; q < nb; ++q)
        if (r <= q) M[(size_t)(jb + q) * n + jb + r] = T[q][r];
    __syncwarp();
#pragma unroll
    for (int c = 0; c < CHOL_NB; ++c) T[r][c] = (r < nb && c <= r) ? x[c] : 0.f;
    __syncwarp();
    for (int q = 0; q < CHOL_NB; ++q) Li[q * CHOL_NB + r] = T[q][r];
}

// Rows i >= jb + nb of the panel: l_i = a_i L11^{-T} = a_i Li^T, a tile product (16 rows x 32
// columns per block of 128 threads; each thread 4 columns of one row).
template <class T>
__device__ __forceinline__ void chol_trsm_block(int n, int jb, T* M, const T* Li, int bx, T (*As)[CHOL_NB + 1],
                                                T (*Ls)[CHOL_NB + 1]) {
    const int nb = min(CHOL_NB, n - jb);
    const int i0 = jb + nb + bx * 16;
    for (int t = threadIdx.x; t < 16 * CHOL_NB; t += 128) {
        const int r = t / CHOL_NB, c = t % CHOL_NB;
        As[r][c] = (i0 + r < n && c < nb) ? M[(size_t)(i0 + r) * n + jb + c] : T(0);
    }
    for (int t = threadIdx.x; t < CHOL_NB * CHOL_NB; t += 128) Ls[t / CHOL_NB][t % CHOL_NB] = Li[t];
    __syncthreads();
    const int row = threadIdx.x / 8, c0 = (threadIdx.x % 8) * 4;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int m = 0; m < CHOL_NB; ++m) {
        const T a = As[row][m];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += a * Ls[c0 + q][m];
    }
    const int i = i0 + row;
    if (i < n)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + q < nb) M[(size_t)i * n + jb + c0 + q] = acc[q];
}

// Tile products for the dense factorisation, the inverse and its refinement: one 256-thread block
// computes a 64 x 64 tile, each thread a 4 x 4 block of it, from 32-wide slices of the operands
// staged in shared memory.  FP64 issue bounds the FP64 instantiations on this part, so every FMA
// reads its operands from registers loaded once per slice.
constexpr int DT_T = 64;           // tile edge
constexpr int DT_K = 32;           // slice depth

// Loads rows [r0, r0 + 64) x columns [c0, c0 + 32) of a row-major matrix with leading dimension ld
// (zero outside rows < nr, columns < nc) into S[64][33] (row r, column c at S[r][c]).
// (256 threads, 8 elements each: the loads of a thread are all issued before the first store.)
constexpr int DT_PER = DT_T * DT_K / 256;

template <class T>
__device__ __forceinline__ void dt_fetch_rows(T (&v)[DT_PER], const T* M, int ld, int r0, int c0, int nr, int nc) {
#pragma unroll
    for (int q = 0; q < DT_PER; ++q) {
        const int t = threadIdx.x + q * 256, r = t / DT_K, c = t % DT_K;
        v[q] = (r0 + r < nr && c0 + c < nc) ? M[(size_t)(r0 + r) * ld + c0 + c] : T(0);
    }
}
template <class T>
__device__ __forceinline__ void dt_store_rows(T (*S)[DT_K + 1], const T (&v)[DT_PER]) {
#pragma unroll
    for (int q = 0; q < DT_PER; ++q) {
        const int t = threadIdx.x + q * 256;
        S[t / DT_K][t % DT_K] = v[q];
    }
}
template <class T>
__device__ __forceinline__ void dt_load_rows(T (*S)[DT_K + 1], const T* M, int ld, int r0, int c0, int nr, int nc) {
    T v[DT_PER];
    dt_fetch_rows<T>(v, M, ld, r0, c0, nr, nc);
    dt_store_rows<T>(S, v);
}

// Loads rows [k0, k0 + 32) x columns [c0, c0 + 64) into S[64][33] transposed (S[c][k]).
template <class T>
__device__ __forceinline__ void dt_fetch_cols(T (&v)[DT_PER], const T* M, int ld, int k0, int c0, int nk, int nc) {
#pragma unroll
    for (int q = 0; q < DT_PER; ++q) {
        const int t = threadIdx.x + q * 256, k = t / DT_T, c = t % DT_T;
        v[q] = (k0 + k < nk && c0 + c < nc) ? M[(size_t)(k0 + k) * ld + c0 + c] : T(0);
    }
}
template <class T>
__device__ __forceinline__ void dt_store_cols(T (*S)[DT_K + 1], const T (&v)[DT_PER]) {
#pragma unroll
    for (int q = 0; q < DT_PER; ++q) {
        const int t = threadIdx.x + q * 256;
        S[t % DT_T][t / DT_T] = v[q];
    }
}
template <class T>
__device__ __forceinline__ void dt_load_cols(T (*S)[DT_K + 1], const T* M, int ld, int k0, int c0, int nk, int nc) {
    T v[DT_PER];
    dt_fetch_cols<T>(v, M, ld, k0, c0, nk, nc);
    dt_store_cols<T>(S, v);
}

// acc[a][b] += sum_k X[ty * 4 + a][k] * Y[tx * 4 + b][k] over one slice.
template <class T>
__device__ __forceinline__ void dt_mac(const T (*X)[DT_K + 1], const T (*Y)[DT_K + 1], T (&acc)[4][4], int tx, int ty) {
#pragma unroll 4
    for (int k = 0; k < DT_K; ++k) {
        T xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = X[ty * 4 + a][k];
#pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Y[tx * 4 + b][k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += xa[a] * yb[b];
    }
}

// Trailing update of the lower triangle: a_ik -= sum_m l_im l_km over the panel columns
// [jb, jb + nb), for jb + nb <= k <= i; block (bi, bk) with bk <= bi covers a 64 x 64 tile.
template <class T>
__device__ __forceinline__ void chol_syrk_block(int n, int jb, T* M, int bi, int bk, T (*Li)[DT_K + 1],
                                                T (*Lk)[DT_K + 1]) {
    const int nb = min(CHOL_NB, n - jb);
    const int t0 = jb + nb;
    const int i0 = t0 + bi * DT_T, k0 = t0 + bk * DT_T;
    dt_load_rows<T>(Li, M, n, i0, jb, n, jb + nb);
    dt_load_rows<T>(Lk, M, n, k0, jb, n, jb + nb);
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    dt_mac<T>(Li, Lk, acc, tx, ty);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, k = k0 + tx * 4 + b;
            if (i < n && k <= i) M[(size_t)i * n + k] -= acc[a][b];
        }
}

// Inverse of the lower factor, W = L^{-1}, by row panels (a triangular solve L W = I): panel p's
// rows of W are Li = L_pp^{-1} times the panel's rows of the running right-hand side R (R = I to
// start, held in W), for columns j < e = the panel's end; W is lower triangular, so columns from e
// on stay zero.  A tile product: 32 rows x 16 columns per block of 128 threads, each thread 4 rows
// of one column.
template <class T>
__device__ __forceinline__ void trinv_panel_block(int n, int jb, const T* Li, T* W, int bx, T (*Rs)[17],
                                                  T (*Ls)[CHOL_NB + 1]) {
    const int nb = min(CHOL_NB, n - jb);
    const int e = jb + nb;
    const int j0 = bx * 16;
    for (int t = threadIdx.x; t < CHOL_NB * 16; t += 128) {
        const int r = t / 16, c = t % 16;
        Rs[r][c] = (r < nb && j0 + c < e) ? W[(size_t)(jb + r) * n + j0 + c] : T(0);
    }
    for (int t = threadIdx.x; t < CHOL_NB * CHOL_NB; t += 128) Ls[t / CHOL_NB][t % CHOL_NB] = Li[t];
    __syncthreads();
    const int col = threadIdx.x % 16, r0 = (threadIdx.x / 16) * 4;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int m = 0; m < CHOL_NB; ++m) {
        const T v = Rs[m][col];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += Ls[r0 + q][m] * v;
    }
    const int j = j0 + col;
    if (j < e)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (r0 + q < nb) W[(size_t)(jb + r0 + q) * n + j] = acc[q];
}

// Rows below panel p: R_ij -= sum_m l_i,jb+m w_jb+m,j for i >= e, j < e (e = the panel's end).
template <class T>
__device__ __forceinline__ void trinv_update_block(int n, int jb, const T* L, T* W, int bx, int by,
                                                   T (*Ls)[DT_K + 1], T (*Ws)[DT_K + 1]) {
    const int nb = min(CHOL_NB, n - jb);
    const int e = jb + nb;
    const int i0 = e + by * DT_T, j0 = bx * DT_T;
    dt_load_rows<T>(Ls, L, n, i0, jb, n, e);        // rows i, panel columns
    dt_load_cols<T>(Ws, W, n, jb, j0, e, e);        // panel rows of W, columns j < e (transposed)
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    dt_mac<T>(Ls, Ws, acc, tx, ty);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < n && j < e) W[(size_t)i * n + j] -= acc[a][b];
        }
}

// One launch per panel for its rows of L (blocks [0, nt), chol_trsm_block) and its rows of W (the
// other blocks, trinv_panel_block): both need only Li and the data before the panel, and they
// write disjoint arrays, so the factorisation and W = L^{-1} advance in the same chain of launches.
template <class T>
__global__ void __launch_bounds__(128) k_panel_rows(int n, int jb, T* M, const T* Li, T* W, int nt, const int* fail) {
    __shared__ T buf[CHOL_NB * (CHOL_NB + 1)];                  // As[16][33] or Rs[32][17]
    __shared__ T Ls[CHOL_NB][CHOL_NB + 1];
    if (*(volatile int*)fail) return;
    if ((int)blockIdx.x < nt)
        chol_trsm_block<T>(n, jb, M, Li, blockIdx.x, reinterpret_cast<T(*)[CHOL_NB + 1]>(buf), Ls);
    else
        trinv_panel_block<T>(n, jb, Li, W, blockIdx.x - nt, reinterpret_cast<T(*)[17]>(buf), Ls);
}

// One launch per panel for the trailing update of L's lower triangle (blocks [0, ns): the lower
// triangle of tiles, row-major) and the update of W's rows below the panel (the other blocks, wx
// tiles per row of tiles).  The trailing update writes columns from the panel's end on, the W update
// reads L only in the panel's columns.
template <class T>
__global__ void __launch_bounds__(256) k_panel_update(int n, int jb, T* M, T* W, int ns, int wx, const int* fail) {
    __shared__ T S0[DT_T][DT_K + 1], S1[DT_T][DT_K + 1];
    if (*(volatile int*)fail) return;
    const int b = blockIdx.x;
    if (b < ns) {
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
        chol_syrk_block<T>(n, jb, M, bi, b - bi * (bi + 1) / 2, S0, S1);
    } else {
        const int q = b - ns;
        trinv_update_block<T>(n, jb, M, W, q % wx, q / wx, S0, S1);
    }
}

// A^{-1} = W^T W, tile (bi, bj) with bj <= bi: x_ij = sum_k w_ki w_kj over k >= i0 (W is lower
// triangular), written at (i, j) and (j, i).  The k range of a tile is cut into pieces of LA_KS:
// one CTA per piece writes its partial tile to part[item], and k_lauum_sum adds a tile's pieces in
// order (deterministic).  Without the cut, the first row of tiles carried the whole k range on one
// SM.
constexpr int LA_KS = 256;

template <class T>
__global__ void __launch_bounds__(256) k_lauum_part(int n, const T* W, const int4* items, T* part, const int* fail) {
    __shared__ T Wi[DT_T][DT_K + 1], Wj[DT_T][DT_K + 1];
    if (*(volatile int*)fail) return;
    const int4 it = items[blockIdx.x];                        // bi, bj, k0, k1
    const int i0 = it.x * DT_T, j0 = it.y * DT_T;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int k0 = it.z; k0 < it.w; k0 += DT_K) {
        dt_load_cols<T>(Wi, W, n, k0, i0, it.w, n);
        dt_load_cols<T>(Wj, W, n, k0, j0, it.w, n);
        __syncthreads();
        dt_mac<T>(Wi, Wj, acc, tx, ty);
        __syncthreads();
    }
    T* o = part + (size_t)blockIdx.x * DT_T * DT_T;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) o[(ty * 4 + a) * DT_T + tx * 4 + b] = acc[a][b];
}

// Tile t: sum its pieces first[t] .. first[t] + cnt[t] - 1 in order.
template <class T>
__global__ void __launch_bounds__(256) k_lauum_sum(int n, const int4* items, const int* first, const int* cnt,
                                                    const T* part, T* X, const int* fail) {
    if (*(volatile int*)fail) return;
    const int f = first[blockIdx.x], c = cnt[blockIdx.x];
    const int4 it = items[f];
    const int i0 = it.x * DT_T, j0 = it.y * DT_T;
    for (int e = threadIdx.x; e < DT_T * DT_T; e += 256) {
        T v = part[(size_t)f * DT_T * DT_T + e];
        for (int q = 1; q < c; ++q) v += part[(size_t)(f + q) * DT_T * DT_T + e];
        const int i = i0 + e / DT_T, j = j0 + e % DT_T;
        if (i < n && j < n) {
            X[(size_t)i * n + j] = v;
            X[(size_t)j * n + i] = v;
        }
    }
}

template <class T>
__global__ void k_identity(int n, T* W) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    W[t] = i == j ? T(1) : T(0);
}

// Dense Cholesky inverse of the n x n SPD matrix in M (lower triangle read, L left there) into
// Ainv (full, symmetric).  *fail = 1 on a non-positive or non-finite pivot.
template <class T>
void dense_chol_inverse(int n, T* M, T* Ainv, int* fail, cudaStream_t s) {
    // the pieces of W^T W (host tables copied first: pageable copies return once staged)
    const int tiles_all = (n + DT_T - 1) / DT_T;
    std::vector<int4> items;
    std::vector<int> first, cnt;
    for (int bi = 0; bi < tiles_all; ++bi)
        for (int bj = 0; bj <= bi; ++bj) {
            first.push_back((int)items.size());
            for (int k0 = bi * DT_T; k0 < n; k0 += LA_KS) items.push_back(make_int4(bi, bj, k0, std::min(n, k0 + LA_KS)));
            cnt.push_back((int)items.size() - first.back());
        }
    Tmp<int4> ditems(items.size(), s);
    Tmp<int> dfirst(first.size(), s), dcnt(cnt.size(), s);
    Tmp<T> part(items.size() * DT_T * DT_T, s);
    h2d(ditems.get(), items.data(), items.size(), s);
    h2d(dfirst.get(), first.data(), first.size(), s);
    h2d(dcnt.get(), cnt.data(), cnt.size(), s);
    const int np = (n + CHOL_NB - 1) / CHOL_NB;
    Tmp<T> Li((size_t)np * CHOL_NB * CHOL_NB, s);               // L_pp^{-1} of every panel
    // W = L^{-1} in a scratch of its own, formed panel by panel with the factorisation; then
    // A^{-1} = W^T W
    Tmp<T> W((size_t)n * n, s);
    k_identity<T><<<(int)(((int64_t)n * n + TPB - 1) / TPB), TPB, 0, s>>>(n, W.get());
    for (int jb = 0; jb < n; jb += CHOL_NB) {
        const int nb = std::min(CHOL_NB, n - jb);
        const int e = jb + nb;
        T* li = Li.get() + (size_t)(jb / CHOL_NB) * CHOL_NB * CHOL_NB;
        if constexpr (std::is_same<T, float>::value) k_chol_diag_warp<<<1, 32, 0, s>>>(n, jb, M, li, fail);
        else k_chol_diag<T><<<1, CHOL_DT, 0, s>>>(n, jb, M, li, fail);
        const int below = n - e;
        const int nt = (below + 15) / 16;
        k_panel_rows<T><<<nt + (e + 15) / 16, 128, 0, s>>>(n, jb, M, li, W.get(), nt, fail);
        if (below > 0) {
            const int tiles = (below + DT_T - 1) / DT_T, ns = tiles * (tiles + 1) / 2;
            const int wx = (e + DT_T - 1) / DT_T;
            k_panel_update<T><<<ns + wx * tiles, 256, 0, s>>>(n, jb, M, W.get(), ns, wx, fail);
        }
    }
    k_lauum_part<T><<<(int)items.size(), 256, 0, s>>>(n, W.get(), ditems.get(), part.get(), fail);
    k_lauum_sum<T><<<(int)first.size(), 256, 0, s>>>(n, ditems.get(), dfirst.get(), dcnt.get(), part.get(), Ainv, fail);
    CPC_LAUNCH_CK();
}

// --------------------------------------------------------------------------------------------
// Refinement of an approximate inverse by Newton-Schulz steps (Schulz's iteration for the
// inverse): X <- X (2I - A_c X) = X + X E with E = I - A_c X, so E_new = E^2 in exact arithmetic.
// E is formed in FP64 from the sparse A_c and the FP64 X; the correction X E needs only the
// relative accuracy of E's size, so it is a tile product in FP32 (X and E rounded), added to X in
// FP64.  From the FP32 Cholesky inverse (max |E| about 1e-5 at kappa 6e5) two steps reach the FP64
// rounding level.  At most INV_STEPS steps; once max |E| <= INV_SKIP (the rounding level) the later
// kernels return at once, and the last max |E| formed decides (INV_TOL) whether X is kept.
// --------------------------------------------------------------------------------------------
constexpr int INV_STEPS = 3;
constexpr double INV_TOL = 1e-12;
constexpr double INV_SKIP = 1e-13;
constexpr int INV_ROWS = 4;             // rows of E per block of k_inv_resid

// max |E| of an earlier step (bits of a non-negative double) at the rounding level: stop refining
__device__ __forceinline__ bool inv_converged(const unsigned long long* e) {
    return e && __longlong_as_double((long long)*(volatile unsigned long long*)e) <= INV_SKIP;
}

template <class A, class B>
__global__ void k_convert(int64_t count, const A* x, B* y, const int* fail) {
    if (*(volatile int*)fail) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = B(x[t]);
}

// E = I - A_c X, rows [INV_ROWS blockIdx.y, + INV_ROWS), columns over the threads; E (if not null) is stored rounded
// to FP32.  The largest |E_ij| goes to *emax as the bits of a non-negative double (which order as
// unsigned integers); a NaN or an infinity counts as infinity.  Nothing is done if the previous
// step's max |E| (prev, may be null) had reached the rounding level.
__global__ void __launch_bounds__(256) k_inv_resid(int n, const int* ptr, const int* col, const double* val,
                                                   const double* X, float* E, unsigned long long* emax,
                                                   const unsigned long long* prev, const int* fail) {
    __shared__ double wmax[8];
    if (*(volatile int*)fail || inv_converged(prev)) return;
    const int j = blockIdx.x * 256 + threadIdx.x;
    double m = 0.0;
    for (int i = blockIdx.y * INV_ROWS; i < min(n, (int)(blockIdx.y + 1) * INV_ROWS) && j < n; ++i) {
        double e = i == j ? 1.0 : 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) e -= val[p] * X[(size_t)col[p] * n + j];
        if (E) E[(size_t)i * n + j] = (float)e;
        const double a = fabs(e);
        m = a <= DBL_MAX ? fmax(m, a) : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmax(m, wmax[w]);
        atomicMax(emax, (unsigned long long)__double_as_longlong(m));
    }
}

// X += Xf E as FP32 tiles (Xf = X rounded to FP32), with the sum in FP64; Xn receives the new X
// rounded to FP32 for the next step (a buffer of its own: other blocks still read Xf).  Nothing is
// done if this step's max |E| (emax) is at the rounding level.
__global__ void __launch_bounds__(256) k_inv_correct(int n, const float* Xf, const float* E, double* X, float* Xn,
                                                     const unsigned long long* emax, const int* fail) {
    __shared__ float Xs[DT_T][DT_K + 1], Es[DT_T][DT_K + 1];
    if (*(volatile int*)fail || inv_converged(emax)) return;
    const int i0 = blockIdx.y * DT_T, j0 = blockIdx.x * DT_T;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    float xv[DT_PER], ev[DT_PER];                              // the next slice, fetched during the products
    dt_fetch_rows<float>(xv, Xf, n, i0, 0, n, n);              // rows i, columns k
    dt_fetch_cols<float>(ev, E, n, 0, j0, n, n);               // rows k, columns j (transposed)
    for (int k0 = 0; k0 < n; k0 += DT_K) {
        dt_store_rows<float>(Xs, xv);
        dt_store_cols<float>(Es, ev);
        __syncthreads();
        if (k0 + DT_K < n) {
            dt_fetch_rows<float>(xv, Xf, n, i0, k0 + DT_K, n, n);
            dt_fetch_cols<float>(ev, E, n, k0 + DT_K, j0, n, n);
        }
        dt_mac<float>(Xs, Es, acc, tx, ty);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < n && j < n) {
                const double v = X[(size_t)i * n + j] + (double)acc[a][b];
                X[(size_t)i * n + j] = v;
                Xn[(size_t)i * n + j] = (float)v;
            }
        }
}

// X = A_c^{-1} from the FP32 Cholesky inverse and up to INV_STEPS Newton-Schulz steps.  *fail32 = 1
// if the FP32 factorisation broke down (the later kernels then do nothing); emax[k] = max |E| before
// step k, emax[INV_STEPS] after the last step (all zero-initialised by the caller; entries after
// the first at the rounding level stay 0).
void refined_inverse(const Csr& Ac, double* X, int* fail32, unsigned long long* emax, cudaStream_t s) {
    const int n = Ac.n;
    const size_t nn = (size_t)n * n;
    Tmp<float> Xa(nn, s), Xb(nn, s), E(nn, s);
    {
        Tmp<float> M(nn, s);
        CPC_CK(cudaMemsetAsync(M.get(), 0, sizeof(float) * nn, s));
        k_csr_to_dense<float><<<nblk(n), TPB, 0, s>>>(n, Ac.ptr.p, Ac.col.p, Ac.val.p, M.get());
        dense_chol_inverse<float>(n, M.get(), Xa.get(), fail32, s);
    }
    k_convert<float, double><<<(int)((nn + TPB - 1) / TPB), TPB, 0, s>>>((int64_t)nn, Xa.get(), X, fail32);
    float* xf = Xa.get();
    float* xn = Xb.get();
    const dim3 rgrid((n + 255) / 256, (n + INV_ROWS - 1) / INV_ROWS), tgrid((n + DT_T - 1) / DT_T, (n + DT_T - 1) / DT_T);
    for (int k = 0; k < INV_STEPS; ++k) {
        k_inv_resid<<<rgrid, 256, 0, s>>>(n, Ac.ptr.p, Ac.col.p, Ac.val.p, X, E.get(), emax + k,
                                          k ? emax + k - 1 : nullptr, fail32);
        k_inv_correct<<<tgrid, 256, 0, s>>>(n, xf, E.get(), X, xn, emax + k, fail32);
        std::swap(xf, xn);
    }
    k_inv_resid<<<rgrid, 256, 0, s>>>(n, Ac.ptr.p, Ac.col.p, Ac.val.p, X, nullptr, emax + INV_STEPS,
                                      emax + INV_STEPS - 1, fail32);
    CPC_LAUNCH_CK();
}

// The residual the refinement ended with: the first max |E| at the rounding level, else the last.
double refined_residual(const unsigned long long* emax_host) {
    double e = 0.0;
    for (int k = 0; k <= INV_STEPS; ++k) {
        std::memcpy(&e, &emax_host[k], sizeof e);
        if (e <= INV_SKIP) return e;
    }
    return e;
}

// ============================================================================================
// Host orchestration
// ============================================================================================
void copy_csr_in(const cpc_csr& in, Csr& A, cudaStream_t s) {
    A.n = A.m = in.n;
    A.nnz = in.nnz;
    A.ptr.alloc(in.n + 1);
    A.col.alloc(in.nnz);
    A.val.alloc(in.nnz);
    const cudaMemcpyKind kind = in.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CPC_CK(cudaMemcpyAsync(A.ptr.p, in.rowptr, sizeof(int) * (in.n + 1), kind, s));
    CPC_CK(cudaMemcpyAsync(A.col.p, in.colidx, sizeof(int) * in.nnz, kind, s));
    CPC_CK(cudaMemcpyAsync(A.val.p, in.vals, sizeof(double) * in.nnz, kind, s));
}

// Level DAG (lower or upper) -> levels per row; returns the number of levels.
int dag_levels(const Csr& A, bool upper, int* lvl, cudaStream_t s) {
    const int n = A.n;
    k_fill_int<<<nblk(n), TPB, 0, s>>>(lvl, n, -1);
    Tmp<int> cnt(1, s);
    CPC_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int), s));
    int round = 0;
    for (;;) {
        for (int k = 0; k < 16; ++k, ++round)
            k_dag_round<<<nblk(n), TPB, 0, s>>>(n, A.ptr.p, A.col.p, lvl, round, upper ? 1 : 0, cnt.get());
        CPC_LAUNCH_CK();
        const int done = d2h(cnt.get(), s);
        if (done == n) break;
        if (round > n + 16) fail(CPC_EINVAL, "triangular dependency graph has a cycle");
    }
    // number of levels = max level + 1
    size_t tmp = 0;
    Tmp<int> mx(1, s);
    CPC_CK(cub::DeviceReduce::Max(nullptr, tmp, lvl, mx.get(), n, s));
    Tmp<char> t(tmp, s);
    CPC_CK(cub::DeviceReduce::Max(t.get(), tmp, lvl, mx.get(), n, s));
    return d2h(mx.get(), s) + 1;
}

void setup_ic0(Handle& h, cudaStream_t s) {
    Csr& A = h.Aic;
    const int n = A.n;
    h.lu.alloc(A.nnz);
    CPC_CK(cudaMemcpyAsync(h.lu.p, A.val.p, sizeof(double) * A.nnz, cudaMemcpyDeviceToDevice, s));
    h.lu_diag.alloc(n);
    {
        Tmp<int> bad(1, s);
        CPC_CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
        k_validate<<<nblk(n), TPB, 0, s>>>(n, A.ptr.p, A.col.p, (int)A.nnz, bad.get(), h.lu_diag.p);
        if (d2h(bad.get(), s)) fail(CPC_EINVAL, "invalid CSR for the IC(0) ordering");
    }
    // forward levels, factorisation level by level
    Tmp<int> lvl(n, s);
    h.ic_levels_L = dag_levels(A, false, lvl.get(), s);
    DBuf<int> slotsL, rowsL;
    int nslotsL = 0;
    std::vector<int> segL;
    grouped_slots(n, lvl.get(), h.ic_levels_L, CHUNK, s, slotsL, nslotsL, segL, &rowsL);
    // level g has rows rowsL[gstart..], count from segments: recompute counts from the slot layout
    std::vector<int> hc(h.ic_levels_L);
    {
        Tmp<int> cnt(h.ic_levels_L, s);
        CPC_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int) * h.ic_levels_L, s));
        k_group_count<<<nblk(n), TPB, 0, s>>>(n, lvl.get(), cnt.get());
        CPC_CK(cudaMemcpyAsync(hc.data(), cnt.get(), sizeof(int) * h.ic_levels_L, cudaMemcpyDeviceToHost, s));
        CPC_CK(cudaStreamSynchronize(s));
    }
    h.ic_rows_L1 = h.ic_levels_L > 1 ? hc[1] : 0;
    Tmp<int> failrow(1, s);
    k_fill_int<<<1, 1, 0, s>>>(failrow.get(), 1, INT_MAX);
    // rows of more than 64 entries are eliminated by a warp each
    int most = 0;
    {
        Tmp<int> mx(1, s);
        CPC_CK(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
        k_max_rowlen<<<nblk(n), TPB, 0, s>>>(n, A.ptr.p, mx.get());
        CPC_LAUNCH_CK();
        most = d2h(mx.get(), s);
    }
    const bool long_rows = most > 64;
    int off = 0;
    for (int g = 0; g < h.ic_levels_L; ++g) {
        if (long_rows) {
            k_ic0_level_warp<<<nblk(hc[g], IC_WARPS), IC_WARPS * 32, 0, s>>>(rowsL.p + off, hc[g], A.ptr.p, A.col.p,
                                                                             h.lu_diag.p, h.lu.p, failrow.get());
            if (most > IC_WROW)
                k_ic0_level<<<nblk(hc[g], 128), 128, 0, s>>>(rowsL.p + off, hc[g], A.ptr.p, A.col.p, h.lu_diag.p,
                                                              h.lu.p, failrow.get(), IC_WROW + 1);
        } else {
            k_ic0_level<<<nblk(hc[g], 128), 128, 0, s>>>(rowsL.p + off, hc[g], A.ptr.p, A.col.p, h.lu_diag.p, h.lu.p,
                                                          failrow.get(), 0);
        }
        off += hc[g];
    }
    CPC_LAUNCH_CK();
    const int fr = d2h(failrow.get(), s);
    if (fr != INT_MAX) fail(CPC_EFACTOR, "IC(0) pivot not positive at row " + std::to_string(fr));
    // triangular-solve layouts: L by forward levels, U by backward levels; rows/cols renamed to the
    // original numbering when the IC ordering is a permutation
    const int* imap = h.ic_order.p;
    build_sell(A.ptr.p, A.col.p, h.lu.p, slotsL, nslotsL, segL, CHUNK, SELL_LOWER, false, imap, h.L, s);
    h.ic_levels_U = dag_levels(A, true, lvl.get(), s);
    // backward solve processes levels of the upper DAG in ascending order
    DBuf<int> slotsU;
    int nslotsU = 0;
    std::vector<int> segU;
    grouped_slots(n, lvl.get(), h.ic_levels_U, CHUNK, s, slotsU, nslotsU, segU);
    build_sell(A.ptr.p, A.col.p, h.lu.p, slotsU, nslotsU, segU, CHUNK, SELL_UPPER, true, imap, h.U, s);
    CPC_CK(cudaStreamSynchronize(s));
}

__global__ void k_count_eq(int n, const int* a, int v, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && a[i] == v) atomicAdd(cnt, 1);
}

// Red-black IC(0) in B_co.  With the IC order = (fine colour, index) of a 2-colouring, red rows
// (colour 0, first) have no entries in L and black rows none in U.  Black rows with at least one
// neighbour form the second forward level; when that is every black row, step (2) of B_co reduces
// to one pass over them: z_b += (t_b - sum_{j red} l_bj t_j) / u_bb.  The red rows' backward step
// is left out: step (3) starts with a Gauss-Seidel step on the red rows, which overwrites z there
// without reading it.
void setup_ic_rb(Handle& h, bool colour_ic, cudaStream_t s) {
    h.ic_rb = false;
    if (!colour_ic || h.lev.size() < 2 || h.lev[0].ncolours != 2 || h.ic_levels_L != 2 || h.ic_levels_U != 2) return;
    const Level& L0 = h.lev[0];
    Tmp<int> cnt(1, s);
    CPC_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int), s));
    k_count_eq<<<nblk(L0.n), TPB, 0, s>>>(L0.n, L0.colour.p, 1, cnt.get());
    const int black = d2h(cnt.get(), s);
    if (black != h.ic_rows_L1) return;
    h.ic_black_c0 = h.L.seg[1];
    h.ic_black_c1 = h.L.seg[2];
    if (h.opt.precision == CPC_PREC_FP64) {
        h.ic_uinv64.alloc(h.n);
        k_slot_to_nat<<<nblk(h.U.nslots), TPB, 0, s>>>(h.U.nslots, h.U.perm.p, h.U.dinv.p, h.ic_uinv64.p);
    } else {
        h.ic_uinv32.alloc(h.n);
        k_slot_to_nat<<<nblk(h.U.nslots), TPB, 0, s>>>(h.U.nslots, h.U.perm.p, h.U.dinv32.p, h.ic_uinv32.p);
    }
    CPC_LAUNCH_CK();
    CPC_CK(cudaStreamSynchronize(s));
    h.ic_rb = true;
}

// Chunk-height autotuning: with tune, the colour-grouped copy of A_l is also built with C/2 and 2C
// (within 4..32) around the row-length rule, each is timed on a forward Gauss-Seidel sweep replayed
// from a graph (time_gs_sweep), and a candidate replaces the rule's layout only when it is more
// than 3% faster.  C sets the threads per row (32 / C) of every kernel on that copy.
void setup_level_sells(Level& L, cudaStream_t s, bool last, bool tune) {
    // colour-grouped A_l (Gauss-Seidel and residual)
    if (!last) {
        auto build_grouped = [&](int C, Sell& out) {
            DBuf<int> slots;
            int nslots = 0;
            std::vector<int> seg;
            grouped_slots(L.n, L.colour.p, L.ncolours, C, s, slots, nslots, seg);
            build_sell(L.A.ptr.p, L.A.col.p, L.A.val.p, slots, nslots, seg, C, SELL_OFFDIAG, true, nullptr, out, s);
            CPC_CK(cudaStreamSynchronize(s));
        };
        const int ca = choose_chunk((double)(L.A.nnz - L.n) / std::max(1, L.n));
        build_grouped(ca, L.S);
        if (!tune && ca < 32) {
            // One wave: a colour step whose CTAs do not all fit on the GPU at once runs in two
            // waves, and only the first wave's matrix loads overlap the previous step.  If the
            // widest colour needs more CTAs than fit and twice the chunk height (half the lanes
            // per row, about twice the entries per lane) would fit, take twice the chunk height.
            int widest = 0;
            for (size_t c = 0; c + 1 < L.S.seg.size(); ++c) widest = std::max(widest, L.S.seg[c + 1] - L.S.seg[c]);
            const int blocks = (widest + GS_WARPS_PER_BLOCK - 1) / GS_WARPS_PER_BLOCK;
            const int blocks2 = (widest / 2 + GS_WARPS_PER_BLOCK) / GS_WARPS_PER_BLOCK;
            if (blocks > gs_resident_blocks(L.S.lanes) && blocks2 <= gs_resident_blocks(16)) build_grouped(2 * ca, L.S);
        }
        if (tune) {
            float best = time_gs_sweep(L.S, L.n);
            for (int C : {ca / 2, ca * 2}) {
                if (C < 4 || C > 32) continue;
                Sell cand;
                build_grouped(C, cand);
                const float t = time_gs_sweep(cand, L.n);
                if (t < 0.97f * best) {
                    best = t;
                    L.S = std::move(cand);
                }
            }
        }
        DBuf<int> ps;
        int pn = 0;
        std::vector<int> pseg;
        const int cp = choose_chunk((double)L.P.nnz / std::max(1, L.P.n));
        natural_slots(L.P.n, cp, s, ps, pn, pseg);
        build_sell(L.P.ptr.p, L.P.col.p, L.P.val.p, ps, pn, pseg, cp, SELL_ALL, false, nullptr, L.SP, s);
        DBuf<int> rs;
        int rn = 0;
        std::vector<int> rseg;
        const int cr = choose_chunk((double)L.R.nnz / std::max(1, L.R.n));
        natural_slots(L.R.n, cr, s, rs, rn, rseg);
        build_sell(L.R.ptr.p, L.R.col.p, L.R.val.p, rs, rn, rseg, cr, SELL_ALL, false, nullptr, L.SR, s);
        CPC_CK(cudaStreamSynchronize(s));
    }
}

// Natural-order Gauss-Seidel ("standard GS", Section 3.3): the group of row i is its wavefront in the
// lower-triangular dependency graph of A_l, w(i) = 1 + max w(j) over j < i with a_ij != 0 (0 when
// there is none).  Rows of one wavefront are not coupled, and the pattern is symmetric, so every
// coupled j > i lies in a later wavefront.  Ascending wavefronts therefore reproduce the sequential
// forward sweep i = 0, ..., n-1 exactly, and descending wavefronts the backward sweep.
void wavefront_levels(Handle& h, cudaStream_t s) {
    const int nl = (int)h.lev.size();
    for (int l = 0; l + 1 < nl; ++l) {
        Level& L = h.lev[l];
        L.colour.alloc(L.n);
        L.ncolours = dag_levels(L.A, false, L.colour.p, s);
    }
}

// Smoothing colours of levels [0, nl - 1): the breadth-first parity 2-colouring if the pattern
// graph is bipartite, else Jones-Plassmann with peel-round priority; all levels in one cooperative
// launch of k_colour.
void colour_levels(Handle& h, cudaStream_t s) {
    const int nl = (int)h.lev.size();
    if (nl < 2) return;
    const int nj = nl - 1;
    if (nj > COL_MAXL) fail(CPC_ESETUP, "too many levels to colour");
    int64_t tot = 0;
    for (int l = 0; l < nj; ++l) tot += h.lev[l].n;
    Tmp<int> work((size_t)5 * tot, s), scal((size_t)COL_NS * nj, s), err(1, s);
    Tmp<unsigned long long> bar(1, s);
    Tmp<ColLev> dlev(nj, s);
    std::vector<ColLev> hl(nj);
    std::vector<int> hs((size_t)COL_NS * nj, 0);
    int64_t off = 0;
    for (int l = 0; l < nj; ++l) {
        Level& L = h.lev[l];
        L.colour.alloc(L.n);
        ColLev& V = hl[l];
        V.n = L.n;
        V.ptr = L.A.ptr.p;
        V.col = L.A.col.p;
        V.colour = L.colour.p;
        V.deg = work.get() + off;
        V.dec = V.deg + L.n;
        V.rnd = V.dec + L.n;
        V.blk = V.rnd + L.n;
        V.w = (unsigned*)(V.blk + L.n);
        V.scal = scal.get() + (size_t)COL_NS * l;
        off += (int64_t)5 * L.n;
        hs[(size_t)COL_NS * l + CS_DMIN] = INT_MAX;
        hs[(size_t)COL_NS * l + CS_DMIN + 1] = INT_MAX;
    }
    CPC_CK(cudaMemcpyAsync(dlev.get(), hl.data(), sizeof(ColLev) * nj, cudaMemcpyHostToDevice, s));
    CPC_CK(cudaMemcpyAsync(scal.get(), hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, s));
    CPC_CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    CPC_CK(cudaMemsetAsync(bar.get(), 0, sizeof(unsigned long long), s));
    int dev = 0, sms = 0, per_sm = 0;
    CPC_CK(cudaGetDevice(&dev));
    CPC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CPC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colour, COL_TPB, 0));
    if (per_sm < 1) fail(CPC_ESETUP, "colouring kernel does not fit on an SM");
    // every CTA that fits, one thread per point at most, at least one CTA per level
    const int grid = (int)std::max<int64_t>(nj, std::min<int64_t>((int64_t)per_sm * sms, nblk(tot, COL_TPB)));
    const ColLev* pl = dlev.get();
    int nn = nj;
    unsigned long long* pbar = bar.get();
    int* perr = err.get();
    void* args[] = {(void*)&pl, &nn, &pbar, &perr};
    CPC_CK(cudaLaunchCooperativeKernel((void*)k_colour, grid, COL_TPB, args, 0, s));
    CPC_LAUNCH_CK();
    const int e = d2h(err.get(), s);
    if (e == 1) fail(CPC_ESETUP, "colouring: a grid barrier gave up");
    if (e == 2) fail(CPC_ESETUP, "peel rounds did not terminate");
    if (e == 3) fail(CPC_ESETUP, "colouring did not terminate");
    if (e == 4) fail(CPC_ESETUP, "colouring: a union-find join did not complete");
    Tmp<int> mx(nj, s);
    CPC_CK(cudaMemsetAsync(mx.get(), 0, sizeof(int) * nj, s));
    for (int l = 0; l < nj; ++l) k_max_int<<<nblk(h.lev[l].n), TPB, 0, s>>>(h.lev[l].colour.p, h.lev[l].n, mx.get() + l);
    CPC_LAUNCH_CK();
    std::vector<int> hm(nj);
    CPC_CK(cudaMemcpyAsync(hm.data(), mx.get(), sizeof(int) * nj, cudaMemcpyDeviceToHost, s));
    CPC_CK(cudaStreamSynchronize(s));
    for (int l = 0; l < nj; ++l) h.lev[l].ncolours = hm[l] + 1;
}

// One coarsening step on level l; returns false when l becomes the coarsest level.
bool coarsen(Handle& h, int l, cudaStream_t s) {
    Level& L = h.lev[l];
    const int n = L.n;
    const int64_t nnz = L.A.nnz;
    Tmp<int> tpos(nnz, s), cnt(n, s), bad(1, s);
    Tmp<uint8_t> strong(nnz, s), sel(n, s);
    Tmp<int8_t> st(n, s);
    CPC_CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_transpose_pos<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, tpos.get(), bad.get());
    if (d2h(bad.get(), s)) fail(CPC_EINVAL, "matrix is not structurally symmetric");
    k_strength<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, L.A.val.p, h.opt.theta, strong.get());
    k_st_count<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, tpos.get(), strong.get(), cnt.get());
    k_pmis_init<<<nblk(n), TPB, 0, s>>>(n, cnt.get(), st.get());
    Tmp<int> undec(1, s);
    // rounds in batches of 4 per read-back of the undecided count (the last round's): rounds after
    // every point is decided change nothing
    for (int round = 0;; round += 4) {
        for (int k = 0; k < 4; ++k) {
            k_pmis_select<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, tpos.get(), strong.get(), cnt.get(),
                                                  st.get(), sel.get());
            k_pmis_setc<<<nblk(n), TPB, 0, s>>>(n, sel.get(), st.get());
            CPC_CK(cudaMemsetAsync(undec.get(), 0, sizeof(int), s));
            k_pmis_setf<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, strong.get(), st.get(), undec.get());
        }
        CPC_LAUNCH_CK();
        if (d2h(undec.get(), s) == 0) break;
        if (round > n) fail(CPC_ESETUP, "PMIS did not terminate");
    }
    L.cf.alloc(n);
    k_cf_flags<<<nblk(n), TPB, 0, s>>>(n, st.get(), L.cf.p);
    Tmp<int> cidx(n + 1, s), ccnt(n + 1, s);
    CPC_CK(cudaMemsetAsync(ccnt.get() + n, 0, sizeof(int), s));
    CPC_CK(cudaMemcpyAsync(ccnt.get(), L.cf.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    exclusive_scan(ccnt.get(), cidx.get(), n + 1, s);
    const int nc = d2h(cidx.get() + n, s);
    if (nc == 0 || nc == n) {
        L.cf.release();
        return false;
    }
    // interpolation
    Csr& P = L.P;
    P.n = n; P.m = nc;
    Tmp<int> pcnt(n + 1, s);
    k_interp_count<<<nblk(n + 1), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, strong.get(), L.cf.p, pcnt.get());
    P.ptr.alloc(n + 1);
    exclusive_scan(pcnt.get(), P.ptr.p, n + 1, s);
    P.nnz = d2h(P.ptr.p + n, s);
    P.col.alloc(P.nnz);
    P.val.alloc(P.nnz);
    k_interp_fill<<<nblk(n), TPB, 0, s>>>(n, L.A.ptr.p, L.A.col.p, L.A.val.p, strong.get(), L.cf.p, cidx.get(),
                                          P.ptr.p, P.col.p, P.val.p);
    CPC_LAUNCH_CK();
    transpose(P, L.R, s);
    // Galerkin coarse operator A_c = R (A P)
    Csr AP;
    spgemm(L.A, P, AP, s);
    h.lev.emplace_back();
    Level& Lc = h.lev.back();
    spgemm(h.lev[l].R, AP, Lc.A, s);
    Lc.n = Lc.A.n;
    Lc.A.m = Lc.A.n;
    Lc.nnz = Lc.A.nnz;
    CPC_CK(cudaStreamSynchronize(s));
    return true;
}

}  // namespace

// ============================================================================================
void tpfa_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask, int* rowptr, int* col,
                   double* val, cudaStream_t s) {
    const int n = nx * ny * nz;
    Tmp<int> len(n + 1, s);
    CPC_CK(cudaMemsetAsync(len.get() + n, 0, sizeof(int), s));
    k_tpfa_rowlen<<<nblk(n), TPB, 0, s>>>(nx, ny, nz, len.get());
    exclusive_scan(len.get(), rowptr, n + 1, s);
    k_tpfa_fill<<<nblk(n), TPB, 0, s>>>(nx, ny, nz, logk, kzr, dmask, rowptr, col, val);
    CPC_LAUNCH_CK();
}

void setup_handle(Handle& h, const cpc_csr& in) {
    cudaStream_t s = h.s;
    h.n = in.n;
    h.nnz = in.nnz;
    h.lev.clear();
    h.lev.emplace_back();
    {
        Level& L0 = h.lev[0];
        copy_csr_in(in, L0.A, s);
        L0.n = in.n;
        L0.nnz = in.nnz;
        Tmp<int> bad(1, s), diag(in.n, s);
        CPC_CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
        k_validate<<<nblk(in.n), TPB, 0, s>>>(in.n, L0.A.ptr.p, L0.A.col.p, in.nnz, bad.get(), diag.get());
        CPC_LAUNCH_CK();
        const int b = d2h(bad.get(), s);
        if (b & 1) fail(CPC_EINVAL, "invalid row pointers");
        if (b & 2) fail(CPC_EINVAL, "column index out of range or not ascending");
        if (b & 4) fail(CPC_EINVAL, "missing diagonal entry");
    }
    cudaEvent_t e0, e1, e2;
    CPC_CK(cudaEventCreate(&e0));
    CPC_CK(cudaEventCreate(&e1));
    CPC_CK(cudaEventCreate(&e2));
    struct EvGuard {
        cudaEvent_t a, b, c;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c); }
    } guard{e0, e1, e2};

    const bool colour_ic = h.opt.ic_order == 1;
    // natural-order IC(0) first (a breakdown is reported before any AMG work)
    CPC_CK(cudaEventRecord(e0, s));
    if (!colour_ic) {
        Level& L0 = h.lev[0];
        h.Aic.n = h.Aic.m = L0.n;
        h.Aic.nnz = L0.nnz;
        h.Aic.ptr.alloc(L0.n + 1);
        h.Aic.col.alloc(L0.nnz);
        h.Aic.val.alloc(L0.nnz);
        CPC_CK(cudaMemcpyAsync(h.Aic.ptr.p, L0.A.ptr.p, sizeof(int) * (L0.n + 1), cudaMemcpyDeviceToDevice, s));
        CPC_CK(cudaMemcpyAsync(h.Aic.col.p, L0.A.col.p, sizeof(int) * L0.nnz, cudaMemcpyDeviceToDevice, s));
        CPC_CK(cudaMemcpyAsync(h.Aic.val.p, L0.A.val.p, sizeof(double) * L0.nnz, cudaMemcpyDeviceToDevice, s));
        setup_ic0(h, s);
    }
    CPC_CK(cudaEventRecord(e1, s));
    // AMG hierarchy; phase boundaries are timed for cpc_setup_phases_ms
    cudaEvent_t ph[3];
    for (auto& e : ph) CPC_CK(cudaEventCreate(&e));
    struct PhGuard {
        cudaEvent_t* e;
        ~PhGuard() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); }
    } phguard{ph};
    for (int l = 0;; ++l) {
        const bool stop = h.lev[l].n <= h.opt.coarse_max || (int)h.lev.size() >= h.opt.max_levels;
        if (stop || !coarsen(h, l, s)) break;
    }
    CPC_CK(cudaEventRecord(ph[0], s));
    // The smoothing colours first, on the setup stream: one cooperative kernel at full occupancy
    // (measured: other kernels do not start beside a resident cooperative grid on this part, so
    // the coarsest inverse is not overlapped with it).  Then the coarsest inverse on a second
    // stream beside the layouts (ordinary kernels that share the GPU): the layouts need the colours,
    // the inverse only the coarsest operator.  The layouts' allocations still wait for the device
    // now and then, so the overlap is partial (measured: 49.7 -> 47 ms of AMG setup at 1M).
    const int nl = (int)h.lev.size();
    if (h.opt.gs_order == CPC_GS_NATURAL) wavefront_levels(h, s);
    else colour_levels(h, s);
    CPC_CK(cudaEventRecord(ph[1], s));
    cudaStream_t s2;
    CPC_CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    struct S2 {
        cudaStream_t q;
        ~S2() { cudaStreamSynchronize(q); cudaStreamDestroy(q); }
    } s2guard{s2};
    CPC_CK(cudaStreamWaitEvent(s2, ph[1], 0));
    Level& Lc = h.lev[nl - 1];
    h.nc = Lc.n;
    if (h.nc > DENSE_MAX) fail(CPC_ESETUP, "coarsest level too large for the dense solve");
    h.Ainv.alloc((size_t)h.nc * h.nc);
    // flags[0]: FP64 factorisation failure, flags[1]: FP32 factorisation failure
    Tmp<int> inv_fail(2, s2);
    Tmp<unsigned long long> emax(INV_STEPS + 2, s2);
    cudaEvent_t c0, c1;
    CPC_CK(cudaEventCreate(&c0));
    CPC_CK(cudaEventCreate(&c1));
    struct CGuard {
        cudaEvent_t a, b;
        ~CGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } cguard{c0, c1};
    CPC_CK(cudaEventRecord(c0, s2));
    CPC_CK(cudaMemsetAsync(inv_fail.get(), 0, 2 * sizeof(int), s2));
    CPC_CK(cudaMemsetAsync(emax.get(), 0, (INV_STEPS + 2) * sizeof(unsigned long long), s2));
    refined_inverse(Lc.A, h.Ainv.p, inv_fail.get() + 1, emax.get(), s2);
    CPC_CK(cudaEventRecord(c1, s2));
    // The layouts run beside the inverse on a stream of their own at the device's greatest
    // priority (at equal priority their kernels waited behind the inverse's grids in the block
    // scheduler: 11.4 against 4.5 ms at 1M), with their buffers allocated stream-ordered on it.
    cudaStream_t s3;
    {
        int prio_least = 0, prio_greatest = 0;
        CPC_CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
        CPC_CK(cudaStreamCreateWithPriority(&s3, cudaStreamNonBlocking, prio_greatest));
    }
    S2 s3guard{s3};
    CPC_CK(cudaStreamWaitEvent(s3, ph[1], 0));
    {
        AllocOn layouts_alloc(s3);
        for (int l = 0; l < nl; ++l) setup_level_sells(h.lev[l], s3, l == nl - 1, h.opt.autotune == 1 && l > 0);
        // fine A in natural order for the SpMVs
        DBuf<int> slots;
        int nslots = 0;
        std::vector<int> seg;
        natural_slots(h.n, CHUNK, s3, slots, nslots, seg);
        build_sell(h.lev[0].A.ptr.p, h.lev[0].A.col.p, h.lev[0].A.val.p, slots, nslots, seg, CHUNK, SELL_OFFDIAG,
                   true, nullptr, h.Anat, s3);
        build_dia(h.n, h.lev[0].A.ptr.p, h.lev[0].A.col.p, h.lev[0].A.val.p, h.Anat, s3);
        if (nl > 1) build_dia(h.n, h.lev[0].A.ptr.p, h.lev[0].A.col.p, h.lev[0].A.val.p, h.lev[0].S, s3, true);
        CPC_CK(cudaStreamSynchronize(s3));
    }
    CPC_CK(cudaEventRecord(ph[2], s3));                         // layouts done
    CPC_CK(cudaStreamWaitEvent(s, ph[2], 0));
    {   // keep the refined inverse if its residual reached INV_TOL, else the FP64 Cholesky inverse
        const int f32 = d2h(inv_fail.get() + 1, s2);
        unsigned long long eb[INV_STEPS + 1];
        CPC_CK(cudaMemcpyAsync(eb, emax.get(), sizeof eb, cudaMemcpyDeviceToHost, s2));
        CPC_CK(cudaStreamSynchronize(s2));
        const double e = refined_residual(eb);
        h.inv_method = 1;
        h.inv_resid = f32 ? INFINITY : e;
        if (f32 || !(e <= INV_TOL)) {
            h.inv_method = 0;
            {
                Tmp<double> M((size_t)h.nc * h.nc, s2);
                CPC_CK(cudaMemsetAsync(M.get(), 0, sizeof(double) * h.nc * h.nc, s2));
                k_csr_to_dense<double><<<nblk(h.nc), TPB, 0, s2>>>(h.nc, Lc.A.ptr.p, Lc.A.col.p, Lc.A.val.p, M.get());
                dense_chol_inverse<double>(h.nc, M.get(), h.Ainv.p, inv_fail.get(), s2);
            }
            k_inv_resid<<<dim3((h.nc + 255) / 256, (h.nc + INV_ROWS - 1) / INV_ROWS), 256, 0, s2>>>(
                h.nc, Lc.A.ptr.p, Lc.A.col.p, Lc.A.val.p, h.Ainv.p, nullptr, emax.get() + INV_STEPS + 1, nullptr,
                inv_fail.get());
            CPC_LAUNCH_CK();
            CPC_CK(cudaEventRecord(c1, s2));
            const unsigned long long eb64 = d2h(emax.get() + INV_STEPS + 1, s2);
            std::memcpy(&h.inv_resid, &eb64, sizeof(double));
        }
    }
    if (d2h(inv_fail.get(), s2)) fail(CPC_ESETUP, "coarsest operator is not positive definite");
    CPC_CK(cudaStreamWaitEvent(s, c1, 0));
    CPC_CK(cudaEventRecord(e2, s));
    if (colour_ic) {
        // IC(0) of the colour-ordered fine matrix: order = rows sorted by (colour, index)
        Level& L0 = h.lev[0];
        if (nl < 2) fail(CPC_EINVAL, "colour-ordered IC(0) needs at least two AMG levels");
        DBuf<int> rows;
        {
            DBuf<int> slots;
            int nslots = 0;
            std::vector<int> seg;
            grouped_slots(L0.n, L0.colour.p, L0.ncolours, CHUNK, s, slots, nslots, seg, &rows);
        }
        h.ic_order = std::move(rows);
        Tmp<int> inv(L0.n, s), len(L0.n + 1, s);
        k_inverse_perm<<<nblk(L0.n), TPB, 0, s>>>(L0.n, h.ic_order.p, inv.get());
        h.Aic.n = h.Aic.m = L0.n;
        h.Aic.nnz = L0.nnz;
        h.Aic.ptr.alloc(L0.n + 1);
        h.Aic.col.alloc(L0.nnz);
        h.Aic.val.alloc(L0.nnz);
        k_perm_rowlen<<<nblk(L0.n + 1), TPB, 0, s>>>(L0.n, L0.A.ptr.p, h.ic_order.p, len.get());
        exclusive_scan(len.get(), h.Aic.ptr.p, L0.n + 1, s);
        k_perm_fill<<<nblk(L0.n), TPB, 0, s>>>(L0.n, L0.A.ptr.p, L0.A.col.p, L0.A.val.p, h.ic_order.p, inv.get(),
                                               h.Aic.ptr.p, h.Aic.col.p, h.Aic.val.p);
        CPC_LAUNCH_CK();
        cudaEvent_t e3;
        CPC_CK(cudaEventCreate(&e3));
        CPC_CK(cudaEventRecord(e3, s));
        setup_ic0(h, s);
        cudaEvent_t e4;
        CPC_CK(cudaEventCreate(&e4));
        CPC_CK(cudaEventRecord(e4, s));
        CPC_CK(cudaEventSynchronize(e4));
        float a = 0.f;
        cudaEventElapsedTime(&a, e3, e4);
        cudaEventDestroy(e3);
        cudaEventDestroy(e4);
        h.ms_ic0 = a;
    }
    CPC_CK(cudaEventSynchronize(e2));
    float a = 0.f, b = 0.f;
    CPC_CK(cudaEventElapsedTime(&a, e0, e1));
    CPC_CK(cudaEventElapsedTime(&b, e1, e2));
    if (!colour_ic) h.ms_ic0 = a;
    h.ms_amg = b;
    {   // the coarsest inverse (own stream) overlaps the layouts: each is timed on its stream
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        CPC_CK(cudaEventElapsedTime(&t[0], e1, ph[0]));
        CPC_CK(cudaEventElapsedTime(&t[1], ph[0], ph[1]));
        CPC_CK(cudaEventElapsedTime(&t[2], c0, c1));
        CPC_CK(cudaEventElapsedTime(&t[3], ph[1], ph[2]));
        for (int i = 0; i < 4; ++i) h.ms_phase[i] = t[i];
    }

    // precision of the preconditioner data
    const int prec = h.opt.precision;
    for (int l = 0; l < nl; ++l) {
        Level& L = h.lev[l];
        L.vt = prec == CPC_PREC_FP64 ? VT_F64 : (prec == CPC_PREC_FP32_BF16 && l > 0 ? VT_BF16 : VT_F32);
        if (l < nl - 1) {
            sell_lowp(L.S, L.vt, s);
            sell_lowp(L.SP, L.vt == VT_BF16 ? VT_F32 : L.vt, s);
            sell_lowp(L.SR, L.vt == VT_BF16 ? VT_F32 : L.vt, s);
            if (L.vt == VT_F64) {
                L.dnat64.alloc(L.n);
                k_slot_to_nat<<<nblk(L.S.nslots), TPB, 0, s>>>(L.S.nslots, L.S.perm.p, L.S.dinv.p, L.dnat64.p);
            } else {
                L.dnat32.alloc(L.n);
                k_slot_to_nat<<<nblk(L.S.nslots), TPB, 0, s>>>(L.S.nslots, L.S.perm.p, L.S.dinv32.p, L.dnat32.p);
            }
            CPC_LAUNCH_CK();
        }
        const size_t n = L.n;
        if (L.vt == VT_F64) { L.x64.alloc(n); L.f64.alloc(n); L.r64.alloc(n); }
        else { L.x32.alloc(n); L.f32.alloc(n); L.r32.alloc(n); }
    }
    if (prec != CPC_PREC_FP64) {
        sell_lowp(h.Anat, VT_F32, s);
        sell_lowp(h.L, VT_F32, s);
        sell_lowp(h.U, VT_F32, s);
        h.Ainv32.alloc((size_t)h.nc * h.nc);
        k_to_f32<<<nblk((int64_t)h.nc * h.nc), TPB, 0, s>>>((int64_t)h.nc * h.nc, h.Ainv.p, h.Ainv32.p);
        h.z32.alloc(h.n); h.t32.alloc(h.n); h.y32.alloc(h.n);
    }
    setup_ic_rb(h, colour_ic, s);
    setup_tail(h, h.opt.tail_nnz_max);
    // PCG and preconditioner vectors
    const size_t n = h.n;
    h.b.alloc(n); h.x.alloc(n); h.r.alloc(n); h.z.alloc(n); h.p.alloc(n); h.q.alloc(n);
    h.t.alloc(n); h.y.alloc(n);
    h.partial.alloc(4 * NPART);
    h.counter.alloc(8);
    CPC_CK(cudaMemsetAsync(h.counter.p, 0, sizeof(unsigned) * 8, s));
    h.state.alloc(1);
    CPC_CK(cudaMemsetAsync(h.state.p, 0, sizeof(PcgState), s));
    h.hist.alloc(HIST_CAP);
    h.flags.alloc(8);
    CPC_CK(cudaMemsetAsync(h.flags.p, 0, sizeof(int) * 8, s));
    CPC_CK(cudaStreamSynchronize(s));
    CPC_LAUNCH_CK();
}

}  // namespace cpc
