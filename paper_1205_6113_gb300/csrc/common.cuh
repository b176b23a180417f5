// common.cuh -- internal types of the cpc library (device buffers, CSR, SELL-C, handle).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cpc.h"

namespace cpc {

// ---------------------------------------------------------------------------------------------
// Errors: internal code throws cpc::Error; every C entry point catches it and returns the code.
// ---------------------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

#define CPC_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw ::cpc::Error{CPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define CPC_LAUNCH_CK() CPC_CK(cudaGetLastError())

inline void fail(int code, const std::string& msg) { throw Error{code, msg}; }

// ---------------------------------------------------------------------------------------------
// Device buffer (owning, move-only).
// ---------------------------------------------------------------------------------------------
// Stream on which DBuf::alloc takes its memory while an AllocOn scope is open (this thread only).
// cudaMalloc and cudaFree can wait for the work queued on the whole device, so a setup phase that
// runs beside another stream's kernels allocates stream-ordered instead, from the device's default
// pool.  The buffer is owned like any other: released inside the scope with cudaFreeAsync on that
// stream, after it with cudaFree (which accepts pool memory).  Code that uses a buffer on a stream
// of its own opens AllocOn(nullptr).
inline cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}
struct AllocOn {
    cudaStream_t prev;
    explicit AllocOn(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocOn() { alloc_stream() = prev; }
    AllocOn(const AllocOn&) = delete;
    AllocOn& operator=(const AllocOn&) = delete;
};

// alloc_async: a stream-ordered buffer for setup temporaries, freed on the same stream, so that its
// release does not wait for the whole device as cudaFree does; the stream must outlive it.
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t fs = nullptr;              // stream of a stream-ordered buffer
    bool pooled = false;                    // taken from the pool inside an AllocOn scope
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), fs(o.fs), pooled(o.pooled) {
        o.p = nullptr; o.n = 0; o.fs = nullptr; o.pooled = false;
    }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; fs = o.fs; pooled = o.pooled;
            o.p = nullptr; o.n = 0; o.fs = nullptr; o.pooled = false;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;          // keep a valid pointer for empty arrays
        if (cudaStream_t s = alloc_stream()) {
            CPC_CK(cudaMallocAsync(&p, count * sizeof(T), s));
            pooled = true;
        } else {
            CPC_CK(cudaMalloc(&p, count * sizeof(T)));
        }
        n = count;
    }
    void alloc_async(size_t count, cudaStream_t s) {
        release();
        if (count == 0) count = 1;
        CPC_CK(cudaMallocAsync(&p, count * sizeof(T), s));
        n = count;
        fs = s;
    }
    void release() {
        if (p) {
            if (fs) cudaFreeAsync(p, fs);
            else if (pooled && alloc_stream()) cudaFreeAsync(p, alloc_stream());
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
        fs = nullptr;
        pooled = false;
    }
    T* get() const { return p; }
};

// Stream-ordered temporary (setup scratch): freed on the stream when it goes out of scope.
template <class T>
struct Tmp {
    T* p = nullptr;
    cudaStream_t s = nullptr;
    Tmp(size_t count, cudaStream_t st) : s(st) {
        if (count == 0) count = 1;
        CPC_CK(cudaMallocAsync(&p, count * sizeof(T), s));
    }
    Tmp(const Tmp&) = delete;
    Tmp& operator=(const Tmp&) = delete;
    ~Tmp() { if (p) cudaFreeAsync(p, s); }
    T* get() const { return p; }
};

// Device CSR with FP64 values; n rows, m columns, columns ascending within a row.
struct Csr {
    int n = 0, m = 0;
    int64_t nnz = 0;
    DBuf<int> ptr, col;
    DBuf<double> val;
};

// Value storage types of the preconditioner data.
enum VType { VT_F64 = 0, VT_F32 = 1, VT_BF16 = 2 };

struct DiaOff {
    int o[8];
};

// SELL-C storage of a set of matrix rows in a chosen slot order (C in {32, 16, 8, 4}).
//   slot s holds row perm[s] (or -1 for padding); chunk k = slots [Ck, Ck+C) is processed by one
//   warp with G = 32/C lanes per row; entry w of the row in slot Ck + r lives at
//   val/col[cptr[k] + w*C + r], so that every warp-wide load covers 32 consecutive elements.
//   With split_diag the diagonal is kept apart in diag[s] and val/col hold off-diagonals only.
//   Padding entries have val 0 and col = -1; kernels skip them (no load is issued).
//   seg[] (host) gives chunk ranges: segment g is chunks [seg[g], seg[g+1]) -- a colour of a
//   Gauss-Seidel sweep or a level of a triangular solve.
struct Sell {
    int C = 32;                        // chunk height (rows per warp); 32 / C lanes share a row
    int nslots = 0, nchunks = 0;
    int64_t nelem = 0;
    int lanes = 0;                     // most entries one lane holds: ceil(widest chunk / 32)
    DBuf<int> perm, cptr, col;
    DBuf<double> val, diag, dinv;      // FP64 copy (always); dinv = 1 / diag (split diagonal only)
    DBuf<float> val32, diag32, dinv32; // FP32 copy (mixed precision)
    DBuf<__nv_bfloat16> val16;         // BF16 copy of off-diagonals (coarse levels, mode 2)
    std::vector<int> seg;
    // Diagonal storage (structured grids): when every off-diagonal entry lies on one of ndiag <= 8
    // offsets col - row (ascending, padded with 0), entry d of slot s is dval[d * nslots + s], 0 where
    // the row has no such entry.  Kernels for this form read no column indices and no chunk
    // pointers; the SELL arrays above are kept for the other kernels.
    int ndiag = 0;
    DiaOff doff{};
    DBuf<double> dval;
    DBuf<float> dval32;
    // Gauss-Seidel copy of the diagonal form (colour-grouped fine level): per slot the ndiag values
    // -a_ij / a_ii side by side, gval[s * ndiag + d], so that x_i = f_i / a_ii + sum_d g_d x_j.
    DBuf<double> gval;
    DBuf<float> gval32;
};

}  // namespace cpc
