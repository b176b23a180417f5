// noalloc.cu -- two-point-flux assembly that allocates no device memory.
//
// cpc_tpfa_assemble() obtains its scan scratch (row lengths and the prefix-sum temporaries) from
// the stream-ordered allocator.  Some callers cannot allow any allocation inside a library call:
// simulators that hand out all device memory from their own pool and forbid cudaMalloc /
// cudaMallocAsync after start-up, and real-time loops that cannot afford an allocation's implicit
// synchronisation.  For them, cpc_tpfa_assemble_noalloc() produces the same CSR using a scratch
// array that lives in the library image itself: a file-scope __device__ array of
// NA_MAX_BLOCKS ints (64 KiB), which every GPU that loads this library holds until the process
// exits.  The array stores one partial row count per block of NA_TPB cells, so the largest grid
// this entry point accepts is NA_TPB * NA_MAX_BLOCKS = 16,777,216 cells (for example 256^3).
//
// The array is shared by every call in the process and keeps the last call's contents.  Each
// call overwrites every entry it reads before reading it, so no clearing is needed, but calls
// whose work overlaps on the GPU (other streams, other host threads) race on it: order them.
#include <climits>
#include <mutex>

#include "../../include/cpc.h"

namespace {

constexpr int NA_TPB = 1024;                      // cells per block
constexpr int NA_MAX_BLOCKS = 16384;              // scratch entries
constexpr long long NA_MAX_CELLS = (long long)NA_TPB * NA_MAX_BLOCKS;
constexpr int NA_MAX_DEVICES = 64;

// Per-block row counts, then their exclusive prefix sums (the block's first row offset).
static __device__ __align__(256) int g_na_block_rows[NA_MAX_BLOCKS];

__device__ __forceinline__ int na_row_len(int c, int nx, int ny, int nz) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    return 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
}

// Exclusive prefix sum over the block (NA_TPB threads); *total receives the block's sum.
__device__ int na_block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[NA_TPB / 32];
    __shared__ int block_total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int s = warp_sums[lane];          // NA_TPB / 32 == 32 warps
        int si = s;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        warp_sums[lane] = si - s;
        if (lane == 31) block_total = si;
    }
    __syncthreads();
    const int out = warp_sums[w] + incl - v;
    *total = block_total;
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(NA_TPB) k_na_count(int nx, int ny, int nz, int* block_rows) {
    const int n = nx * ny * nz;
    const int c = blockIdx.x * NA_TPB + threadIdx.x;
    const int len = c < n ? na_row_len(c, nx, ny, nz) : 0;
    int total;
    na_block_exclusive_scan(len, &total);
    if (threadIdx.x == 0) block_rows[blockIdx.x] = total;
}

// One block: in-place exclusive scan of the per-block counts; writes rowptr[n] = nnz.
__global__ void __launch_bounds__(NA_TPB) k_na_scan(int nblocks, int* block_rows, int* rowptr, int n) {
    constexpr int PER = NA_MAX_BLOCKS / NA_TPB;   // 16 entries per thread
    const int base = threadIdx.x * PER;
    int local[PER];
    int sum = 0;
    for (int q = 0; q < PER; ++q) {
        const int idx = base + q;
        local[q] = idx < nblocks ? block_rows[idx] : 0;
        sum += local[q];
    }
    int total;
    int run = na_block_exclusive_scan(sum, &total);
    for (int q = 0; q < PER; ++q) {
        const int idx = base + q;
        if (idx < nblocks) block_rows[idx] = run;
        run += local[q];
    }
    if (threadIdx.x == 0) rowptr[n] = total;
}

__device__ __forceinline__ double na_harmonic(double a, double b) { return (2.0 * a * b) / (a + b); }

// Row offsets and entries of every cell.  Entry order per row: z-, y-, x-, diagonal, x+, y+, z+;
// the diagonal sums the neighbour transmissibilities in that order, then the Dirichlet half-cell
// terms in face order x0, x1, y0, y1, z0, z1 (Section 4, Eq. model with c = 0).
__global__ void __launch_bounds__(NA_TPB) k_na_fill(int nx, int ny, int nz, const double* logk, double kzr,
                                                      int dmask, const int* block_rows, int* rowptr, int* col,
                                                      double* val) {
    const int n = nx * ny * nz;
    const int c = blockIdx.x * NA_TPB + threadIdx.x;
    const int len = c < n ? na_row_len(c, nx, ny, nz) : 0;
    int total;
    const int off = na_block_exclusive_scan(len, &total) + block_rows[blockIdx.x];
    if (c >= n) return;
    rowptr[c] = off;
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const int sxy = nx * ny;
    const double kc = exp(logk[c]);
    const double kzc = kzr * kc;
    int nb[6];
    double t[6];
    int cnt = 0;
    if (k > 0)      { nb[cnt] = c - sxy; t[cnt++] = na_harmonic(kzc, kzr * exp(logk[c - sxy])); }
    if (j > 0)      { nb[cnt] = c - nx;  t[cnt++] = na_harmonic(kc, exp(logk[c - nx])); }
    if (i > 0)      { nb[cnt] = c - 1;   t[cnt++] = na_harmonic(kc, exp(logk[c - 1])); }
    const int nlow = cnt;
    if (i < nx - 1) { nb[cnt] = c + 1;   t[cnt++] = na_harmonic(kc, exp(logk[c + 1])); }
    if (j < ny - 1) { nb[cnt] = c + nx;  t[cnt++] = na_harmonic(kc, exp(logk[c + nx])); }
    if (k < nz - 1) { nb[cnt] = c + sxy; t[cnt++] = na_harmonic(kzc, kzr * exp(logk[c + sxy])); }
    double d = 0.0;
    for (int q = 0; q < cnt; ++q) d += t[q];
    if ((dmask & 1) && i == 0)       d += 2.0 * kc;
    if ((dmask & 2) && i == nx - 1)  d += 2.0 * kc;
    if ((dmask & 4) && j == 0)       d += 2.0 * kc;
    if ((dmask & 8) && j == ny - 1)  d += 2.0 * kc;
    if ((dmask & 16) && k == 0)      d += 2.0 * kzc;
    if ((dmask & 32) && k == nz - 1) d += 2.0 * kzc;
    int p = off;
    for (int q = 0; q < nlow; ++q) { col[p] = nb[q]; val[p] = -t[q]; ++p; }
    col[p] = c; val[p] = d; ++p;
    for (int q = nlow; q < cnt; ++q) { col[p] = nb[q]; val[p] = -t[q]; ++p; }
}

// Device address of the scratch array, looked up once per device (with that device current).
std::mutex g_na_mu;
int* g_na_addr[NA_MAX_DEVICES] = {};

int na_scratch(int** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return CPC_ECUDA;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        int* ptr = nullptr;
        if (cudaGetSymbolAddress((void**)&ptr, g_na_block_rows) != cudaSuccess || !ptr) return CPC_ECUDA;
        g_na_addr[dev] = ptr;
    }
    *out = g_na_addr[dev];
    return CPC_OK;
}

}  // namespace

extern "C" int cpc_tpfa_assemble_noalloc(int32_t nx, int32_t ny, int32_t nz, const double* logk,
                                         double kz_ratio, int32_t dirichlet_mask, int32_t* rowptr,
                                         int32_t* colidx, double* vals, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !logk || !rowptr || !colidx || !vals || !(kz_ratio > 0.0)) return CPC_EINVAL;
    const long long n = (long long)nx * ny * nz;
    if (n > NA_MAX_CELLS) return CPC_EINVAL;      // beyond the scratch array's capacity
    const long long faces = (long long)(nx - 1) * ny * nz + (long long)nx * (ny - 1) * nz + (long long)nx * ny * (nz - 1);
    if (n + 2 * faces > INT_MAX) return CPC_EINVAL;
    int* scratch = nullptr;
    const int rc = na_scratch(&scratch);
    if (rc != CPC_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((n + NA_TPB - 1) / NA_TPB);
    k_na_count<<<nblocks, NA_TPB, 0, s>>>(nx, ny, nz, scratch);
    k_na_scan<<<1, NA_TPB, 0, s>>>(nblocks, scratch, rowptr, (int)n);
    k_na_fill<<<nblocks, NA_TPB, 0, s>>>(nx, ny, nz, logk, kz_ratio, dirichlet_mask, scratch, rowptr, colidx, vals);
    return cudaGetLastError() == cudaSuccess ? CPC_OK : CPC_ECUDA;
}
