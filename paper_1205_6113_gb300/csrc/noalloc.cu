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
#include <cuda.h>

#include <climits>
#include <mutex>
#include <string>

#include "../../include/cpc.h"
#include "tpfa_cell.cuh"

namespace cpc {
// The library's thread-local error text (api.cu), read back by cpc_last_error(NULL).
void set_global_error(const std::string& msg);
}  // namespace cpc

namespace {

constexpr int NA_TPB = 1024;                      // cells per block
constexpr int NA_MAX_BLOCKS = 16384;              // scratch entries
constexpr long long NA_MAX_CELLS = (long long)NA_TPB * NA_MAX_BLOCKS;
constexpr int NA_MAX_DEVICES = 64;

// Per-block row counts, then their exclusive prefix sums (the block's first row offset).
static __device__ __align__(256) int g_na_block_rows[NA_MAX_BLOCKS];

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
    const int len = c < n ? cpc::tpfa_row_len(c, nx, ny, nz) : 0;
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

// Row offsets and entries of every cell: each block finds its rows' offsets from its own scan and
// the block prefix, then writes its cells' rows with the same per-cell code as cpc_tpfa_assemble.
__global__ void __launch_bounds__(NA_TPB) k_na_fill(int nx, int ny, int nz, const double* logk, double kzr,
                                                      int dmask, const int* block_rows, int* rowptr, int* col,
                                                      double* val) {
    const int n = nx * ny * nz;
    const int c = blockIdx.x * NA_TPB + threadIdx.x;
    const int len = c < n ? cpc::tpfa_row_len(c, nx, ny, nz) : 0;
    int total;
    const int off = na_block_exclusive_scan(len, &total) + block_rows[blockIdx.x];
    if (c >= n) return;
    rowptr[c] = off;
    cpc::tpfa_fill_row(c, nx, ny, nz, logk, kzr, dmask, off, col, val);
}

// Device address of the scratch array, looked up once per device with that device current, and
// again whenever the device's current context is not the one the address was taken in: a
// cudaDeviceReset between calls ends the old context, the library image is loaded again into the
// new one, and the array may then live at another address.  The context is identified by its
// unique id (cuCtxGetId), fetched through the runtime's driver entry points.
std::mutex g_na_mu;
int* g_na_addr[NA_MAX_DEVICES] = {};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long na_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (CtxGetCurrentFn)f1;
            get_id = (CtxGetIdFn)f2;
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

const char* na_scratch(int** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return "no usable current device";
    std::lock_guard<std::mutex> lock(g_na_mu);
    const unsigned long long ctx = na_context_id();      // 0 before the runtime made a context
    if (!g_na_addr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
        int* ptr = nullptr;
        if (cudaGetSymbolAddress((void**)&ptr, g_na_block_rows) != cudaSuccess || !ptr)
            return "cudaGetSymbolAddress of the scratch array failed";
        g_na_addr[dev] = ptr;
        g_na_ctx[dev] = na_context_id();                 // the context the lookup ran in
    }
    *out = g_na_addr[dev];
    return nullptr;
}

int na_fail(int code, const std::string& msg) {
    cpc::set_global_error("cpc_tpfa_assemble_noalloc: " + msg);
    return code;
}

// Launches one kernel and returns that launch's own error (earlier errors are not consumed).
template <class... KArgs, class... Args>
cudaError_t na_launch(void (*k)(KArgs...), int grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(NA_TPB, 1, 1);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace

extern "C" int cpc_tpfa_assemble_noalloc(int32_t nx, int32_t ny, int32_t nz, const double* logk,
                                         double kz_ratio, int32_t dirichlet_mask, int32_t* rowptr,
                                         int32_t* colidx, double* vals, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !logk || !rowptr || !colidx || !vals || !(kz_ratio > 0.0))
        return na_fail(CPC_EINVAL, "invalid arguments");
    const long long n = (long long)nx * ny * nz;
    if (n > NA_MAX_CELLS)                                 // beyond the scratch array's capacity
        return na_fail(CPC_EINVAL, "grid has more than 16,777,216 cells (the scratch array's limit)");
    const long long faces = (long long)(nx - 1) * ny * nz + (long long)nx * (ny - 1) * nz + (long long)nx * ny * (nz - 1);
    if (n + 2 * faces > INT_MAX) return na_fail(CPC_EINVAL, "nonzero count overflows int32");
    int* scratch = nullptr;
    if (const char* why = na_scratch(&scratch)) return na_fail(CPC_ECUDA, why);
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((n + NA_TPB - 1) / NA_TPB);
    cudaError_t e = na_launch(k_na_count, nblocks, s, (int)nx, (int)ny, (int)nz, scratch);
    if (e == cudaSuccess) e = na_launch(k_na_scan, 1, s, nblocks, scratch, (int*)rowptr, (int)n);
    if (e == cudaSuccess)
        e = na_launch(k_na_fill, nblocks, s, (int)nx, (int)ny, (int)nz, logk, kz_ratio, (int)dirichlet_mask,
                      (const int*)scratch, (int*)rowptr, (int*)colidx, vals);
    if (e != cudaSuccess) return na_fail(CPC_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return CPC_OK;
}
