// handle.cuh -- the solver handle: hierarchy, IC(0) factor, work vectors, captured graphs.
#pragma once

#include "common.cuh"

namespace cpc {

constexpr int CHUNK = 32;            // SELL chunk height = warp width
constexpr int DENSE_MAX = 4096;      // largest coarsest level solved by the dense inverse
constexpr int HIST_CAP = 100001;     // residual-history capacity on the device
constexpr int NPART = 1024;          // partial-sum slots for deterministic reductions
constexpr int NPRECOND = 6;          // CPC_PRECOND_* values

// One AMG level (0 = finest).
struct Level {
    int n = 0;
    int64_t nnz = 0;
    Csr A;                  // A_l, natural order, FP64
    Csr P, R;               // interpolation to this level from level l+1, and R = P^T
    DBuf<int> cf, colour;   // C/F splitting, smoothing colour (natural order)
    int ncolours = 0;
    Sell S;                 // rows grouped by colour, diagonal split: Gauss-Seidel and residual
    Sell SP, SR;            // P and R, natural row order
    VType vt = VT_F64;      // storage type of this level's operators in the preconditioner
    DBuf<double> dnat64;    // 1 / a_ii in natural row order (first colour step from a zero guess)
    DBuf<float> dnat32;
    DBuf<double> x64, f64, r64;
    DBuf<float> x32, f32, r32;
};

// Batched PCG state: block vectors [n][Kp] (Kp = K rounded up to 32), level vectors in the
// preconditioner's precision (raw bytes), per-column scalars, and the captured graph.
struct Batched {
    int K = 0, Kp = 0;
    bool adjoint = false;
    DBuf<double> b, x, r, p, q, xfwd;
    DBuf<char> z, t, y;
    std::vector<DBuf<char>> lx, lf, lr;
    DBuf<double> S, partial, kfwd;
    // block CG: K x K matrices [KM_COUNT][Kp][Kp], Gram partials, column vectors [KV_COUNT][Kp], flags
    DBuf<double> kmat, kpart, kvec;
    DBuf<int> kflag;
    double* user_b = nullptr;
    double* user_x = nullptr;
    double* user_lambda = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

// Device-side scalars of one PCG run (all reductions finish in fixed order).
struct PcgState {
    double bnorm, rz, rz_old, pq, alpha, beta, rr, tol, res;
    int k, maxit, status, pad;
};

struct Handle {
    cpc_options opt{};
    cudaStream_t s = nullptr;
    int n = 0;
    int64_t nnz = 0;
    std::vector<Level> lev;
    Sell Anat;              // fine A in natural row order, diagonal split (SpMVs of PCG and B_co)
    // IC(0) (Algorithm 3.1, k = 0) of the fine A in the IC ordering
    Csr Aic;                // A in the IC ordering (same as lev[0].A for natural order)
    DBuf<double> lu;        // factor values on the pattern of Aic
    DBuf<int> lu_diag;      // position of the diagonal in each row of Aic
    DBuf<int> ic_order;     // ic row q <- original row ic_order[q] (empty: natural)
    int ic_levels_L = 0, ic_levels_U = 0;
    // Red-black IC(0) in B_co: black rows of L (chunks [ic_black_c0, ic_black_c1)) and 1 / u_ii in
    // natural order, when the IC order is the fine 2-colouring with every black row coupled.
    bool ic_rb = false;
    int ic_rows_L1 = 0, ic_black_c0 = 0, ic_black_c1 = 0;
    DBuf<double> ic_uinv64;
    DBuf<float> ic_uinv32;
    Sell L, U;              // strictly-lower rows by forward level; upper rows by backward level
    // coarsest level: dense inverse
    int nc = 0;
    DBuf<double> Ainv;
    DBuf<float> Ainv32;
    int inv_method = 0;     // 1: FP32 Cholesky inverse + Newton-Schulz steps; 0: FP64 Cholesky inverse
    double inv_resid = 0;   // max |I - A_c Ainv| measured after setup
    // fine-level vectors
    DBuf<double> b, x, r, z, p, q, t, y;
    DBuf<float> z32, t32, y32;
    DBuf<double> bt, yt;    // IC-ordered copies when the IC ordering is not natural
    DBuf<float> bt32, yt32;
    // reductions and PCG state
    DBuf<double> partial;
    DBuf<unsigned> counter;
    DBuf<PcgState> state;
    DBuf<double> hist;
    DBuf<int> flags;        // [0] IC factor failure row + 1, [1] coarse Cholesky failure
    cudaGraph_t graph[NPRECOND] = {};
    cudaGraphExec_t gexec[NPRECOND] = {};
    int64_t body_nodes[NPRECOND] = {};
    // coarse levels >= tail_start run as one cluster kernel (tail.cu)
    int tail_start = 0;
    int tail_cluster = 0;
    size_t tail_smem = 0;
    DBuf<char> tail_desc;
    DBuf<char> tail_img;
    std::vector<DBuf<int>> tail_seg;
    Batched bat;
    float ms_ic0 = 0.f, ms_amg = 0.f;
    float ms_phase[4] = {0.f, 0.f, 0.f, 0.f};   // AMG setup: coarsening, colouring, coarsest inverse, layouts
    std::string err;
    ~Handle();
};

// adjoint.cu
void tpfa_gradient(int nx, int ny, int nz, const double* logk, double kzr, int dmask, const double* lam,
                   const double* p, double* g, cudaStream_t s);

// setup.cu
void tpfa_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask, int* rowptr,
                   int* col, double* val, cudaStream_t s);
// Mixed-hybrid (p, lambda) system of Section 4 on unit bricks (mhfem.cu): sizes, then assembly.
int64_t mhfem_size(int nx, int ny, int nz, int dmask, int64_t* nunk);
void mhfem_assemble(int nx, int ny, int nz, const double* logk, double kzr, int dmask, int* rowptr, int* col,
                    double* val, cudaStream_t s);
void setup_handle(Handle& h, const cpc_csr& A);

// batched.cu
void solve_batched(Handle& h, int K, const double* b, double* x, double* lambda, double tol, int maxit,
                   int* iters, int* status, int* iters_adj, int* status_adj);
// Structural checks of every device layout (check.cu); counts[5]: out of range, coverage,
// Gauss-Seidel races, triangular-solve races, layouts checked.
void check_layouts(Handle& h, int64_t* counts);

// Block PCG (O'Leary 1980) on K <= 64 columns; returns CPC_OK, CPC_ENOCONV or CPC_EBREAKDOWN.
int solve_block(Handle& h, int K, const double* b, double* x, double tol, int maxit, int* iters, double* res);
void destroy_batched(Handle& h);

// tail.cu
void setup_tail(Handle& h, int64_t tail_nnz_max);
// Milliseconds of one forward Gauss-Seidel sweep over the colour groups of S (FP64, zero vectors),
// replayed from a CUDA graph as in the solve: the cost the chunk-height autotuner compares.
float time_gs_sweep(const Sell& S, int n);
void record_tail(Handle& h, int level, const void* f0, void* x0, cudaStream_t s);

// solve.cu
void record_precond(Handle& h, int which, const double* r, void* z, cudaStream_t s);
void apply_precond(Handle& h, int which, const double* r, double* z);
void spmv_fine(Handle& h, const double* x, double* y, cudaStream_t s);
void solve_pcg(Handle& h, const double* b, double* x, double tol, int maxit, int* iters,
               double* res_hist, int hist_cap, int* status);
void level_apply(Handle& h, int l, int op, const double* x, double* y);
double sweep_time_us(Handle& h, int l, int reps);
// Warps (SELL chunks) per block of the colour-step kernel, and how many of its blocks the GPU
// holds at once (all SMs) for an operator whose lanes hold at most `lanes` entries (FP64).
constexpr int GS_WARPS_PER_BLOCK = 4;
int gs_resident_blocks(int lanes);
void destroy_graphs(Handle& h);
void ensure_solve_graph(Handle& h, int which);

}  // namespace cpc
