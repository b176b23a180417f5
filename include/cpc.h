/*
 * cpc.h -- C ABI of the GB300 combined-preconditioned CG library ("cpc").
 *
 * The library solves A u = f for a symmetric positive definite sparse A (Section 2, Eq.
 * linear_system of Hu, Wu, Wu, Xu, Zhang, Zhang, Zikatanov, "Combined Preconditioning with
 * Applications in Reservoir Simulation") by preconditioned conjugate gradients.  The default
 * preconditioner is the combined preconditioner B_co of Algorithm 2.1 / Eq. barB,
 *     I - B_co A = (I - S^T A)(I - B A)(I - S A),
 * with S one algebraic-multigrid V-cycle (Algorithm 3.2, Gauss-Seidel smoothing on every level,
 * Section 3.3) and B the IC(0) factorisation (Algorithm 3.1 with k = 0, Section 3.3).  Setup
 * (IC(0) factorisation, AMG hierarchy) and solve both run on the GPU.
 *
 * Conventions for every entry point:
 *  - Sizes are int32; matrices are CSR with int32 row pointers and column indices, rows sorted by
 *    column, the diagonal present in every row, structurally symmetric.
 *  - Vectors are float64 DEVICE pointers owned by the caller unless a name says _host.
 *  - Work is issued on the stream given in cpc_options.stream (a cudaStream_t; NULL = legacy
 *    default stream).  Entry points that return host-visible results (iteration counts,
 *    residual histories, timings) synchronise that stream before returning; the others are
 *    asynchronous and stream-ordered.
 *  - Return codes (never abort, never trap):
 *      CPC_OK 0, CPC_EINVAL 1 (bad argument or CSR), CPC_EFACTOR 2 (IC(0) pivot <= 0 or not
 *      finite), CPC_ENOCONV 3 (maxit reached; x holds the last iterate), CPC_EBREAKDOWN 4 (CG
 *      breakdown: p^T A p <= 0, r^T z <= 0 or NaN), CPC_ECUDA 5 (CUDA error), CPC_ETIMEOUT 6 (a
 *      bounded device wait gave up), CPC_ESETUP 7 (AMG setup failure).
 *    cpc_last_error() describes the last failure on a handle.
 */
#ifndef CPC_H
#define CPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CPC_OK = 0, CPC_EINVAL = 1, CPC_EFACTOR = 2, CPC_ENOCONV = 3, CPC_EBREAKDOWN = 4,
    CPC_ECUDA = 5, CPC_ETIMEOUT = 6, CPC_ESETUP = 7
};

/* Preconditioners (Section 5, Table 2 protocol). */
enum {
    CPC_PRECOND_BCO = 0,    /* B_co, Algorithm 2.1: S, then B, then S^T                         */
    CPC_PRECOND_AMG = 1,    /* S~ = S + S^T - S^T A S: two V-cycles ("AMG(GS)", Section 5)       */
    CPC_PRECOND_IC0 = 2,    /* B = IC(0) alone ("ILU(0)", Section 5)                             */
    CPC_PRECOND_BHAT = 3,   /* additive B^ = S~ + B, Eq. Ba with W_1 = V, Pi_1 = I, A_1^{-1} = B  */
    CPC_PRECOND_NONE = 4,   /* identity (plain CG)                                               */
    CPC_PRECOND_AMG_ILU = 5 /* "AMG(ILU(0))", Section 5: two V-cycles whose finest smoother is one  */
                            /* IC(0) step u += B (f - A u) before and after the coarse correction    */
                            /* (GS on the other levels).  Single right-hand side only.               */
};

/* Precision of the preconditioner (the outer PCG is always FP64). */
enum {
    CPC_PREC_FP64 = 0,      /* everything FP64                                                   */
    CPC_PREC_FP32 = 1,      /* V-cycles, IC(0) and the SpMVs inside B_co in FP32                 */
    CPC_PREC_FP32_BF16 = 2  /* as FP32, with coarse-level operators stored in BF16               */
};

/* Gauss-Seidel ordering of the AMG smoother S_l (Section 3.3). */
enum {
    CPC_GS_MULTICOLOUR = 0, /* rows in colour-major order: a 2-colouring by breadth-first parity on a  */
                            /* bipartite level, else a greedy colouring; one parallel step per colour */
    CPC_GS_NATURAL = 1      /* the natural row order of each level ("standard GS"): one step per      */
                            /* wavefront of the lower-triangular dependency graph, giving exactly the */
                            /* sequential sweep i = 0..n-1 (and n-1..0 for S_l^T).  Far more steps.   */
};

/* Largest accepted cpc_options.max_levels: the smoothing colourings of all levels but the
   coarsest are computed in one launch that holds per-level state for 24 levels. */
#define CPC_MAX_LEVELS 25

/* CSR matrix, caller-owned; cpc_setup copies what it needs. */
typedef struct {
    int32_t n;              /* rows = columns                                                    */
    int32_t nnz;            /* = rowptr[n]                                                       */
    const int32_t* rowptr;  /* [n + 1]                                                           */
    const int32_t* colidx;  /* [nnz], ascending within each row                                  */
    const double* vals;     /* [nnz]                                                             */
    int32_t on_device;      /* 1: the three arrays are device pointers, 0: host pointers         */
} cpc_csr;

typedef struct {
    int32_t precond;        /* CPC_PRECOND_*                                       (default BCO) */
    int32_t precision;      /* CPC_PREC_*                                          (default FP64)*/
    int32_t ic_order;       /* 0: natural order (level-scheduled); 1: multicolour order of the
                               finest level's Gauss-Seidel colouring                (default 0)   */
    int32_t gs_order;       /* CPC_GS_*; CPC_GS_NATURAL needs ic_order = 0 and tail_nnz_max <= 0
                                                                                    (default 0)   */
    double theta;           /* strength threshold of the AMG coarsening            (0.12)        */
    int32_t coarse_max;     /* stop coarsening at n_l <= coarse_max                (2048)        */
    int32_t max_levels;     /* at most this many levels, 1..CPC_MAX_LEVELS          (20)          */
    int32_t autotune;       /* 1: each coarse level's SELL chunk height C (and so its threads per
                               row, 32 / C) is picked at setup by timing a Gauss-Seidel sweep of
                               the candidates C/2, C, 2C around the row-length rule; 0: the rule
                               alone.  Timing can pick differently from one setup to the next,
                               which changes rounding (not the method).            (default 0)   */
    int64_t tail_nnz_max;   /* > 0: coarse levels run as one cluster kernel with their operators
                               in shared memory when they fit and have at most this many
                               nonzeros; 0 (default) or < 0: every level by separate launches,
                               which measures faster on GB300                                     */
    void* stream;           /* cudaStream_t used by every call on the handle       (NULL)        */
} cpc_options;

typedef struct cpc_handle cpc_handle;   /* opaque, library-owned */

/* Fill *opt with the defaults listed above.  Returns CPC_OK, or CPC_EINVAL if opt is NULL. */
int cpc_default_options(cpc_options* opt);

/*
 * Two-point-flux pressure matrix of the model problem -div(k grad p) = f (Section 4, Eq. model,
 * with c = 0) on an nx x ny x nz grid of unit cells, cell (i,j,k) numbered i + nx (j + ny k).
 * logk[n]: natural log of the cell permeability k (device); k_z = kz_ratio * k.  Face
 * transmissibility 2 k_a k_b / (k_a + k_b); faces flagged in dirichlet_mask (bits x0, x1, y0, y1,
 * z0, z1 = 1, 2, 4, 8, 16, 32) are held at p = 0 through the half-cell term 2 k (2 k_z).
 * Outputs (device, caller-allocated): rowptr[n + 1], colidx[nnz], vals[nnz] with
 * nnz = cpc_tpfa_nnz(nx, ny, nz); columns ascending.  Asynchronous on `stream`.
 */
int64_t cpc_tpfa_nnz(int32_t nx, int32_t ny, int32_t nz);
int cpc_tpfa_assemble(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                      int32_t dirichlet_mask, int32_t* rowptr, int32_t* colidx, double* vals,
                      void* stream);

/*
 * Mixed-hybrid system of Section 4 (Eq. alge_sys) for the lowest-order Raviart-Thomas element on
 * the same grid of unit cells, in (pressure, multiplier) form: unknowns are the n cell pressures,
 * then the multipliers of the x-, y- and z-faces, each family in (k, j, i) order, leaving out the
 * faces flagged in dirichlet_mask (bits as above; p = 0 there).  Entries (columns ascending):
 * cell row (c, sum over its six faces of 6 k_f), (f, -6 k_f) per free face; face row (L, -6 k_L),
 * (R, -6 k_R) for its cells, (o, 2 k_c) for the opposite face o of each cell c, (f, 4 k_L + 4 k_R);
 * k_f = k on x and y faces, k_z = kz_ratio k on z faces.  The matrix is SPD with positive
 * off-diagonal face-face entries (not an M-matrix).
 * cpc_mhfem_size returns nnz and writes the number of unknowns (host only; -1 when a size
 * exceeds int32).  cpc_mhfem_assemble writes rowptr[n_unknowns + 1], colidx[nnz], vals[nnz]
 * (device, caller-allocated) from logk[n] (device); asynchronous on `stream`.
 */
int64_t cpc_mhfem_size(int32_t nx, int32_t ny, int32_t nz, int32_t dirichlet_mask, int64_t* n_unknowns);
int cpc_mhfem_assemble(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                       int32_t dirichlet_mask, int32_t* rowptr, int32_t* colidx, double* vals, void* stream);

/*
 * Adjoint gradient through the assembly above: g_c = -lambda^T (dA/dtheta_c) p with theta = logk.
 * For A(theta) p = q and a misfit J(p), with A lambda = dJ/dp (A is symmetric, so the solver of
 * A serves), g = dJ/dtheta.  A face contributes dT/dtheta_c (lambda_c - lambda_j)(p_c - p_j) with
 * dT/dtheta_c = 2 k_c k_j^2 / (k_c + k_j)^2 (k_z on z faces), a Dirichlet face 2 k_c lambda_c p_c.
 * Not a passage of the paper: the differentiable-solve extension of its model problem (Section 4).
 * logk, lambda, p, g: device, n = nx ny nz each.  Asynchronous on `stream`.
 */
int cpc_tpfa_gradient(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                      int32_t dirichlet_mask, const double* lambda, const double* p, double* g,
                      void* stream);

/*
 * Same result as cpc_tpfa_assemble (identical rowptr, colidx and vals) without allocating any
 * device memory: for callers that cannot call cudaMalloc or cudaMallocAsync inside a library
 * call, such as simulators that own every device allocation through their own pool, or loops
 * that cannot take an allocation's synchronisation.  The paper has no counterpart; this is a
 * deployment variant of the assembly above.
 * Scratch: a 64 KiB array inside the library image (one int per block of 1024 cells), held by
 * every GPU that loads the library until the process exits.  Grids of more than 16,777,216 cells
 * (nx * ny * nz) are rejected with CPC_EINVAL.  The first call on each device looks up the
 * array's device address with that device current (and again after the device's context has
 * been replaced, e.g. by cudaDeviceReset); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (every call rewrites what it
 * reads), so calls whose work overlaps on the GPU race: order them on one stream.
 * Returns CPC_OK, CPC_EINVAL or CPC_ECUDA; on failure cpc_last_error(NULL) says why.
 * Asynchronous on `stream`.
 */
int cpc_tpfa_assemble_noalloc(int32_t nx, int32_t ny, int32_t nz, const double* logk,
                              double kz_ratio, int32_t dirichlet_mask, int32_t* rowptr,
                              int32_t* colidx, double* vals, void* stream);

/*
 * Build the solver for A: IC(0) factorisation (Algorithm 3.1, k = 0) and the AMG hierarchy
 * A_l = P_l^T A_{l+1} P_l (Section 3.2), both on the GPU.  On success *out owns all device
 * memory it needs; release it with cpc_destroy.  On failure *out is NULL and the return code
 * says why (CPC_EINVAL, CPC_EFACTOR, CPC_ESETUP, CPC_ECUDA).  Synchronous.
 */
int cpc_setup(const cpc_csr* A, const cpc_options* opt, cpc_handle** out);

/* Release every resource of the handle (NULL is ignored). */
void cpc_destroy(cpc_handle* h);

/* Text of the last error on h (or of the last failed cpc_setup when h is NULL). */
const char* cpc_last_error(const cpc_handle* h);

/*
 * PCG on A x = b with x_0 = 0 and the handle's preconditioner, stopping when
 * ||b - A x_k||_2 / ||b||_2 < tol (recursive residual) or after maxit iterations.
 * b[n], x[n]: device pointers (x is output only).  *iters = iterations taken;
 * res_hist[k] = ||r_k|| / ||b|| for k = 0..*iters (at most hist_cap values written; res_hist
 * may be NULL).  Runs the whole iteration loop on the device; synchronises the stream.
 * Returns CPC_OK, CPC_ENOCONV, CPC_EBREAKDOWN, CPC_ECUDA or CPC_EINVAL.
 */
int cpc_solve(cpc_handle* h, const double* b, double* x, double tol, int32_t maxit,
              int32_t* iters, double* res_hist, int32_t hist_cap);

/* As cpc_solve, with b and x in HOST memory: the library copies b in and x out itself. */
int cpc_solve_host(cpc_handle* h, const double* b_host, double* x_host, double tol,
                   int32_t maxit, int32_t* iters, double* res_hist, int32_t hist_cap);

/*
 * PCG on K = nrhs independent right-hand sides at once (1 <= nrhs <= 128), same preconditioner and
 * stopping rule per column as cpc_solve; every matrix and preconditioner pass serves all columns
 * (one read of the matrix per K solves).  B, X: device, [n][nrhs] row-major (entry (i, k) at
 * i * nrhs + k).  iters[nrhs] (host) receives each column's iteration count, status[nrhs] (host,
 * may be NULL) its status code.  The whole loop is one CUDA graph.  Not a passage of the paper:
 * the many-right-hand-side use of its solver.  Synchronises the stream.
 */
int cpc_solve_batched(cpc_handle* h, int32_t nrhs, const double* B, double* X, double tol,
                      int32_t maxit, int32_t* iters, int32_t* status);

/*
 * Block PCG (O'Leary 1980) on K = nrhs right-hand sides (1 <= nrhs <= 64) coupled in one block
 * Krylov space, with the handle's preconditioner applied to all K columns at once:
 *   Q = A P, alpha = (P^T Q)^{-1} gamma, X += P alpha, R -= Q alpha, Z = M R,
 *   beta = gamma^{-1} (Z^T R), gamma = Z^T R, P = Z + P beta  (gamma_0 = Z_0^T R_0, P_0 = Z_0),
 * with the K x K systems solved by Cholesky in FP64.  Stops when every column has
 * ||r_k||_2 / ||b_k||_2 < tol (recursive residual).  B, X: device, [n][nrhs] row-major as in
 * cpc_solve_batched.  *iters = block iterations taken; res[nrhs] (host, may be NULL) the final
 * relative residual of each column.  Not a passage of the paper: the coupled-column variant of the
 * many-right-hand-side solve.  Returns CPC_OK, CPC_ENOCONV, CPC_EBREAKDOWN (a K x K matrix not
 * positive definite: a rank-deficient block; X holds the last good iterate), CPC_EINVAL (nrhs out
 * of range, a zero column, or the AMG(ILU(0)) preconditioner) or CPC_ECUDA.  Synchronises the
 * stream once per iteration.
 */
int cpc_solve_block(cpc_handle* h, int32_t nrhs, const double* B, double* X, double tol, int32_t maxit,
                    int32_t* iters, double* res);

/*
 * As cpc_solve_batched, then in the same graph the adjoint solves A Lambda = G with
 * G[i][k] = X[i][k] where B[i][k] != 0 and 0 elsewhere (the gradient of
 * J_k = 1/2 sum over the source cells of column k of X[i][k]^2).  X receives the forward
 * solutions, Lambda the adjoint solutions; iters_fwd / iters_adj (host, [nrhs]) the counts.
 */
int cpc_solve_batched_adjoint(cpc_handle* h, int32_t nrhs, const double* B, double* X, double* Lambda,
                              double tol, int32_t maxit, int32_t* iters_fwd, int32_t* iters_adj);

/* z = M r for one application of a preconditioner (which = CPC_PRECOND_*; -1 = the handle's).
 * r[n], z[n] device.  Asynchronous.  cpc_apply_Bcom is which = CPC_PRECOND_BCO. */
int cpc_apply_precond(cpc_handle* h, int32_t which, const double* r, double* z);
int cpc_apply_Bcom(cpc_handle* h, const double* r, double* z);

/* y = A x with the fine matrix (FP64).  x[n], y[n] device.  Asynchronous. */
int cpc_spmv(cpc_handle* h, const double* x, double* y);

/* Setup timings in milliseconds (GPU events): IC(0) factorisation and AMG hierarchy. */
int cpc_setup_time_ms(const cpc_handle* h, double* ms_ic0, double* ms_amg);

/* The AMG setup of cpc_setup_time_ms split into its phases (GPU events, milliseconds): ms[0]
 * coarsening (strength, C/F splitting, interpolation and the Galerkin products A_l = P_l^T A_{l+1}
 * P_l of Section 3.2, all levels), ms[1] smoothing colours (or natural-order wavefronts) of all
 * levels, ms[2] the coarsest level's explicit inverse (Algorithm 3.2, step 2(b); see
 * cpc_coarse_inverse_info), ms[3] the kernels' layouts (built beside the inverse).  At most cap
 * (<= 4) values are written.  Host memory. */
int cpc_setup_phases_ms(const cpc_handle* h, double* ms, int32_t cap);

/* How the coarsest level's explicit inverse X = A_c^{-1} (Algorithm 3.2, step 2(b)) was formed:
 * *method = 1 for the FP32 Cholesky inverse refined by three Newton-Schulz steps
 * X <- X + X (I - A_c X), the residual I - A_c X in FP64 and the product X (I - A_c X) in FP32;
 * *method = 0 for the FP64 Cholesky inverse, taken when the FP32 factorisation meets a
 * non-positive pivot or the refined max |I - A_c X| stays above 1e-12.  *residual = the final
 * max_ij |(I - A_c X)_ij|, computed on the device in FP64.  Either pointer may be NULL.  Host
 * memory.  Returns CPC_OK, or CPC_EINVAL if h is NULL. */
int cpc_coarse_inverse_info(const cpc_handle* h, int32_t* method, double* residual);

/* ---- inspection (tests and diagnostics; all synchronous, outputs in HOST memory) ---------- */

/* Kernel launches of one cpc_solve with the handle's preconditioner: *per_iteration nodes in the
 * captured loop body (one PCG iteration) and *fixed launches outside the loop.  Builds the solve
 * graph if it does not exist yet. */
int cpc_solve_launches(cpc_handle* h, int64_t* per_iteration, int64_t* fixed);

/* Profiling: *us = microseconds per forward Gauss-Seidel sweep (colours ascending, one dependent
 * launch per colour, Section 3.3) of level `level` (0 <= level < levels - 1), in the handle's
 * preconditioner precision, replayed from a CUDA graph as inside the solve: `reps` sweeps
 * (1..1000) per replay, best of three replays after a warm-up.  Overwrites the level's work
 * vectors.  Synchronous. */
int cpc_sweep_time_us(cpc_handle* h, int32_t level, int32_t reps, double* us);

/* Number of AMG levels (finest = 0). */
int cpc_num_levels(const cpc_handle* h);

/* info[0..5] = n_l, nnz(A_l), number of smoothing colours, columns of P_l (= n_{l+1}),
 * nnz(P_l), number of IC(0) levels (level 0 only, else 0). */
int cpc_level_info(const cpc_handle* h, int32_t level, int64_t* info);

/* Storage of the smoother's copy of A_l: info[0] = rows per chunk C, info[1] = number of stored
 * diagonals (0 = SELL with column indices; 4, 6 or 8 = the diagonal form used when every
 * off-diagonal entry lies on at most 8 offsets col - row, as on a structured grid), info[2] =
 * slots (rows padded to chunks).  Level 0 reports the same for the natural-order copy of A in
 * info[3..5].  Returns CPC_EINVAL for a bad level; the coarsest level reports zeros. */
int cpc_level_layout(const cpc_handle* h, int32_t level, int64_t* info);

/*
 * Structural check of every device layout of the handle, a stand-in for a memory and race
 * sanitizer (every index a solve kernel gathers through comes from these layouts).  counts[5]
 * (host) receives: [0] indices out of range (slot rows, chunk pointers, columns, diagonal offsets,
 * group boundaries); [1] rows missing from or repeated in a layout; [2] pairs of coupled rows
 * (a_ij != 0) in one Gauss-Seidel colour group, which one launch would update in parallel
 * (Section 3.3); [3] IC(0) factor entries whose row's triangular-solve level is not after its
 * column's (Algorithm 3.1); [4] the number of layouts checked.  All but [4] are 0 for a sound
 * handle.  Synchronises the stream; allocates temporary device memory.
 */
int cpc_check_layouts(const cpc_handle* h, int64_t* counts);

/* Copy A_l (CSR, natural order) to host arrays sized from cpc_level_info. */
int cpc_level_matrix(const cpc_handle* h, int32_t level, int32_t* rowptr, int32_t* colidx,
                     double* vals);

/* Copy P_l (n_l x n_{l+1} CSR) to host arrays. */
int cpc_level_interp(const cpc_handle* h, int32_t level, int32_t* rowptr, int32_t* colidx,
                     double* vals);

/* Copy the C/F splitting (1 = C, 0 = F) and the smoothing colour of every row of level l (with
 * CPC_GS_NATURAL: the row's wavefront of the lower-triangular dependency graph of A_l). */
int cpc_level_splitting(const cpc_handle* h, int32_t level, int32_t* cf, int32_t* colour);

/* Copy the IC(0) factor values (L strictly below the diagonal, U on and above) laid out on the
 * pattern of the fine A in the IC ordering (natural order: the input CSR pattern). */
int cpc_ic0_values(const cpc_handle* h, double* lu);

/* Level operators on device vectors, for parity tests: op 0 y = A_l x; 1 y = S_l x (forward
 * Gauss-Seidel sweep, zero guess); 2 y = S_l^T x (backward sweep); 3 y = A_l^{-1} x (coarsest
 * level); 4 y = V-cycle from level l with zero initial guess; 5 one forward Gauss-Seidel sweep on
 * A_l y = x starting from the given y (one launch per colour, nothing else).  Asynchronous. */
int cpc_level_apply(cpc_handle* h, int32_t level, int32_t op, const double* x, double* y);

#ifdef __cplusplus
}
#endif

#endif /* CPC_H */
