// api.cu -- the extern "C" entry points of include/cpc.h: argument checks, error capture, and
// dispatch into setup.cu / solve.cu.  No exception or CUDA error crosses the C boundary.
#include <algorithm>
#include <cstring>
#include <new>

#include "handle.cuh"

struct cpc_handle {
    cpc::Handle h;
};

namespace cpc {
Handle::~Handle() {
    destroy_graphs(*this);
    destroy_batched(*this);
}
}  // namespace cpc

namespace {

thread_local std::string g_setup_err;

template <class F>
int guarded(cpc_handle* h, F&& f) {
    try {
        f();
        return CPC_OK;
    } catch (const cpc::Error& e) {
        if (h) h->h.err = e.msg;
        else g_setup_err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (h) h->h.err = "host allocation failed";
        else g_setup_err = "host allocation failed";
        return CPC_ECUDA;
    } catch (...) {
        if (h) h->h.err = "unexpected error";
        else g_setup_err = "unexpected error";
        return CPC_ECUDA;
    }
}

}  // namespace

namespace cpc {
void set_global_error(const std::string& msg) { g_setup_err = msg; }
}  // namespace cpc

extern "C" {

int cpc_default_options(cpc_options* opt) {
    if (!opt) return CPC_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->precond = CPC_PRECOND_BCO;
    opt->precision = CPC_PREC_FP64;
    opt->ic_order = 0;
    opt->gs_order = CPC_GS_MULTICOLOUR;
    opt->theta = 0.12;
    opt->coarse_max = 2048;
    opt->autotune = 0;
    opt->max_levels = 20;
    opt->tail_nnz_max = 0;
    opt->stream = nullptr;
    return CPC_OK;
}

int64_t cpc_tpfa_nnz(int32_t nx, int32_t ny, int32_t nz) {
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    const int64_t faces = (int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + (int64_t)nx * ny * (nz - 1);
    return (int64_t)nx * ny * nz + 2 * faces;
}

int cpc_tpfa_assemble(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                      int32_t dirichlet_mask, int32_t* rowptr, int32_t* colidx, double* vals, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !logk || !rowptr || !colidx || !vals) return CPC_EINVAL;
    if ((int64_t)nx * ny * nz > INT32_MAX || cpc_tpfa_nnz(nx, ny, nz) > INT32_MAX) return CPC_EINVAL;
    if (!(kz_ratio > 0.0)) return CPC_EINVAL;
    return guarded(nullptr, [&] {
        cpc::tpfa_assemble(nx, ny, nz, logk, kz_ratio, dirichlet_mask, rowptr, colidx, vals, (cudaStream_t)stream);
    });
}

int64_t cpc_mhfem_size(int32_t nx, int32_t ny, int32_t nz, int32_t dirichlet_mask, int64_t* n_unknowns) {
    if (nx < 1 || ny < 1 || nz < 1 || !n_unknowns || (int64_t)nx * ny * nz > INT32_MAX) return -1;
    const int64_t nnz = cpc::mhfem_size(nx, ny, nz, dirichlet_mask, n_unknowns);
    if (*n_unknowns > INT32_MAX || nnz > INT32_MAX) return -1;
    return nnz;
}

int cpc_mhfem_assemble(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                       int32_t dirichlet_mask, int32_t* rowptr, int32_t* colidx, double* vals, void* stream) {
    int64_t nu = 0;
    if (!logk || !rowptr || !colidx || !vals || !(kz_ratio > 0.0) ||
        cpc_mhfem_size(nx, ny, nz, dirichlet_mask, &nu) < 0)
        return CPC_EINVAL;
    return guarded(nullptr, [&] {
        cpc::mhfem_assemble(nx, ny, nz, logk, kz_ratio, dirichlet_mask, rowptr, colidx, vals, (cudaStream_t)stream);
    });
}

int cpc_tpfa_gradient(int32_t nx, int32_t ny, int32_t nz, const double* logk, double kz_ratio,
                      int32_t dirichlet_mask, const double* lambda, const double* p, double* g, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !logk || !lambda || !p || !g || !(kz_ratio > 0.0)) return CPC_EINVAL;
    if ((int64_t)nx * ny * nz > INT32_MAX) return CPC_EINVAL;
    return guarded(nullptr, [&] {
        cpc::tpfa_gradient(nx, ny, nz, logk, kz_ratio, dirichlet_mask, lambda, p, g, (cudaStream_t)stream);
    });
}

int cpc_setup(const cpc_csr* A, const cpc_options* opt, cpc_handle** out) {
    if (!out) return CPC_EINVAL;
    *out = nullptr;
    if (!A || A->n <= 0 || A->nnz < A->n || !A->rowptr || !A->colidx || !A->vals) {
        g_setup_err = "invalid CSR arguments";
        return CPC_EINVAL;
    }
    cpc_options o;
    if (opt) o = *opt; else cpc_default_options(&o);
    if (o.precond < 0 || o.precond > CPC_PRECOND_AMG_ILU || o.precision < 0 || o.precision > CPC_PREC_FP32_BF16 ||
        o.ic_order < 0 || o.ic_order > 1 || !(o.theta > 0.0 && o.theta < 1.0) || o.coarse_max < 1 || o.autotune < 0 || o.autotune > 1 ||
        o.max_levels < 1 || o.max_levels > CPC_MAX_LEVELS || o.gs_order < CPC_GS_MULTICOLOUR || o.gs_order > CPC_GS_NATURAL) {
        g_setup_err = "invalid options";
        return CPC_EINVAL;
    }
    if (o.gs_order == CPC_GS_NATURAL && (o.ic_order != 0 || o.tail_nnz_max > 0)) {
        g_setup_err = "natural-order Gauss-Seidel needs natural-order IC(0) and no cluster kernel";
        return CPC_EINVAL;
    }
    cpc_handle* h = new (std::nothrow) cpc_handle();
    if (!h) return CPC_ECUDA;
    h->h.opt = o;
    h->h.s = (cudaStream_t)o.stream;
    const int rc = guarded(nullptr, [&] { cpc::setup_handle(h->h, *A); });
    if (rc != CPC_OK) {
        cudaStreamSynchronize(h->h.s);
        delete h;
        cudaGetLastError();
        return rc;
    }
    *out = h;
    return CPC_OK;
}

void cpc_destroy(cpc_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->h.s);
    delete h;
}

const char* cpc_last_error(const cpc_handle* h) {
    return h ? h->h.err.c_str() : g_setup_err.c_str();
}

static int do_solve(cpc_handle* h, const double* b, double* x, double tol, int32_t maxit, int32_t* iters,
                    double* res_hist, int32_t hist_cap) {
    if (!h || !b || !x || !iters || maxit < 0 || !(tol >= 0.0)) return CPC_EINVAL;
    int status = CPC_OK;
    const int rc = guarded(h, [&] {
        int it = 0;
        cpc::solve_pcg(h->h, b, x, tol, maxit, &it, res_hist, hist_cap, &status);
        *iters = it;
    });
    if (rc != CPC_OK) return rc;
    if (status == CPC_ENOCONV) h->h.err = "not converged within maxit";
    if (status == CPC_EBREAKDOWN) h->h.err = "CG breakdown (p^T A p <= 0, r^T z <= 0 or not finite)";
    return status;
}

int cpc_solve(cpc_handle* h, const double* b, double* x, double tol, int32_t maxit, int32_t* iters,
              double* res_hist, int32_t hist_cap) {
    return do_solve(h, b, x, tol, maxit, iters, res_hist, hist_cap);
}

int cpc_solve_host(cpc_handle* h, const double* b_host, double* x_host, double tol, int32_t maxit,
                   int32_t* iters, double* res_hist, int32_t hist_cap) {
    return do_solve(h, b_host, x_host, tol, maxit, iters, res_hist, hist_cap);
}

int cpc_solve_batched(cpc_handle* h, int32_t nrhs, const double* B, double* X, double tol, int32_t maxit,
                      int32_t* iters, int32_t* status) {
    if (!h || nrhs < 1 || nrhs > 128 || !B || !X || !iters || maxit < 0 || !(tol >= 0.0)) return CPC_EINVAL;
    return guarded(h, [&] { cpc::solve_batched(h->h, nrhs, B, X, nullptr, tol, maxit, iters, status, nullptr, nullptr); });
}

int cpc_check_layouts(const cpc_handle* h, int64_t* counts) {
    if (!h || !counts) return CPC_EINVAL;
    cpc_handle* hh = const_cast<cpc_handle*>(h);
    return guarded(hh, [&] { cpc::check_layouts(hh->h, counts); });
}

int cpc_solve_block(cpc_handle* h, int32_t nrhs, const double* B, double* X, double tol, int32_t maxit,
                    int32_t* iters, double* res) {
    if (!h || nrhs < 1 || nrhs > 64 || !B || !X || !iters || maxit < 0 || !(tol >= 0.0)) return CPC_EINVAL;
    int status = CPC_OK;
    const int rc = guarded(h, [&] { status = cpc::solve_block(h->h, nrhs, B, X, tol, maxit, iters, res); });
    if (rc != CPC_OK) return rc;
    if (status == CPC_ENOCONV) h->h.err = "block CG not converged within maxit";
    if (status == CPC_EBREAKDOWN) h->h.err = "block CG breakdown (a K x K matrix is not positive definite)";
    return status;
}

int cpc_solve_batched_adjoint(cpc_handle* h, int32_t nrhs, const double* B, double* X, double* Lambda, double tol,
                              int32_t maxit, int32_t* iters_fwd, int32_t* iters_adj) {
    if (!h || nrhs < 1 || nrhs > 128 || !B || !X || !Lambda || !iters_fwd || !iters_adj || maxit < 0 || !(tol >= 0.0))
        return CPC_EINVAL;
    return guarded(h, [&] {
        cpc::solve_batched(h->h, nrhs, B, X, Lambda, tol, maxit, iters_fwd, nullptr, iters_adj, nullptr);
    });
}

int cpc_apply_precond(cpc_handle* h, int32_t which, const double* r, double* z) {
    if (!h || !r || !z) return CPC_EINVAL;
    if (which < 0) which = h->h.opt.precond;
    return guarded(h, [&] { cpc::apply_precond(h->h, which, r, z); });
}

int cpc_apply_Bcom(cpc_handle* h, const double* r, double* z) {
    return cpc_apply_precond(h, CPC_PRECOND_BCO, r, z);
}

int cpc_spmv(cpc_handle* h, const double* x, double* y) {
    if (!h || !x || !y) return CPC_EINVAL;
    return guarded(h, [&] { cpc::spmv_fine(h->h, x, y, h->h.s); });
}

int cpc_setup_time_ms(const cpc_handle* h, double* ms_ic0, double* ms_amg) {
    if (!h || !ms_ic0 || !ms_amg) return CPC_EINVAL;
    *ms_ic0 = h->h.ms_ic0;
    *ms_amg = h->h.ms_amg;
    return CPC_OK;
}

int cpc_solve_launches(cpc_handle* h, int64_t* per_iteration, int64_t* fixed) {
    if (!h || !per_iteration || !fixed) return CPC_EINVAL;
    return guarded(h, [&] {
        cpc::ensure_solve_graph(h->h, h->h.opt.precond);
        *per_iteration = h->h.body_nodes[h->h.opt.precond];
        *fixed = 1;
    });
}

int cpc_setup_phases_ms(const cpc_handle* h, double* ms, int32_t cap) {
    if (!h || !ms || cap < 0) return CPC_EINVAL;
    for (int i = 0; i < cap && i < 4; ++i) ms[i] = h->h.ms_phase[i];
    return CPC_OK;
}

int cpc_coarse_inverse_info(const cpc_handle* h, int32_t* method, double* residual) {
    if (!h) return CPC_EINVAL;
    if (method) *method = h->h.inv_method;
    if (residual) *residual = h->h.inv_resid;
    return CPC_OK;
}

int cpc_sweep_time_us(cpc_handle* h, int32_t level, int32_t reps, double* us) {
    if (!h || !us) return CPC_EINVAL;
    return guarded(h, [&] { *us = cpc::sweep_time_us(h->h, level, reps); });
}

int cpc_num_levels(const cpc_handle* h) { return h ? (int)h->h.lev.size() : -1; }

int cpc_level_info(const cpc_handle* h, int32_t level, int64_t* info) {
    if (!h || !info || level < 0 || level >= (int)h->h.lev.size()) return CPC_EINVAL;
    const cpc::Level& L = h->h.lev[level];
    info[0] = L.n;
    info[1] = L.A.nnz;
    info[2] = L.ncolours;
    info[3] = L.P.m;
    info[4] = L.P.nnz;
    info[5] = level == 0 ? h->h.ic_levels_L : 0;
    return CPC_OK;
}

int cpc_level_layout(const cpc_handle* h, int32_t level, int64_t* info) {
    if (!h || !info || level < 0 || level >= (int)h->h.lev.size()) return CPC_EINVAL;
    const cpc::Level& L = h->h.lev[level];
    const bool last = level == (int)h->h.lev.size() - 1;
    info[0] = last ? 0 : L.S.C;
    info[1] = last ? 0 : L.S.ndiag;
    info[2] = last ? 0 : L.S.nslots;
    const cpc::Sell& A = h->h.Anat;
    info[3] = level == 0 ? A.C : 0;
    info[4] = level == 0 ? A.ndiag : 0;
    info[5] = level == 0 ? A.nslots : 0;
    return CPC_OK;
}

static int copy_csr_out(cpc_handle* hh, const cpc::Csr& A, int32_t* rowptr, int32_t* colidx, double* vals) {
    return guarded(hh, [&] {
        CPC_CK(cudaStreamSynchronize(hh->h.s));
        CPC_CK(cudaMemcpy(rowptr, A.ptr.p, sizeof(int) * (A.n + 1), cudaMemcpyDeviceToHost));
        if (A.nnz) {
            CPC_CK(cudaMemcpy(colidx, A.col.p, sizeof(int) * A.nnz, cudaMemcpyDeviceToHost));
            CPC_CK(cudaMemcpy(vals, A.val.p, sizeof(double) * A.nnz, cudaMemcpyDeviceToHost));
        }
    });
}

int cpc_level_matrix(const cpc_handle* h, int32_t level, int32_t* rowptr, int32_t* colidx, double* vals) {
    if (!h || !rowptr || !colidx || !vals || level < 0 || level >= (int)h->h.lev.size()) return CPC_EINVAL;
    cpc_handle* hh = const_cast<cpc_handle*>(h);
    return copy_csr_out(hh, h->h.lev[level].A, rowptr, colidx, vals);
}

int cpc_level_interp(const cpc_handle* h, int32_t level, int32_t* rowptr, int32_t* colidx, double* vals) {
    if (!h || !rowptr || !colidx || !vals || level < 0 || level + 1 >= (int)h->h.lev.size()) return CPC_EINVAL;
    cpc_handle* hh = const_cast<cpc_handle*>(h);
    return copy_csr_out(hh, h->h.lev[level].P, rowptr, colidx, vals);
}

int cpc_level_splitting(const cpc_handle* h, int32_t level, int32_t* cf, int32_t* colour) {
    if (!h || !cf || !colour || level < 0 || level + 1 >= (int)h->h.lev.size()) return CPC_EINVAL;
    cpc_handle* hh = const_cast<cpc_handle*>(h);
    const cpc::Level& L = h->h.lev[level];
    return guarded(hh, [&] {
        CPC_CK(cudaStreamSynchronize(hh->h.s));
        CPC_CK(cudaMemcpy(cf, L.cf.p, sizeof(int) * L.n, cudaMemcpyDeviceToHost));
        CPC_CK(cudaMemcpy(colour, L.colour.p, sizeof(int) * L.n, cudaMemcpyDeviceToHost));
    });
}

int cpc_ic0_values(const cpc_handle* h, double* lu) {
    if (!h || !lu) return CPC_EINVAL;
    cpc_handle* hh = const_cast<cpc_handle*>(h);
    return guarded(hh, [&] {
        CPC_CK(cudaStreamSynchronize(hh->h.s));
        CPC_CK(cudaMemcpy(lu, h->h.lu.p, sizeof(double) * h->h.Aic.nnz, cudaMemcpyDeviceToHost));
    });
}

int cpc_level_apply(cpc_handle* h, int32_t level, int32_t op, const double* x, double* y) {
    if (!h || !x || !y) return CPC_EINVAL;
    return guarded(h, [&] { cpc::level_apply(h->h, level, op, x, y); });
}

}  // extern "C"
