// adjoint.cu -- gradient of a misfit through the two-point-flux assembly (the adjoint method).
//
// For A(theta) p = q with theta = log k and a misfit J(p), dJ/dtheta_c = -lambda^T (dA/dtheta_c) p
// where A lambda = dJ/dp (A is symmetric, so the same solver handle serves).  A face between cells
// c and j contributes T (e_c - e_j)(e_c - e_j)^T to A with dT/dtheta_c = 2 k_c k_j^2 / (k_c + k_j)^2
// (k_z = kz_ratio k on z faces); a Dirichlet face contributes 2 k_c e_c e_c^T.  k = exp(log k) is
// formed once per cell; then one thread per cell reads k, lambda and p of the cell and its six
// neighbours (cache-resident stencil) and writes g: HBM-bound.
#include "device.cuh"
#include "handle.cuh"

namespace cpc {

namespace {

__device__ __forceinline__ double dT(double a, double b) { return 2.0 * a * b * b / ((a + b) * (a + b)); }

// k_c = exp(theta_c), once per cell (FP64 exp is a long instruction sequence on this part).
__global__ void k_exp(int64_t n, const double* __restrict__ logk, double* __restrict__ k) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        k[c] = exp(logk[c]);
}

__global__ void k_tpfa_gradient(int nx, int ny, int nz, const double* __restrict__ kk, double kzr, int dmask,
                                const double* __restrict__ lam, const double* __restrict__ p, double* __restrict__ g) {
    const int n = nx * ny * nz;
    const int sxy = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int i = c % nx, j = (c / nx) % ny, k = c / sxy;
        const double kc = kk[c];
        const double kzc = kzr * kc;
        const double lc = lam[c], pc = p[c];
        double s = 0.0;
        if (k > 0)      { const int o = c - sxy; s += dT(kzc, kzr * kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        if (j > 0)      { const int o = c - nx;  s += dT(kc, kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        if (i > 0)      { const int o = c - 1;   s += dT(kc, kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        if (i < nx - 1) { const int o = c + 1;   s += dT(kc, kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        if (j < ny - 1) { const int o = c + nx;  s += dT(kc, kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        if (k < nz - 1) { const int o = c + sxy; s += dT(kzc, kzr * kk[o]) * (lc - lam[o]) * (pc - p[o]); }
        double b = 0.0;
        if ((dmask & 1) && i == 0)       b += 2.0 * kc;
        if ((dmask & 2) && i == nx - 1)  b += 2.0 * kc;
        if ((dmask & 4) && j == 0)       b += 2.0 * kc;
        if ((dmask & 8) && j == ny - 1)  b += 2.0 * kc;
        if ((dmask & 16) && k == 0)      b += 2.0 * kzc;
        if ((dmask & 32) && k == nz - 1) b += 2.0 * kzc;
        g[c] = -(s + b * lc * pc);
    }
}

}  // namespace

void tpfa_gradient(int nx, int ny, int nz, const double* logk, double kzr, int dmask, const double* lam,
                   const double* p, double* g, cudaStream_t s) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    Tmp<double> k(n, s);
    k_exp<<<grid, 256, 0, s>>>(n, logk, k.get());
    k_tpfa_gradient<<<grid, 256, 0, s>>>(nx, ny, nz, k.get(), kzr, dmask, lam, p, g);
    CPC_LAUNCH_CK();
}

}  // namespace cpc
