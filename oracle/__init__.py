"""CPU oracle for combined-preconditioned CG -- TEST INFRASTRUCTURE ONLY.

Plain FP64 code (``oracle.cpp``, plus the Lanczos helper below) that follows the
paper's algorithms step by step.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import it.  The CUDA library never
imports, links or calls anything here, and this package imports nothing from the
CUDA library.

Operator codes for :meth:`Oracle.apply` / :meth:`Oracle.pcg`:
``BCO`` (Algorithm 2.1, Eq. barB), ``S`` (one V-cycle, Algorithm 3.2), ``ST`` (its
adjoint), ``B`` (IC(0), Algorithm 3.1 with k = 0), ``STILDE`` (two cycles,
S~ = S + S^T - S^T A S), ``BHAT`` (additive S~ + B, Eq. Ba), ``A``, ``I``,
``S_ILU`` (one V-cycle with IC(0) as the finest smoother) and ``AMG_ILU`` (two such
cycles: AMG(ILU(0)) of Section 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "_liboracle.so")
LIB_OMP = os.path.join(HERE, "_liboracle_omp.so")

BCO, S, ST, B, STILDE, BHAT, A, I, S_ILU, AMG_ILU = range(10)
OPS = {"bco": BCO, "amg": STILDE, "ilu": B, "bhat": BHAT, "none": I, "amg_ilu": AMG_ILU}

STATUS = {0: "ok", 1: "invalid argument", 2: "IC(0) breakdown", 3: "not converged",
          4: "CG breakdown", 7: "AMG setup failure"}


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.cpp with g++ (plain FP64, no FMA contraction).  The default library is
    single-threaded; with openmp a second library is built with -fopenmp, whose parallel loops
    serve only to time the oracle on all host cores."""
    target = LIB_OMP if openmp else LIB
    if force or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(SRC):
        tmp = target + ".%d.tmp" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off"]
                              + (["-fopenmp"] if openmp else []) + ["-o", tmp, SRC])
        os.replace(tmp, target)
    return target


_libs = {}


def lib(openmp: bool = False):
    if openmp not in _libs:
        L = ctypes.CDLL(build(openmp=openmp))
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        L.orc_threads.restype = i32
        L.orc_threads.argtypes = []
        L.orc_tpfa_nnz.restype = i32
        L.orc_tpfa_nnz.argtypes = [i32, i32, i32]
        L.orc_tpfa.restype = i32
        L.orc_tpfa.argtypes = [i32, i32, i32, P, f64, i32, P, P, P]
        L.orc_tpfa_gradient.restype = i32
        L.orc_tpfa_gradient.argtypes = [i32, i32, i32, P, f64, i32, P, P, P]
        L.orc_create.restype = P
        L.orc_create.argtypes = [i32, P, P, P, f64, i32, i32, i32, i32, P]
        L.orc_destroy.argtypes = [P]
        L.orc_nlevels.restype = i32
        L.orc_nlevels.argtypes = [P]
        for name in ("orc_level_sizes", "orc_level_A", "orc_level_P", "orc_level_cf_colour",
                     "orc_ic0_values", "orc_level_apply", "orc_apply", "orc_pcg", "orc_mhfem_size",
                     "orc_mhfem"):
            getattr(L, name).restype = i32
        L.orc_level_sizes.argtypes = [P, i32, P]
        L.orc_level_A.argtypes = [P, i32, P, P, P]
        L.orc_level_P.argtypes = [P, i32, P, P, P]
        L.orc_level_cf_colour.argtypes = [P, i32, P, P]
        L.orc_ic0_values.argtypes = [P, P]
        L.orc_level_apply.argtypes = [P, i32, i32, P, P]
        L.orc_apply.argtypes = [P, i32, P, P]
        L.orc_mhfem_size.argtypes = [i32, i32, i32, P, f64, i32, P]
        L.orc_mhfem.argtypes = [i32, i32, i32, P, f64, i32, P, P, P]
        L.orc_pcg.argtypes = [P, i32, P, P, f64, i32, P, P, P, P, i32, P]
        _libs[openmp] = L
    return _libs[openmp]


def threads(openmp: bool = False) -> int:
    """Threads the oracle's parallel loops use (1 for the default library)."""
    return int(lib(openmp).orc_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class Csr:
    """Host CSR matrix (int32 indices, float64 values)."""

    def __init__(self, n, rowptr, col, val, m=None):
        self.n = int(n)
        self.m = int(m if m is not None else n)
        self.rowptr = _i32(rowptr)
        self.col = _i32(col)
        self.val = _f64(val)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.m))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.col[p]] += self.val[p]
        return D

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.n)


def tpfa(nx, ny, nz, logk, kz_ratio, dirichlet) -> Csr:
    """Two-point-flux matrix of Section 4's model problem (c = 0) on an nx x ny x nz grid."""
    n = nx * ny * nz
    nnz = lib().orc_tpfa_nnz(nx, ny, nz)
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    logk = _f64(logk)
    st = lib().orc_tpfa(nx, ny, nz, _p(logk), float(kz_ratio), int(dirichlet), _p(rowptr), _p(col), _p(val))
    if st:
        raise ValueError("orc_tpfa failed: %d" % st)
    return Csr(n, rowptr, col, val)


def mhfem(nx, ny, nz, logk, kz_ratio, dirichlet) -> Csr:
    """The mixed-hybrid (p, lambda) system of Section 5, Eq. alge_sys, on unit bricks (oracle.cpp)."""
    logk = _f64(logk)
    sz = np.zeros(2, np.int32)
    if lib().orc_mhfem_size(nx, ny, nz, _p(logk), float(kz_ratio), int(dirichlet), _p(sz)):
        raise ValueError("bad grid")
    n, nnz = int(sz[0]), int(sz[1])
    ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    lib().orc_mhfem(nx, ny, nz, _p(logk), float(kz_ratio), int(dirichlet), _p(ptr), _p(col), _p(val))
    return Csr(n, ptr, col, val)


def mhfem_problem(prob):
    """(A, b) of the mixed-hybrid system for a structured-grid problem: b = cell sources, 0 on faces."""
    A = mhfem(prob.nx, prob.ny, prob.nz, prob.logk, prob.kz_ratio, prob.dirichlet)
    b = np.zeros(A.n)
    b[:prob.n] = prob.rhs()
    return A, b


def tpfa_gradient(nx, ny, nz, logk, kz_ratio, dirichlet, lam, p) -> np.ndarray:
    """g = -lambda^T (dA/dlog k) p for the two-point-flux matrix (adjoint gradient through the assembly)."""
    logk, lam, p = _f64(logk), _f64(lam), _f64(p)
    g = np.zeros(nx * ny * nz)
    if lib().orc_tpfa_gradient(nx, ny, nz, _p(logk), float(kz_ratio), int(dirichlet), _p(lam), _p(p), _p(g)):
        raise ValueError("orc_tpfa_gradient failed")
    return g


def well_means(p, wells_cells) -> np.ndarray:
    """Mean pressure over the cells of each well."""
    return np.array([np.mean(p[np.asarray(c)]) for c in wells_cells])


def misfit_gradient(A: Csr, prob, logk, wells_cells, d, orc=None, tol=1e-12):
    """J = 1/2 sum_w (mean_w p - d_w)^2 with A(logk) p = q, and dJ/dlog k by the adjoint method."""
    orc = orc or Oracle(A)
    q = prob.rhs()
    p = orc.pcg(q, op=BCO, tol=tol, maxit=2000)["x"]
    r = well_means(p, wells_cells) - d
    dJdp = np.zeros_like(p)
    for w, c in enumerate(wells_cells):
        dJdp[np.asarray(c)] += r[w] / len(c)
    lam = orc.pcg(dJdp, op=BCO, tol=tol, maxit=2000)["x"]
    return 0.5 * float(r @ r), tpfa_gradient(prob.nx, prob.ny, prob.nz, logk, prob.kz_ratio, prob.dirichlet, lam, p)


def tpfa_problem(prob) -> Csr:
    return tpfa(prob.nx, prob.ny, prob.nz, prob.logk, prob.kz_ratio, prob.dirichlet)


class OracleError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s (status %d) %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Oracle:
    """The oracle's solver state: AMG hierarchy, IC(0) factor and the preconditioners."""

    def __init__(self, A: Csr, theta=0.12, coarse_max=2048, max_levels=20, gs_natural=False,
                 ic_colour_order=False, openmp=False):
        self.Amat = A
        self._lib = lib(openmp)
        st = ctypes.c_int(0)
        self._h = self._lib.orc_create(A.n, _p(A.rowptr), _p(A.col), _p(A.val), float(theta),
                                   int(coarse_max), int(max_levels), int(gs_natural),
                                   int(ic_colour_order), ctypes.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.n = A.n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return self._lib.orc_nlevels(self._h)

    def level_sizes(self, l):
        s = np.zeros(5, np.int32)
        if self._lib.orc_level_sizes(self._h, l, _p(s)):
            raise IndexError(l)
        return dict(n=int(s[0]), nnz=int(s[1]), ncolours=int(s[2]), nc=int(s[3]), nnzP=int(s[4]))

    def level_A(self, l) -> Csr:
        s = self.level_sizes(l)
        ptr = np.zeros(s["n"] + 1, np.int32)
        col = np.zeros(s["nnz"], np.int32)
        val = np.zeros(s["nnz"], np.float64)
        self._lib.orc_level_A(self._h, l, _p(ptr), _p(col), _p(val))
        return Csr(s["n"], ptr, col, val)

    def level_P(self, l) -> Csr:
        s = self.level_sizes(l)
        ptr = np.zeros(s["n"] + 1, np.int32)
        col = np.zeros(s["nnzP"], np.int32)
        val = np.zeros(s["nnzP"], np.float64)
        if self._lib.orc_level_P(self._h, l, _p(ptr), _p(col), _p(val)):
            raise IndexError(l)
        return Csr(s["n"], ptr, col, val, m=s["nc"])

    def level_cf_colour(self, l):
        n = self.level_sizes(l)["n"]
        cf = np.zeros(n, np.int32)
        colour = np.zeros(n, np.int32)
        if self._lib.orc_level_cf_colour(self._h, l, _p(cf), _p(colour)):
            raise IndexError(l)
        return cf, colour

    def ic0_values(self) -> np.ndarray:
        lu = np.zeros(self.Amat.nnz, np.float64)
        self._lib.orc_ic0_values(self._h, _p(lu))
        return lu

    def level_apply(self, l, op, x) -> np.ndarray:
        x = _f64(x)
        y = np.zeros_like(x)
        if self._lib.orc_level_apply(self._h, l, op, _p(x), _p(y)):
            raise ValueError("level_apply(%d, %d)" % (l, op))
        return y

    def apply(self, op, r) -> np.ndarray:
        r = _f64(r)
        z = np.zeros_like(r)
        if self._lib.orc_apply(self._h, op, _p(r), _p(z)):
            raise ValueError(op)
        return z

    def pcg(self, b, op=BCO, tol=1e-6, maxit=1000):
        """Returns dict(x, iters, status, res_hist, alpha, beta, true_res)."""
        b = _f64(b)
        x = np.zeros_like(b)
        cap = maxit + 1
        hist = np.zeros(cap)
        alpha = np.zeros(cap)
        beta = np.zeros(cap)
        out = np.zeros(2)
        it = ctypes.c_int(0)
        st = self._lib.orc_pcg(self._h, op, _p(b), _p(x), float(tol), int(maxit), ctypes.byref(it),
                           _p(hist), _p(alpha), _p(beta), cap, _p(out))
        k = it.value
        return dict(x=x, iters=k, status=st, res_hist=hist[:k + 1].copy(), alpha=alpha[:k].copy(),
                    beta=beta[:max(k - 1, 0)].copy(), true_res=float(out[0]))


def block_pcg(orc, Bm, op=BCO, tol=1e-6, maxit=500):
    """Block preconditioned CG (O'Leary 1980) on the K columns of Bm (n x K), X_0 = 0.

    Not a method of the paper: the coupled-column counterpart of solving K right-hand sides at
    once, written out step by step.  With gamma_k = Z_k^T R_k:
        Q = A P,  alpha = (P^T Q)^{-1} gamma,  X += P alpha,  R -= Q alpha,
        Z = M R,  beta = gamma_old^{-1} gamma_new,  P = Z + P beta,
    M the oracle's preconditioner `op` applied column by column.  The iteration stops when every
    column has ||r_k||_2 / ||b_k||_2 < tol.  A K x K system that is not numerically positive
    definite -- a Cholesky pivot at or below 1e-12 times its diagonal entry, i.e. a block column
    within rounding of the span of the others (rank-deficient block) -- stops it with status 4.
    Returns dict(X, iters, status, res_hist) with
    res_hist[k, j] the relative residual of column j after k iterations.
    """
    Bm = np.array(Bm, dtype=np.float64)
    n, K = Bm.shape

    def spd(M):
        try:
            L = np.linalg.cholesky(M)
        except np.linalg.LinAlgError:
            return False
        return bool(np.all(np.diag(L) ** 2 > 1e-12 * np.diag(M)))

    def each(opc, V):
        return np.stack([orc.apply(opc, V[:, j]) for j in range(K)], axis=1)

    X = np.zeros_like(Bm)
    R = Bm.copy()
    bn = np.linalg.norm(Bm, axis=0)
    hist = [np.linalg.norm(R, axis=0) / bn]
    if np.all(hist[0] < tol):
        return dict(X=X, iters=0, status=0, res_hist=np.array(hist))
    Z = each(op, R)
    P = Z.copy()
    gamma = Z.T @ R
    for it in range(1, maxit + 1):
        Q = each(A, P)
        PQ = P.T @ Q
        if not (spd(PQ) and spd(gamma)):
            return dict(X=X, iters=it - 1, status=4, res_hist=np.array(hist))
        alpha = np.linalg.solve(PQ, gamma)
        X += P @ alpha
        R -= Q @ alpha
        hist.append(np.linalg.norm(R, axis=0) / bn)
        if np.all(hist[-1] < tol):
            return dict(X=X, iters=it, status=0, res_hist=np.array(hist))
        Z = each(op, R)
        gamma_new = Z.T @ R
        beta = np.linalg.solve(gamma, gamma_new)
        P = Z + P @ beta
        gamma = gamma_new
    return dict(X=X, iters=maxit, status=3, res_hist=np.array(hist))


def lanczos_tridiag(alpha, beta) -> np.ndarray:
    """Lanczos matrix T_k of the preconditioned operator, built from the CG coefficients.

    Diagonal: 1/alpha_0, then 1/alpha_j + beta_{j-1}/alpha_{j-1}; off-diagonal
    sqrt(beta_{j-1})/alpha_{j-1} (the CG-Lanczos relation, Saad 2003, Section 6.7.3).
    Its extreme eigenvalues estimate those of B A, hence kappa(B A).
    """
    k = len(alpha)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alpha[j] + (beta[j - 1] / alpha[j - 1] if j > 0 else 0.0)
        if j > 0:
            T[j, j - 1] = T[j - 1, j] = np.sqrt(beta[j - 1]) / alpha[j - 1]
    return T


def lanczos_extremes(alpha, beta):
    """(lambda_min, lambda_max) of the Lanczos matrix from a CG run."""
    ev = np.linalg.eigvalsh(lanczos_tridiag(alpha, beta))
    return float(ev[0]), float(ev[-1])


def thm22_bound(m0, m1, rho):
    """Theorem 2.2 read for any m0 <= m1: lambda(B_co A) lies in
    [min_{t in [1-rho,1]} (1-m0) t + m0, max_{t in [1-rho,1]} (1-m1) t + m1]; returns (lo, hi, hi/lo).
    For m1 > 1 >= m0 this is exactly Eq. ine:cond."""
    lo = min((1 - m0) * t + m0 for t in (1 - rho, 1.0))
    hi = max((1 - m1) * t + m1 for t in (1 - rho, 1.0))
    return lo, hi, hi / lo
