"""Python binding of the cpc C ABI (``include/cpc.h``): argument marshalling only.

Every step of the solve runs in the CUDA library ``libcpc.so``; this module loads it
with ctypes, passes device pointers of torch tensors and the current CUDA stream, and
turns return codes into exceptions.  There is no CPU fallback: if the library is
missing or no GPU is present, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpc.so")

PRECOND = {"bco": 0, "amg": 1, "ic0": 2, "ilu": 2, "bhat": 3, "none": 4, "amg_ilu": 5}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_bf16": 2}
GS_ORDER = {"multicolour": 0, "natural": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "IC(0) breakdown", 3: "not converged", 4: "CG breakdown",
          5: "CUDA error", 6: "device wait timeout", 7: "AMG setup failure"}
FACE = {"x0": 1, "x1": 2, "y0": 4, "y1": 8, "z0": 16, "z1": 32}


class CpcError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("cpc: %s (code %d) %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class _Options(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("precision", ctypes.c_int32), ("ic_order", ctypes.c_int32),
                ("gs_order", ctypes.c_int32), ("theta", ctypes.c_double), ("coarse_max", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("autotune", ctypes.c_int32),
                ("tail_nnz_max", ctypes.c_int64), ("stream", ctypes.c_void_p)]


_lib = None

# (name, restype, argtypes) of every exported entry point declared in include/cpc.h
_P, _I32, _I64, _F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = [
    ("cpc_default_options", _I32, [_P]),
    ("cpc_tpfa_nnz", _I64, [_I32, _I32, _I32]),
    ("cpc_tpfa_assemble", _I32, [_I32, _I32, _I32, _P, _F64, _I32, _P, _P, _P, _P]),
    ("cpc_tpfa_gradient", _I32, [_I32, _I32, _I32, _P, _F64, _I32, _P, _P, _P, _P]),
    ("cpc_tpfa_assemble_noalloc", _I32, [_I32, _I32, _I32, _P, _F64, _I32, _P, _P, _P, _P]),
    ("cpc_setup", _I32, [_P, _P, _P]),
    ("cpc_destroy", None, [_P]),
    ("cpc_last_error", ctypes.c_char_p, [_P]),
    ("cpc_solve", _I32, [_P, _P, _P, _F64, _I32, _P, _P, _I32]),
    ("cpc_solve_host", _I32, [_P, _P, _P, _F64, _I32, _P, _P, _I32]),
    ("cpc_solve_batched", _I32, [_P, _I32, _P, _P, _F64, _I32, _P, _P]),
    ("cpc_solve_batched_adjoint", _I32, [_P, _I32, _P, _P, _P, _F64, _I32, _P, _P]),
    ("cpc_solve_block", _I32, [_P, _I32, _P, _P, _F64, _I32, _P, _P]),
    ("cpc_check_layouts", _I32, [_P, _P]),
    ("cpc_mhfem_size", _I64, [_I32, _I32, _I32, _I32, _P]),
    ("cpc_mhfem_assemble", _I32, [_I32, _I32, _I32, _P, _F64, _I32, _P, _P, _P, _P]),
    ("cpc_apply_precond", _I32, [_P, _I32, _P, _P]),
    ("cpc_apply_Bcom", _I32, [_P, _P, _P]),
    ("cpc_spmv", _I32, [_P, _P, _P]),
    ("cpc_setup_time_ms", _I32, [_P, _P, _P]),
    ("cpc_solve_launches", _I32, [_P, _P, _P]),
    ("cpc_sweep_time_us", _I32, [_P, _I32, _I32, _P]),
    ("cpc_setup_phases_ms", _I32, [_P, _P, _I32]),
    ("cpc_coarse_inverse_info", _I32, [_P, _P, _P]),
    ("cpc_num_levels", _I32, [_P]),
    ("cpc_level_info", _I32, [_P, _I32, _P]),
    ("cpc_level_layout", _I32, [_P, _I32, _P]),
    ("cpc_level_matrix", _I32, [_P, _I32, _P, _P, _P]),
    ("cpc_level_interp", _I32, [_P, _I32, _P, _P, _P]),
    ("cpc_level_splitting", _I32, [_P, _I32, _P, _P]),
    ("cpc_ic0_values", _I32, [_P, _P]),
    ("cpc_level_apply", _I32, [_P, _I32, _I32, _P, _P]),
]


def load(path: str = LIB_PATH):
    """Load libcpc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise CpcError(5, "libcpc.so not built (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _torch():
    import torch
    return torch


def _check(rc, h=None):
    if rc != 0:
        msg = load().cpc_last_error(h)
        raise CpcError(rc, msg.decode() if msg else "")


def _dptr(t, dtype):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor of %s" % dtype)
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def tpfa_nnz(nx, ny, nz) -> int:
    return int(load().cpc_tpfa_nnz(nx, ny, nz))


def tpfa_assemble(nx, ny, nz, logk, kz_ratio, dirichlet_mask, stream=None):
    """Two-point-flux matrix on the device from a device log-permeability (cpc_tpfa_assemble)."""
    torch = _torch()
    n = nx * ny * nz
    nnz = tpfa_nnz(nx, ny, nz)
    dev = logk.device
    rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    _check(load().cpc_tpfa_assemble(nx, ny, nz, _dptr(logk, torch.float64), float(kz_ratio), int(dirichlet_mask),
                                    _dptr(rowptr, torch.int32), _dptr(col, torch.int32),
                                    _dptr(val, torch.float64), _stream_ptr(stream)))
    return rowptr, col, val


def mhfem_size(nx, ny, nz, dirichlet_mask):
    """(unknowns, nnz) of the mixed-hybrid system (cpc_mhfem_size)."""
    nu = ctypes.c_int64(0)
    nnz = int(load().cpc_mhfem_size(nx, ny, nz, int(dirichlet_mask), ctypes.byref(nu)))
    if nnz < 0:
        raise CpcError(1, "grid too large for int32 indices")
    return int(nu.value), nnz


def mhfem_assemble(nx, ny, nz, logk, kz_ratio, dirichlet_mask, stream=None):
    """Mixed-hybrid (p, lambda) matrix on the device from a device log-permeability (cpc_mhfem_assemble)."""
    torch = _torch()
    nu, nnz = mhfem_size(nx, ny, nz, dirichlet_mask)
    dev = logk.device
    rowptr = torch.empty(nu + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    _check(load().cpc_mhfem_assemble(nx, ny, nz, _dptr(logk, torch.float64), float(kz_ratio), int(dirichlet_mask),
                                     _dptr(rowptr, torch.int32), _dptr(col, torch.int32),
                                     _dptr(val, torch.float64), _stream_ptr(stream)))
    return rowptr, col, val


def tpfa_gradient(nx, ny, nz, logk, kz_ratio, dirichlet_mask, lam, p, g=None, stream=None):
    """g = -lambda^T (dA/dlog k) p on the device (cpc_tpfa_gradient)."""
    torch = _torch()
    if g is None:
        g = torch.empty_like(p)
    _check(load().cpc_tpfa_gradient(nx, ny, nz, _dptr(logk, torch.float64), float(kz_ratio), int(dirichlet_mask),
                                    _dptr(lam, torch.float64), _dptr(p, torch.float64), _dptr(g, torch.float64),
                                    _stream_ptr(stream)))
    return g


def tpfa_assemble_noalloc(nx, ny, nz, logk, kz_ratio, dirichlet_mask, rowptr, col, val, stream=None):
    """As tpfa_assemble, into caller-provided device tensors, with no device allocation inside
    the library (cpc_tpfa_assemble_noalloc).  Returns the C status code."""
    torch = _torch()
    return int(load().cpc_tpfa_assemble_noalloc(nx, ny, nz, _dptr(logk, torch.float64), float(kz_ratio),
                                                int(dirichlet_mask), _dptr(rowptr, torch.int32),
                                                _dptr(col, torch.int32), _dptr(val, torch.float64),
                                                _stream_ptr(stream)))


class Solver:
    """Combined-preconditioned CG solver on one GPU (a cpc handle).

    ``rowptr, col, val`` are CSR arrays: CUDA tensors (int32, int32, float64) or
    numpy arrays on the host.
    """

    def __init__(self, rowptr, col, val, precond="bco", precision="fp64", ic_order="natural", theta=0.12,
                 coarse_max=2048, max_levels=20, tail_nnz_max=0, autotune=False, gs_order="multicolour",
                 stream=None):
        torch = _torch()
        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = int(rowptr.shape[0]) - 1
        nnz = int(col.shape[0])
        if isinstance(rowptr, np.ndarray):
            self._host = (np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(col, np.int32),
                          np.ascontiguousarray(val, np.float64))
            ptrs = [ctypes.c_void_p(a.ctypes.data) for a in self._host]
            on_dev = 0
        else:
            ptrs = [_dptr(rowptr, torch.int32), _dptr(col, torch.int32), _dptr(val, torch.float64)]
            on_dev = 1
        csr = _Csr(n, nnz, ptrs[0], ptrs[1], ptrs[2], on_dev)
        opt = _Options()
        lib.cpc_default_options(ctypes.byref(opt))
        opt.precond = PRECOND[precond]
        opt.precision = PRECISION[precision]
        opt.ic_order = {"natural": 0, "colour": 1}[ic_order]
        opt.gs_order = GS_ORDER[gs_order]
        opt.theta = float(theta)
        opt.coarse_max = int(coarse_max)
        opt.max_levels = int(max_levels)
        opt.tail_nnz_max = int(tail_nnz_max)
        opt.autotune = 1 if autotune else 0
        opt.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        _check(lib.cpc_setup(ctypes.byref(csr), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.nnz = nnz
        self.precond = precond
        self.precision = precision
        self.ic_order = ic_order
        self.gs_order = gs_order

    def close(self):
        if getattr(self, "_h", None):
            load().cpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solve --------------------------------------------------------------------------------
    def solve(self, b, tol=1e-6, maxit=1000, x=None, hist=True):
        """PCG from x0 = 0 on device vectors; returns (x, iters, status, res_hist)."""
        torch = _torch()
        if x is None:
            x = torch.empty_like(b)
        it = ctypes.c_int32(0)
        cap = maxit + 1 if hist else 0
        h = np.zeros(max(cap, 1))
        rc = load().cpc_solve(self._h, _dptr(b, torch.float64), _dptr(x, torch.float64), float(tol), int(maxit),
                              ctypes.byref(it), ctypes.c_void_p(h.ctypes.data) if hist else None, cap)
        if rc not in (0, 3, 4):
            _check(rc, self._h)
        k = it.value
        return x, k, rc, (h[:k + 1].copy() if hist else None)

    def solve_host(self, b_host, x_host, tol=1e-6, maxit=1000):
        """PCG with b and x in host memory (numpy arrays or pinned CPU tensors)."""
        it = ctypes.c_int32(0)
        pb = b_host.ctypes.data if isinstance(b_host, np.ndarray) else b_host.data_ptr()
        px = x_host.ctypes.data if isinstance(x_host, np.ndarray) else x_host.data_ptr()
        rc = load().cpc_solve_host(self._h, ctypes.c_void_p(pb), ctypes.c_void_p(px), float(tol), int(maxit),
                                   ctypes.byref(it), None, 0)
        if rc not in (0, 3, 4):
            _check(rc, self._h)
        return it.value, rc

    def solve_batched(self, B, tol=1e-6, maxit=1000, X=None):
        """PCG on the columns of B ([n, K] CUDA float64, row-major); returns (X, iters[K], status[K])."""
        torch = _torch()
        if X is None:
            X = torch.empty_like(B)
        K = int(B.shape[1])
        it = np.zeros(K, np.int32)
        st = np.zeros(K, np.int32)
        _check(load().cpc_solve_batched(self._h, K, _dptr(B, torch.float64), _dptr(X, torch.float64), float(tol),
                                        int(maxit), ctypes.c_void_p(it.ctypes.data), ctypes.c_void_p(st.ctypes.data)),
               self._h)
        return X, it, st

    def solve_block(self, B, tol=1e-6, maxit=1000, X=None, check=True):
        """Block PCG on the columns of B ([n, K] CUDA float64, K <= 64); returns (X, iters, res[K], status).
        With check, a status other than ok / not converged raises."""
        torch = _torch()
        if X is None:
            X = torch.empty_like(B)
        K = int(B.shape[1])
        it = ctypes.c_int32(0)
        res = np.zeros(K, np.float64)
        rc = load().cpc_solve_block(self._h, K, _dptr(B, torch.float64), _dptr(X, torch.float64), float(tol),
                                    int(maxit), ctypes.byref(it), ctypes.c_void_p(res.ctypes.data))
        if check and rc not in (0, 3):
            _check(rc, self._h)
        return X, it.value, res, rc

    def solve_batched_adjoint(self, B, tol=1e-6, maxit=1000, X=None, Lam=None):
        """Forward solves of B's columns, then adjoint solves with sources X at B's nonzeros (one graph)."""
        torch = _torch()
        X = torch.empty_like(B) if X is None else X
        Lam = torch.empty_like(B) if Lam is None else Lam
        K = int(B.shape[1])
        itf = np.zeros(K, np.int32)
        ita = np.zeros(K, np.int32)
        _check(load().cpc_solve_batched_adjoint(self._h, K, _dptr(B, torch.float64), _dptr(X, torch.float64),
                                                _dptr(Lam, torch.float64), float(tol), int(maxit),
                                                ctypes.c_void_p(itf.ctypes.data), ctypes.c_void_p(ita.ctypes.data)),
               self._h)
        return X, Lam, itf, ita

    def apply(self, r, which=None, z=None):
        """z = M r for one preconditioner application (which: name or None for the handle's)."""
        torch = _torch()
        if z is None:
            z = torch.empty_like(r)
        w = -1 if which is None else PRECOND[which]
        _check(load().cpc_apply_precond(self._h, w, _dptr(r, torch.float64), _dptr(z, torch.float64)), self._h)
        return z

    def apply_Bcom(self, r, z=None):
        torch = _torch()
        if z is None:
            z = torch.empty_like(r)
        _check(load().cpc_apply_Bcom(self._h, _dptr(r, torch.float64), _dptr(z, torch.float64)), self._h)
        return z

    def spmv(self, x, y=None):
        torch = _torch()
        if y is None:
            y = torch.empty_like(x)
        _check(load().cpc_spmv(self._h, _dptr(x, torch.float64), _dptr(y, torch.float64)), self._h)
        return y

    def setup_time_ms(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load().cpc_setup_time_ms(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    # -- inspection ------------------------------------------------------------------------------
    def solve_launches(self):
        """(kernel launches per PCG iteration, launches outside the loop) of cpc_solve."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().cpc_solve_launches(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    def setup_phases_ms(self):
        """AMG setup phases in ms: coarsening, colouring, coarsest inverse, layouts."""
        ms = np.zeros(4)
        _check(load().cpc_setup_phases_ms(self._h, ctypes.c_void_p(ms.ctypes.data), 4), self._h)
        return dict(zip(("coarsening", "colouring", "coarsest_inverse", "layouts"), [float(v) for v in ms]))

    def coarse_inverse_info(self):
        """(method, residual) of the coarsest level's inverse: method 1 = FP32 Cholesky inverse with
        Newton-Schulz refinement, 0 = FP64 Cholesky inverse; residual = max |I - A_c X|."""
        m, r = ctypes.c_int32(), ctypes.c_double()
        _check(load().cpc_coarse_inverse_info(self._h, ctypes.byref(m), ctypes.byref(r)), self._h)
        return m.value, r.value

    def sweep_time_us(self, l, reps=20):
        """Microseconds per forward Gauss-Seidel sweep of level l, replayed from a CUDA graph."""
        us = ctypes.c_double()
        _check(load().cpc_sweep_time_us(self._h, l, reps, ctypes.byref(us)), self._h)
        return us.value

    @property
    def nlevels(self) -> int:
        return int(load().cpc_num_levels(self._h))

    def level_info(self, l):
        info = np.zeros(6, np.int64)
        _check(load().cpc_level_info(self._h, l, ctypes.c_void_p(info.ctypes.data)), self._h)
        return dict(n=int(info[0]), nnz=int(info[1]), ncolours=int(info[2]), nc=int(info[3]), nnzP=int(info[4]),
                    ic_levels=int(info[5]))

    def level_layout(self, l):
        """Smoother storage of A_l: chunk height, stored diagonals (0 = SELL), slots; level 0 also
        the natural-order copy (nat_*)."""
        info = np.zeros(6, np.int64)
        _check(load().cpc_level_layout(self._h, l, ctypes.c_void_p(info.ctypes.data)), self._h)
        return dict(C=int(info[0]), ndiag=int(info[1]), nslots=int(info[2]), nat_C=int(info[3]),
                    nat_ndiag=int(info[4]), nat_nslots=int(info[5]))

    def level_matrix(self, l):
        i = self.level_info(l)
        ptr = np.zeros(i["n"] + 1, np.int32)
        col = np.zeros(max(i["nnz"], 1), np.int32)
        val = np.zeros(max(i["nnz"], 1), np.float64)
        _check(load().cpc_level_matrix(self._h, l, ctypes.c_void_p(ptr.ctypes.data), ctypes.c_void_p(col.ctypes.data),
                                       ctypes.c_void_p(val.ctypes.data)), self._h)
        return ptr, col[:i["nnz"]], val[:i["nnz"]]

    def level_interp(self, l):
        i = self.level_info(l)
        ptr = np.zeros(i["n"] + 1, np.int32)
        col = np.zeros(max(i["nnzP"], 1), np.int32)
        val = np.zeros(max(i["nnzP"], 1), np.float64)
        _check(load().cpc_level_interp(self._h, l, ctypes.c_void_p(ptr.ctypes.data), ctypes.c_void_p(col.ctypes.data),
                                       ctypes.c_void_p(val.ctypes.data)), self._h)
        return ptr, col[:i["nnzP"]], val[:i["nnzP"]]

    def check_layouts(self):
        """Structural check of the handle's device layouts (cpc_check_layouts): dict of counts."""
        c = np.zeros(5, np.int64)
        _check(load().cpc_check_layouts(self._h, ctypes.c_void_p(c.ctypes.data)), self._h)
        return dict(out_of_range=int(c[0]), coverage=int(c[1]), gs_races=int(c[2]), triangular_races=int(c[3]),
                    layouts=int(c[4]))

    def level_splitting(self, l):
        n = self.level_info(l)["n"]
        cf = np.zeros(n, np.int32)
        colour = np.zeros(n, np.int32)
        _check(load().cpc_level_splitting(self._h, l, ctypes.c_void_p(cf.ctypes.data),
                                          ctypes.c_void_p(colour.ctypes.data)), self._h)
        return cf, colour

    def ic0_values(self):
        lu = np.zeros(self.nnz, np.float64)
        _check(load().cpc_ic0_values(self._h, ctypes.c_void_p(lu.ctypes.data)), self._h)
        return lu

    def level_apply(self, l, op, x, y=None):
        torch = _torch()
        if y is None:
            y = torch.empty_like(x)
        _check(load().cpc_level_apply(self._h, l, op, _dptr(x, torch.float64), _dptr(y, torch.float64)), self._h)
        return y
