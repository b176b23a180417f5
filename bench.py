"""Benchmark: PCG solve time to a 1e-6 relative residual on one GB300.

Headline (``value``): milliseconds per combined-preconditioned (B_co) PCG solve, FP64, on the
128 x 128 x 64 correlated-lognormal two-point-flux matrix (1,048,576 unknowns), inputs resident
in HBM.  The same run times the AMG-alone (S~, two V-cycles) and IC(0)-alone preconditioners and
the FP32 / FP32+BF16 preconditioner variants, the end-to-end solve through host buffers, the
dominant kernel against the measured HBM roofline, and the CPU oracle as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own copy of the problem (independent replicas,
weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1205_6113_gb300 import inputs  # noqa: E402

WORKLOAD = "correlated3d_128x128x64"
TOL = 1e-6
MAXIT = 5000
METRIC = "PCG ms to 1e-6 rel. residual (combined vs AMG/ILU alone, FP32 vs FP64 prec), %HBM peak"
L2_FLUSH_BYTES = 512 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one fine-level Gauss-Seidel launch from the
# committed ncu capture (profiles/k_gs_pk_fine_correlated3d_128x128x64.md); None until a capture
# of the current kernel exists.
TRAFFIC_K_GS_FINE = 48355584


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
                for nm, v in zip(names, s[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# algorithmic bytes (compulsory traffic of each kernel, counted from the data structures)
# ------------------------------------------------------------------------------------------------
def a_pass_bytes(n, nnz, sv=8, sx=8):
    """One sweep over a sparse matrix: values + column indices + row pointers, read x, write y."""
    return nnz * (sv + 4) + 4 * (n + 1) + 2 * n * sx


def dia_pass_bytes(n, nd, sv=8, sx=8):
    """One sweep over a matrix in diagonal form: nd stored diagonals + the diagonal, read x, write y."""
    return n * (nd * sv + sv + 2 * sx)


def bytes_per_iteration(s, precond, sv=8, sx=8, sv_coarse=None):
    sv_coarse = sv if sv_coarse is None else sv_coarse
    nl = s.nlevels
    info = [s.level_info(l) for l in range(nl)]
    lay0 = s.level_layout(0)

    def a_pass(l, svl):
        i = info[l]
        if l == 0 and lay0["ndiag"]:
            return dia_pass_bytes(i["n"], lay0["ndiag"], svl, sx)
        return a_pass_bytes(i["n"], i["nnz"], svl, sx)

    def vcycle(ilu_fine=False):
        b = 0
        for l in range(nl - 1):
            i = info[l]
            svl = sv if l == 0 else sv_coarse
            b += 3 * a_pass(l, svl)                                     # pre sweep, residual, post sweep
            if l == 0 and ilu_fine:                                     # + the two IC(0) solves
                b += 2 * a_pass_bytes(i["n"], i["nnz"], svl, sx)
            b += 2 * a_pass_bytes(i["n"], i["nnzP"], 4 if sx == 4 else 8, sx)   # restriction, prolongation
        c = info[nl - 1]["n"]
        b += c * c * sx
        return b

    n, nnz = info[0]["n"], info[0]["nnz"]
    ic = a_pass_bytes(n, nnz, sv, sx)                                   # L and U together touch A's pattern once
    nat = dia_pass_bytes(n, lay0["nat_ndiag"], 8, 8) if lay0["nat_ndiag"] else a_pass_bytes(n, nnz, 8, 8)
    pcg = nat + 12 * n * 8                                              # q = A p plus the vector updates
    if precond == "bco":
        if lay0["ndiag"] and s.ic_order == "colour":                    # step (2): one pass over the black rows
            return pcg + 2 * vcycle() + dia_pass_bytes(n // 2, lay0["ndiag"], sv, sx) + n // 2 * sx
        return pcg + 2 * vcycle() + a_pass_bytes(n, nnz, sv, sx) + ic
    if precond == "amg":
        return pcg + 2 * vcycle()
    if precond == "ic0":
        return pcg + ic
    if precond == "bhat":
        return pcg + 2 * vcycle() + ic
    if precond == "amg_ilu":
        return pcg + 2 * vcycle(ilu_fine=True)
    return pcg


class SolveFailed(RuntimeError):
    def __init__(self, status, iters):
        super().__init__("solve failed with status %d after %d iterations" % (status, iters))
        self.status, self.iters = status, iters


# ------------------------------------------------------------------------------------------------
def gpu_arm(args, rank, world):
    import torch
    from paper_1205_6113_gb300 import cpc

    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    p = inputs.workload(WORKLOAD)
    logk = torch.tensor(p.logk, device=dev)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    b = torch.tensor(p.rhs(), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        flush.fill_(1.0)

    def dist_barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def time_solves(solver, steps, warmup, tol=TOL):
        iters = []
        for _ in range(warmup):
            _, it, st, _ = solver.solve(b, tol=tol, maxit=MAXIT, hist=False)
            if st != 0:
                raise SolveFailed(st, it)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        dist_barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush_l2()
            ev[k][0].record(stream)
            _, it, st, _ = solver.solve(b, tol=tol, maxit=MAXIT, hist=False)
            ev[k][1].record(stream)
            if st != 0:
                raise SolveFailed(st, it)
            iters.append(it)
        torch.cuda.synchronize()
        dist_barrier()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(c) for a, c in ev]
        return ms, iters, wall

    out = {}
    # headline arm: B_co, FP64
    setups = {}
    t = time.perf_counter()
    s_bco = cpc.Solver(rowptr, col, val, precond="bco", precision="fp64", ic_order="colour")
    setups["bco_fp64"] = dict(zip(("ic0_ms", "amg_ms"), s_bco.setup_time_ms()))
    setups["bco_fp64"]["wall_ms"] = (time.perf_counter() - t) * 1e3
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms, iters, wall = time_solves(s_bco, args.steps, args.warmup)
    clk = clocks.stop()
    out["headline"] = dict(ms=ms, iters=iters, wall=wall)

    # end-to-end through the C ABI with host buffers (pinned): H2D of b, D2H of x inside the timed region
    b_host = torch.tensor(p.rhs()).pin_memory()
    x_host = torch.empty(p.n, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        s_bco.solve_host(b_host, x_host, tol=TOL, maxit=MAXIT)
    e2e_ms = []
    for _ in range(args.steps):
        flush_l2()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, st = s_bco.solve_host(b_host, x_host, tol=TOL, maxit=MAXIT)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert st == 0
    xh = x_host.numpy()
    true_res = float(np.linalg.norm(p.rhs() - csr_matvec(rowptr, col, val, xh)) / np.linalg.norm(p.rhs()))

    # comparison arms (fewer steps: AMG-alone and IC(0)-alone)
    arms = {}
    # (name, preconditioner, precision, IC(0) order, Gauss-Seidel order, timed solves)
    for name, pre, prec, ico, gso, k in [
            ("amg_fp64", "amg", "fp64", "natural", "multicolour", args.steps),
            ("ic0_fp64", "ic0", "fp64", "natural", "multicolour", 2),
            ("ic0_rbic_fp64", "ic0", "fp64", "colour", "multicolour", 2),
            ("bco_natic_fp64", "bco", "fp64", "natural", "multicolour", args.steps),
            ("bco_natgs_fp64", "bco", "fp64", "natural", "natural", 2),
            ("bhat_fp64", "bhat", "fp64", "colour", "multicolour", args.steps),
            ("amg_ilu_fp64", "amg_ilu", "fp64", "colour", "multicolour", args.steps),
            ("bco_fp32", "bco", "fp32", "colour", "multicolour", args.steps),
            ("bco_fp32_bf16", "bco", "fp32_bf16", "colour", "multicolour", args.steps),
            ("amg_fp32", "amg", "fp32", "natural", "multicolour", args.steps)]:
        if world > 1:
            continue
        t = time.perf_counter()
        s = cpc.Solver(rowptr, col, val, precond=pre, precision=prec, ic_order=ico, gs_order=gso)
        setup = dict(zip(("ic0_ms", "amg_ms"), s.setup_time_ms()))
        setup["wall_ms"] = (time.perf_counter() - t) * 1e3
        try:
            slow = name in ("ic0_fp64", "ic0_rbic_fp64", "bco_natgs_fp64")      # one warm-up solve
            m, it, _ = time_solves(s, k, 1 if slow else args.warmup)
        except SolveFailed as e:                 # AMG(ILU(0)) need not be SPD (Section 5): record it
            arms[name] = dict(ms=None, iters=e.iters, status=e.status, setup=setup)
            s.close()
            continue
        x, _, _, _ = s.solve(b, tol=TOL, maxit=MAXIT, hist=False)
        xr = x.cpu().numpy()
        arms[name] = dict(ms=round(float(np.mean(m)), 3), iters=int(it[-1]), setup=setup,
                          true_res=float(np.linalg.norm(p.rhs() - csr_matvec(rowptr, col, val, xr)) / np.linalg.norm(p.rhs())),
                          hbm_frac_solve=None)
        bpi = bytes_per_iteration(s, pre, sv=8 if prec == "fp64" else 4, sx=8 if prec == "fp64" else 4,
                                  sv_coarse=(2 if prec == "fp32_bf16" else None))
        arms[name]["gbs_solve"] = round(bpi * it[-1] / (np.mean(m) * 1e-3) / 1e9, 1)
        s.close()

    # batched: 64 right-hand sides and their adjoints in one graph, FP32 preconditioner
    if world == 1 and not args.no_batched:
        out["batched"] = batched_arm(rowptr, col, val, p, dev, stream, args)

    # the mixed-hybrid system of the same grid (second matrix family), assembled on the device
    if world == 1 and not args.no_mhfem:
        out["mhfem"] = mhfem_arm(p, dev, stream, args)

    # differentiable solve on the 256 x 256 x 128 channel problem: gradient of the well misfit
    if world == 1 and not args.no_adjoint:
        out["adjoint"] = adjoint_arm(dev, stream)

    # dominant kernel (k_gs, the Gauss-Seidel colour sweep: largest share of the ncu launch list):
    # its fine-level launches timed live -- one red and one black launch per event pair, L2 flushed.
    # Algorithmic bytes per launch: half of (24 n + 12 nnz) = the colour's rows of A (values,
    # columns), diagonal, perm, f, x written, and the other colour's x read once.
    xv = torch.randn(p.n, dtype=torch.float64, device=dev)
    yv = torch.zeros_like(xv)
    info0 = s_bco.level_info(0)
    for _ in range(3):
        s_bco.level_apply(0, 5, xv, yv)
    kms = []
    for _ in range(20):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_bco.level_apply(0, 5, xv, yv)
        e1.record(stream)
        torch.cuda.synchronize()
        kms.append(e0.elapsed_time(e1) / info0["ncolours"])
    lay0 = s_bco.level_layout(0)
    if lay0["ndiag"]:       # per row: nd diagonals, 1/a_ii, slot -> row, f_i, x_i written, the other colour's x once
        kbytes = info0["n"] * (8 * lay0["ndiag"] + 36) // info0["ncolours"]
        kname = "k_gs_pk (Gauss-Seidel colour sweep, fine level, red/black, per-slot diagonal records, FP64)"
    else:                   # per row / entry: SELL values + columns, 1/a_ii, f_i, x_i
        kbytes = (24 * info0["n"] + 12 * info0["nnz"]) // info0["ncolours"]
        kname = "k_gs (Gauss-Seidel colour sweep, fine level, red/black, SELL, FP64)"
    peak, peak_kind = peaks()
    k_avg = float(np.mean(kms))
    achieved = kbytes / (k_avg * 1e-3) / 1e9
    # the fine SpMV (same SELL layout), for reference
    sms = []
    for _ in range(20):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_bco.spmv(xv, yv)
        e1.record(stream)
        torch.cuda.synchronize()
        sms.append(e0.elapsed_time(e1))
    if lay0["nat_ndiag"]:
        sbytes = dia_pass_bytes(info0["n"], lay0["nat_ndiag"])
        sname = "k_spmv_dia (fine A, natural order, diagonal form, FP64)"
    else:
        sbytes = a_pass_bytes(info0["n"], info0["nnz"])
        sname = "k_spmv (fine A, SELL-32, FP64)"
    spmv = dict(kernel=sname, bytes_per_launch=sbytes, avg_launch_ms=round(float(np.mean(sms)), 5),
                achieved=round(sbytes / (np.mean(sms) * 1e-3) / 1e9, 1))
    # the coarse colour steps (the largest share of kernel time): one forward sweep per level timed
    # live; algorithmic bytes per sweep = 12 B per off-diagonal entry + 28 B per row (1 / a_ii,
    # slot -> row, f, x written, x read); these steps are bound by dependent-launch latency
    coarse = []
    for l in range(1, s_bco.nlevels - 1):
        inf = s_bco.level_info(l)
        xl = torch.randn(inf["n"], dtype=torch.float64, device=dev)
        yl = torch.zeros_like(xl)
        for _ in range(3):
            s_bco.level_apply(l, 1, xl, yl)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            s_bco.level_apply(l, 1, xl, yl)
        e1.record(stream)
        torch.cuda.synchronize()
        sweep_ms = e0.elapsed_time(e1) / reps
        nbytes = 12 * (inf["nnz"] - inf["n"]) + 28 * inf["n"]
        coarse.append(dict(level=l, n=inf["n"], colours=inf["ncolours"],
                           us_per_step=round(sweep_ms * 1e3 / inf["ncolours"], 2),
                           achieved=round(nbytes / (sweep_ms * 1e-3) / 1e9, 1)))
    coarse_gs = dict(kernel="k_gs (coarse colour steps, FP64, one forward sweep per level)", bound="latency",
                     unit="GB/s", levels=coarse)
    bpi = bytes_per_iteration(s_bco, "bco")
    headline_ms = float(np.mean(ms))
    out.update(dict(p=p, arms=arms, clocks=clk, e2e_ms=e2e_ms, true_res=true_res, setups=setups,
                    roofline=dict(bound="hbm", achieved=round(achieved, 1), peak=peak, unit="GB/s",
                                  frac=round(achieved / peak, 4), traffic=TRAFFIC_K_GS_FINE,
                                  kernel=kname,
                                  bytes_per_launch=kbytes, avg_launch_ms=round(k_avg, 5), peak_kind=peak_kind,
                                  spmv=spmv, coarse_gs=coarse_gs),
                    headline_ms=headline_ms, bytes_per_iter=bpi, nodes=None, nlevels=s_bco.nlevels,
                    levels=[s_bco.level_info(l) for l in range(s_bco.nlevels)]))
    out["solve_gbs"] = bpi * iters[-1] / (headline_ms * 1e-3) / 1e9
    out["launches"] = s_bco.solve_launches()
    return out


def batched_arm(rowptr, col, val, p, dev, stream, args, K=64):
    """64 right-hand sides (rates U[-1,1] at 16 random cells each) plus their adjoints as one
    graph-captured batched solve, against the same 64 forward solves one at a time."""
    import torch
    from paper_1205_6113_gb300 import cpc
    s = cpc.Solver(rowptr, col, val, precond="bco", precision="fp32", ic_order="colour", autotune=True)
    chunk = [s.level_layout(l)["C"] for l in range(s.nlevels - 1)]
    B = torch.tensor(np.ascontiguousarray(inputs.batch_rhs(p.n, K, seed=5).T), device=dev)
    X = torch.empty_like(B)
    Lam = torch.empty_like(B)
    s.solve_batched_adjoint(B, tol=TOL, maxit=MAXIT, X=X, Lam=Lam)
    steps = max(1, min(args.steps, 3))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        _, _, itf, ita = s.solve_batched_adjoint(B, tol=TOL, maxit=MAXIT, X=X, Lam=Lam)
    ev[1].record(stream)
    torch.cuda.synchronize()
    bat_ms = ev[0].elapsed_time(ev[1]) / steps
    fwd_only = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.solve_batched(B, tol=TOL, maxit=MAXIT, X=X)
    torch.cuda.synchronize()
    e0.record(stream)
    s.solve_batched(B, tol=TOL, maxit=MAXIT, X=X)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_batched_ms = e0.elapsed_time(e1)
    # block PCG (O'Leary) on the same 64 columns: coupled through K x K FP64 Gram matrices
    s.solve_block(B, tol=TOL, maxit=MAXIT, X=X)
    torch.cuda.synchronize()
    e0.record(stream)
    _, blk_it, blk_res, blk_st = s.solve_block(B, tol=TOL, maxit=MAXIT, X=X)
    e1.record(stream)
    torch.cuda.synchronize()
    block_ms = e0.elapsed_time(e1)
    cols = [B[:, k].contiguous() for k in range(K)]
    s.solve(cols[0], tol=TOL, maxit=MAXIT, hist=False)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(K):
        _, it, st, _ = s.solve(cols[k], tol=TOL, maxit=MAXIT, hist=False)
        fwd_only.append(it)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    s.close()
    return dict(workload=WORKLOAD + "_64rhs", nrhs=K, precision="fp32 preconditioner",
                batched_fwd_adj_ms=round(bat_ms, 2), batched_solves_per_s=round(2 * K / (bat_ms * 1e-3), 1),
                batched_fwd_ms=round(fwd_batched_ms, 2), batched_fwd_solves_per_s=round(K / (fwd_batched_ms * 1e-3), 1),
                sequential_fwd_ms=round(seq_ms, 2), sequential_solves_per_s=round(K / (seq_ms * 1e-3), 1),
                iters_fwd=[int(itf.min()), int(itf.max())], iters_adj=[int(ita.min()), int(ita.max())],
                iters_sequential=[int(min(fwd_only)), int(max(fwd_only))],
                block_cg_fwd_ms=round(block_ms, 2), block_cg_solves_per_s=round(K / (block_ms * 1e-3), 1),
                block_cg_iters=int(blk_it), block_cg_status=int(blk_st), block_cg_max_res=float(np.max(blk_res)),
                chunk_height_autotuned=chunk)


def mhfem_arm(p, dev, stream, args):
    """The mixed-hybrid (p, lambda) system of the same grid (Section 4, Eq. alge_sys), assembled on
    the device: cell sources, 0 on faces; B_co and AMG alone in FP64, B_co with the FP32
    preconditioner.  IC(0) alone is left out (over a thousand iterations at this size)."""
    import torch
    from paper_1205_6113_gb300 import cpc
    logk = torch.tensor(p.logk, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cpc.mhfem_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    torch.cuda.synchronize()
    e0.record(stream)
    rowptr, col, val = cpc.mhfem_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    e1.record(stream)
    torch.cuda.synchronize()
    asm_ms = e0.elapsed_time(e1)
    nu = int(rowptr.shape[0]) - 1
    b = torch.zeros(nu, dtype=torch.float64, device=dev)
    b[:p.n] = torch.tensor(p.rhs(), device=dev)
    out = dict(workload=WORKLOAD + "_mhfem", unknowns=nu, nnz=int(col.shape[0]), assembly_ms=round(asm_ms, 3))
    steps = max(1, min(args.steps, 3))
    for name, pre, prec in [("bco_fp64", "bco", "fp64"), ("amg_fp64", "amg", "fp64"), ("bco_fp32", "bco", "fp32")]:
        t = time.perf_counter()
        s = cpc.Solver(rowptr, col, val, precond=pre, precision=prec, ic_order="colour")
        setup_ms = (time.perf_counter() - t) * 1e3
        x, it, st, _ = s.solve(b, tol=TOL, maxit=MAXIT, hist=False)
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            e0.record(stream)
            x, it, st, _ = s.solve(b, tol=TOL, maxit=MAXIT, hist=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        xr = x.cpu().numpy()
        res = float(np.linalg.norm(b.cpu().numpy() - csr_matvec(rowptr, col, val, xr)) / np.linalg.norm(b.cpu().numpy()))
        out[name] = dict(ms=round(float(np.mean(ms)), 3), iters=int(it), status=int(st), setup_wall_ms=round(setup_ms, 1),
                         levels=s.nlevels, true_res=res)
        s.close()
    return out


def adjoint_arm(dev, stream, tol=1e-8):
    """dJ/dlog k for J = 1/2 sum_w (mean_w p - d_w)^2 on channels3d_256x256x128: assembly + setup,
    forward solve, adjoint solve (same handle) and the gradient kernel, each timed with CUDA events."""
    import torch
    from paper_1205_6113_gb300 import adjoint, cpc
    p = inputs.workload("channels3d_256x256x128")
    grid = adjoint.Grid(p.nx, p.ny, p.nz, p.kz_ratio, p.dirichlet)
    cells = torch.tensor(inputs.well_columns(p), device=dev, dtype=torch.int64)
    q = torch.tensor(p.rhs(), device=dev)
    with torch.no_grad():
        d = adjoint.well_pressures(adjoint.pressure(torch.tensor(inputs.perturbed_logk(p), device=dev), q, grid,
                                                    tol=tol), cells)
    logk = torch.tensor(p.logk, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    s = cpc.Solver(rowptr, col, val, precond="bco", ic_order="colour")
    ev[1].record(stream)
    x, it_f, st_f, _ = s.solve(q, tol=tol, maxit=MAXIT, hist=False)
    ev[2].record(stream)
    r = adjoint.well_pressures(x, cells) - d
    dJdp = torch.zeros_like(x)
    dJdp.index_add_(0, cells.reshape(-1), (r / cells.shape[1]).repeat_interleave(cells.shape[1]))
    ev[3].record(stream)
    lam, it_a, st_a, _ = s.solve(dJdp, tol=tol, maxit=MAXIT, hist=False)
    g = cpc.tpfa_gradient(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet, lam, x)
    ev[4].record(stream)
    torch.cuda.synchronize()
    # the gradient pass alone (bytes: log k read, k written and read, lambda, p read, g written)
    kms = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cpc.tpfa_gradient(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet, lam, x, g)
        e1.record(stream)
        torch.cuda.synchronize()
        kms.append(e0.elapsed_time(e1))
    kbytes = 6 * 8 * p.n
    res = dict(workload="channels3d_256x256x128", n=p.n, tol=tol, status=(st_f, st_a), iters=(it_f, it_a),
               setup_ms=round(ev[0].elapsed_time(ev[1]), 2), forward_ms=round(ev[1].elapsed_time(ev[2]), 2),
               adjoint_and_gradient_ms=round(ev[3].elapsed_time(ev[4]), 2),
               gradient_kernel_ms=round(float(np.median(kms)), 4),
               gradient_kernel_gbs=round(kbytes / (np.median(kms) * 1e-3) / 1e9, 1),
               misfit=float(0.5 * (r * r).sum()), grad_norm=float(g.norm()))
    s.close()
    return res


def csr_matvec(rowptr, col, val, x):
    rp = rowptr.cpu().numpy()
    c = col.cpu().numpy()
    v = val.cpu().numpy()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return np.bincount(rows, weights=v * x[c], minlength=len(rp) - 1)


def oracle_time(p, sample_iters=None):
    """The oracle (single thread, FP64) on the same matrix: setup once, then one B_co PCG solve."""
    import oracle as O
    A = O.tpfa_problem(p)
    t = time.perf_counter()
    orc = O.Oracle(A)
    setup_s = time.perf_counter() - t
    t = time.perf_counter()
    r = orc.pcg(p.rhs(), op=O.BCO, tol=TOL, maxit=sample_iters or MAXIT)
    solve_s = time.perf_counter() - t
    return orc, r, setup_s, solve_s


def reference_arm(args, rank, world):
    """CPU oracle timed on the host cores (the reference arm: the paper has no code of its own)."""
    import oracle as O
    if rank != 0:
        return
    p = inputs.workload(WORKLOAD)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A)
    sample = 4
    full_iters = orc.pcg(p.rhs(), op=O.BCO, tol=TOL, maxit=MAXIT)["iters"]     # untimed: the full count
    times = []
    for k in range(args.warmup + max(1, args.steps)):
        t = time.perf_counter()
        r = orc.pcg(p.rhs(), op=O.BCO, tol=TOL, maxit=sample)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt / r["iters"])
    per_it_ms = float(np.mean(times)) * 1e3
    value = per_it_ms * full_iters
    line = {"metric": METRIC, "value": round(value, 2), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(value, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": p.n, "nnz": A.nnz, "precond": "B_co", "tol": TOL,
                       "l2": "cpu"},
            "cpu_baseline": {"value": round(value, 2), "unit": "ms", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "each step: %d B_co PCG iterations of the oracle on the %s matrix, "
                                       "scaled by its full iteration count (%d)" % (sample, WORKLOAD, full_iters)},
            "e2e": {"value": round(value, 2), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, world: int) -> float:
    """The slowest rank's time (all ranks call this; a no-op for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_solve(ms_per_step: float, world: int) -> float:
    """Independent replicas: every step solves `world` systems, so the job's time per solve is
    the (slowest) step time over world."""
    return ms_per_step / world


def profile_mode(name):
    """One preconditioner application plus one fine-level sweep between cudaProfilerStart/Stop
    (for `ncu --profile-from-start off`), after two untimed warm-up applications.  With
    name = "blockcg_fp32": one block PCG solve of the 64 right-hand sides of the batched workload
    (FP32 preconditioner) after one untimed warm-up solve."""
    import torch
    from paper_1205_6113_gb300 import cpc
    pre, prec = name.split("_")
    dev = torch.device("cuda:0")
    p = inputs.workload(WORKLOAD)
    logk = torch.tensor(p.logk, device=dev)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    if pre == "blockcg":
        s = cpc.Solver(rowptr, col, val, precond="bco", precision=prec, ic_order="colour")
        B = torch.tensor(np.ascontiguousarray(inputs.batch_rhs(p.n, 64, seed=5).T), device=dev)
        X = torch.empty_like(B)
        s.solve_block(B, tol=TOL, maxit=MAXIT, X=X)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, it, _, st = s.solve_block(B, tol=TOL, maxit=MAXIT, X=X)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profiled": name, "block_iterations": int(it), "status": int(st)}))
        return
    s = cpc.Solver(rowptr, col, val, precond=pre, precision=prec, ic_order="colour")
    r = torch.tensor(p.rhs(), device=dev)
    z = torch.empty_like(r)
    y = torch.zeros_like(r)
    sweep = prec == "fp64"          # level operators are exposed in FP64 mode
    for _ in range(2):
        s.apply(r, z=z)
        if sweep:
            s.level_apply(0, 5, r, y)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s.apply(r, z=z)
    if sweep:
        s.level_apply(0, 5, r, y)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profiled": name, "launches_per_iteration": s.solve_launches()[0]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-mhfem", action="store_true")
    ap.add_argument("--profile", default=None, help="e.g. bco_fp64: one application for ncu, then exit")
    args = ap.parse_args()
    if args.profile:
        profile_mode(args.profile)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    out = gpu_arm(args, rank, world)
    ms_local = max_over_ranks(float(np.sum(out["headline"]["ms"])), world)
    if rank != 0:
        return
    k = args.steps
    ms_per_step = ms_local / k
    value = whole_job_ms_per_solve(ms_per_step, world)
    p = out["p"]
    iters = out["headline"]["iters"][-1]
    per_it, fixed = out["launches"]
    launches = int(sum(fixed + it * per_it for it in out["headline"]["iters"]))
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world, "steps": k,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": p.n, "nnz": int(out["levels"][0]["nnz"]), "precond": "B_co",
                   "precision": "fp64", "ic_order": "red-black (2-colour)", "tol": TOL, "iters": iters, "levels": out["nlevels"],
                   "l2": "flushed (512 MiB write) before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": round(float(np.mean(out["e2e_ms"])), 3), "unit": "ms",
                "h2d_bytes_per_step": 8 * p.n, "d2h_bytes_per_step": 8 * p.n},
        "roofline": out["roofline"],
        "solve_hbm": {"bytes_per_iter": int(out["bytes_per_iter"]), "gbs": round(out["solve_gbs"], 1),
                      "frac": round(out["solve_gbs"] / out["roofline"]["peak"], 4)},
        "arms": out["arms"],
        "setup_ms": out["setups"],
        "true_res": out["true_res"],
        "adjoint": out.get("adjoint"),
        "batched": out.get("batched"),
        "mhfem": out.get("mhfem"),
        "clocks": out["clocks"],
        "gpu_launches": launches,
        "launches_per_iteration": per_it,
        "hierarchy": {"n": [int(l["n"]) for l in out["levels"]], "nnz": [int(l["nnz"]) for l in out["levels"]],
                      "colours": [int(l["ncolours"]) for l in out["levels"][:-1]],
                      "operator_complexity": round(sum(l["nnz"] for l in out["levels"]) / out["levels"][0]["nnz"], 3),
                      "grid_complexity": round(sum(l["n"] for l in out["levels"]) / out["levels"][0]["n"], 3)},
    }
    if not args.no_cpu_baseline and world == 1:
        _, r, setup_s, solve_s = oracle_time(p)
        line["cpu_baseline"] = {"value": round(solve_s * 1e3, 1), "unit": "ms", "cores": 1,
                                "host_cores": os.cpu_count(), "kind": "oracle",
                                "sample": "one full B_co PCG solve (%d iterations) of the %s matrix on one host "
                                          "core, solve phase only (oracle setup %.1f s excluded)"
                                          % (r["iters"], WORKLOAD, setup_s),
                                "iters": r["iters"]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
