"""Benchmark: PCG solve time to a 1e-6 relative residual on one GB300.

Headline (``value``): milliseconds per combined-preconditioned (B_co) PCG solve, FP64, on the
128 x 128 x 64 correlated-lognormal two-point-flux matrix (1,048,576 unknowns), inputs resident
in HBM.  The same run times, per matrix (the 64 x 64 plane, the 1M-unknown correlated field, the
256 x 256 x 128 channel field and the mixed-hybrid system), B_co against AMG alone (S~, two
V-cycles) and IC(0) alone, FP64 and with the FP32 preconditioner; the end-to-end solve through
host buffers; the error of the FP64 and FP32-preconditioned solutions against the FP64 oracle;
the dominant kernel against the measured HBM roofline; and the CPU oracle as a reported baseline
(one core, and OpenMP over the host's cores).

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
# committed ncu capture (profiles/dram_bco_fp64_correlated3d_128x128x64.md); None until a capture
# of the current kernel exists.
TRAFFIC_K_GS_FINE = 48238848
# The same for one forward sweep of every coarse level (the k_gs launches of the sweep, summed,
# cold cache; profiles/dram_bco_fp64_correlated3d_128x128x64.md); None until a capture of the
# current hierarchy exists.
TRAFFIC_COARSE_SWEEP = 230672896


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
            if l == 0 and lay0["ndiag"] and i["ncolours"] == 2 and not ilu_fine:
                # pre and post sweep; the residual after the sweep reads only the first colour's
                # rows and writes zeros for the second (k_resid_dia_first)
                b += 2 * a_pass(l, svl) + dia_pass_bytes(i["n"] // 2, lay0["ndiag"], svl, sx) + i["n"] // 2 * sx
            else:
                b += 3 * a_pass(l, svl)                                 # pre sweep, residual, post sweep
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

    def time_solves(solver, steps, warmup, tol=TOL, rhs=None):
        rhs = b if rhs is None else rhs
        iters = []
        for _ in range(warmup):
            _, it, st, _ = solver.solve(rhs, tol=tol, maxit=MAXIT, hist=False)
            if st != 0:
                raise SolveFailed(st, it)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        dist_barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush_l2()
            ev[k][0].record(stream)
            _, it, st, _ = solver.solve(rhs, tol=tol, maxit=MAXIT, hist=False)
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
    setups["bco_fp64"]["amg_phases_ms"] = {k: round(v, 2) for k, v in s_bco.setup_phases_ms().items()}
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

    # comparison arms on the benchmark matrix: every preconditioner and precision
    # (name, preconditioner, precision, IC(0) order, Gauss-Seidel order, timed solves)
    arms = {}
    if world == 1:
        arms = compare_matrix(cpc, (rowptr, col, val), b, p.rhs(), time_solves, [
            ("amg_fp64", "amg", "fp64", "natural", "multicolour", args.steps),
            ("ic0_fp64", "ic0", "fp64", "natural", "multicolour", 2),
            ("ic0_rbic_fp64", "ic0", "fp64", "colour", "multicolour", 2),
            ("bco_natic_fp64", "bco", "fp64", "natural", "multicolour", args.steps),
            ("bco_natgs_fp64", "bco", "fp64", "natural", "natural", 2),
            ("bhat_fp64", "bhat", "fp64", "colour", "multicolour", args.steps),
            ("amg_ilu_fp64", "amg_ilu", "fp64", "colour", "multicolour", args.steps),
            ("bco_fp32", "bco", "fp32", "colour", "multicolour", args.steps),
            ("bco_fp32_bf16", "bco", "fp32_bf16", "colour", "multicolour", args.steps),
            ("amg_fp32", "amg", "fp32", "natural", "multicolour", args.steps)], args)

    # the same three-way comparison on the other matrices: the 64 x 64 plane (the plain method),
    # the 256 x 256 x 128 channel field (1000:1 contrast, k_z / k = 0.01) and the mixed-hybrid
    # system of the 128 x 128 x 64 field
    matrices = {}
    if world == 1 and not args.no_matrices:
        matrices = other_matrices(cpc, dev, time_solves, args)

    # batched: 64 right-hand sides and their adjoints in one graph, FP32 preconditioner
    if world == 1 and not args.no_batched:
        out["batched"] = batched_arm(rowptr, col, val, p, dev, stream, args)

    # differentiable solve on the 256 x 256 x 128 channel problem: gradient of the well misfit
    if world == 1 and not args.no_adjoint:
        out["adjoint"] = adjoint_arm(dev, stream)

    # solutions of the FP64 and the FP32-preconditioned solver at tol 1e-10, for the comparison with
    # the FP64 oracle (made after the GPU part)
    xs = {}
    if world == 1 and not args.no_cpu_baseline:
        for prec in ("fp64", "fp32"):
            s = s_bco if prec == "fp64" else cpc.Solver(rowptr, col, val, precond="bco", precision=prec,
                                                          ic_order="colour")
            x, it, st, _ = s.solve(b, tol=1e-10, maxit=MAXIT, hist=False)
            xs[prec] = dict(x=x.cpu().numpy(), iters=it, status=st)
            if s is not s_bco:
                s.close()

    # the dominant kernels, timed live on the solver's stream:
    # (1) the coarse-level Gauss-Seidel colour steps (k_gs; the largest share of the solve's kernel
    #     time): one forward sweep per coarse level replayed from a CUDA graph as in the solve.
    #     Algorithmic bytes per sweep: 12 B per off-diagonal entry (value, column) + 28 B per row
    #     (1 / a_ii, slot -> row, f read, x written, x read once).
    peak, peak_kind = peaks()
    coarse, cbytes, cus = [], 0, 0.0
    for l in range(1, s_bco.nlevels - 1):
        inf = s_bco.level_info(l)
        us = s_bco.sweep_time_us(l, reps=20)
        nbytes = 12 * (inf["nnz"] - inf["n"]) + 28 * inf["n"]
        cbytes += nbytes
        cus += us
        coarse.append(dict(level=l, n=inf["n"], colours=inf["ncolours"], us_per_sweep=round(us, 2),
                           us_per_step=round(us / inf["ncolours"], 2), achieved=round(nbytes / (us * 1e-6) / 1e9, 1)))
    coarse_achieved = cbytes / (cus * 1e-6) / 1e9
    # (2) the fine-level colour step (k_gs_pk): one red + one black launch per sweep, L2 flushed
    #     before each sweep (the fine level's 90 MB would otherwise stay in L2 between sweeps,
    #     which it does not inside a solve)
    info0 = s_bco.level_info(0)
    lay0 = s_bco.level_layout(0)
    xv = torch.randn(p.n, dtype=torch.float64, device=dev)
    yv = torch.zeros_like(xv)
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
    fine_us = float(np.mean(kms)) * 1e3
    if lay0["ndiag"]:       # per row: nd diagonals, 1/a_ii, slot -> row, f_i, x_i written, the other colour's x once
        kbytes = info0["n"] * (8 * lay0["ndiag"] + 36) // info0["ncolours"]
        kname = "k_gs_pk (Gauss-Seidel colour step, fine level, red/black, per-slot diagonal records, FP64)"
    else:                   # per row / entry: SELL values + columns, 1/a_ii, f_i, x_i
        kbytes = (24 * info0["n"] + 12 * info0["nnz"]) // info0["ncolours"]
        kname = "k_gs (Gauss-Seidel colour step, fine level, red/black, SELL, FP64)"
    fine = dict(kernel=kname, bytes_per_launch=kbytes, avg_launch_ms=round(fine_us * 1e-3, 5),
                achieved=round(kbytes / (fine_us * 1e-6) / 1e9, 1),
                frac=round(kbytes / (fine_us * 1e-6) / 1e9 / peak, 4), traffic=TRAFFIC_K_GS_FINE)
    # (3) the fine SpMV of PCG (one launch per event pair, L2 flushed)
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
                achieved=round(sbytes / (np.mean(sms) * 1e-3) / 1e9, 1),
                frac=round(sbytes / (np.mean(sms) * 1e-3) / 1e9 / peak, 4))
    bpi = bytes_per_iteration(s_bco, "bco")
    headline_ms = float(np.mean(ms))
    roofline = dict(bound="hbm", achieved=round(coarse_achieved, 1), peak=peak, unit="GB/s",
                    frac=round(coarse_achieved / peak, 4), traffic=TRAFFIC_COARSE_SWEEP,
                    kernel="k_gs (Gauss-Seidel colour steps of the coarse levels 1..%d, FP64): one forward sweep per "
                           "level, aggregated; dependent-launch latency bounds these steps" % (s_bco.nlevels - 2),
                    bytes_per_sweep=int(cbytes), us_per_sweep=round(cus, 2), peak_kind=peak_kind, levels=coarse,
                    fine_gs=fine, spmv=spmv)
    out.update(dict(p=p, arms=arms, matrices=matrices, clocks=clk, e2e_ms=e2e_ms, true_res=true_res,
                    setups=setups, roofline=roofline, headline_ms=headline_ms, bytes_per_iter=bpi, xs=xs,
                    nlevels=s_bco.nlevels, levels=[s_bco.level_info(l) for l in range(s_bco.nlevels)],
                    coarse_inverse=s_bco.coarse_inverse_info()))
    out["solve_gbs"] = bpi * iters[-1] / (headline_ms * 1e-3) / 1e9
    out["launches"] = s_bco.solve_launches()
    return out


def compare_matrix(cpc, csr, b, b_host, time_solves, configs, args, bytes_fn=True):
    """Times each (name, preconditioner, precision, IC(0) order, Gauss-Seidel order, solves) on one
    matrix; records ms, iterations, setup and the true FP64 residual of the last solve."""
    import torch
    rowptr, col, val = csr
    res = {}
    for name, pre, prec, ico, gso, k in configs:
        t = time.perf_counter()
        s = cpc.Solver(rowptr, col, val, precond=pre, precision=prec, ic_order=ico, gs_order=gso)
        torch.cuda.synchronize()
        setup = dict(zip(("ic0_ms", "amg_ms"), [round(v, 2) for v in s.setup_time_ms()]))
        setup["wall_ms"] = round((time.perf_counter() - t) * 1e3, 1)
        try:
            slow = pre == "ic0" or gso == "natural"
            m, it, _ = time_solves(s, k, 1 if slow else args.warmup, rhs=b)
        except SolveFailed as e:                 # AMG(ILU(0)) need not be SPD (Section 5): record it
            res[name] = dict(ms=None, iters=e.iters, status=e.status, setup=setup)
            s.close()
            continue
        x, _, _, _ = s.solve(b, tol=TOL, maxit=MAXIT, hist=False)
        xr = x.cpu().numpy()
        res[name] = dict(ms=round(float(np.mean(m)), 3), iters=int(it[-1]), setup=setup,
                         true_res=float(np.linalg.norm(b_host - csr_matvec(rowptr, col, val, xr)) / np.linalg.norm(b_host)))
        if bytes_fn:
            bpi = bytes_per_iteration(s, pre, sv=8 if prec == "fp64" else 4, sx=8 if prec == "fp64" else 4,
                                      sv_coarse=(2 if prec == "fp32_bf16" else None))
            res[name]["gbs_solve"] = round(bpi * it[-1] / (np.mean(m) * 1e-3) / 1e9, 1)
        s.close()
    return res


def verdict(r):
    """Which of B_co, AMG alone and IC(0) alone (FP64) reaches 1e-6 first, and B_co's margin."""
    cand = {k: v["ms"] for k, v in r.items() if k in ("bco_fp64", "amg_fp64", "ic0_fp64", "ic0_rbic_fp64")
            and v.get("ms") is not None}
    if "bco_fp64" not in cand:
        return None
    best = min(cand, key=cand.get)
    others = {k: v for k, v in cand.items() if k != "bco_fp64"}
    runner = min(others, key=others.get) if others else None
    return dict(fastest=best, bco_vs_best_other=round(others[runner] / cand["bco_fp64"], 3) if runner else None,
                best_other=runner)


def other_matrices(cpc, dev, time_solves, args):
    import torch
    out = {}
    three_way = lambda k, ic_natural=True: [
        ("bco_fp64", "bco", "fp64", "colour", "multicolour", k),
        ("amg_fp64", "amg", "fp64", "natural", "multicolour", k),
        ("ic0_rbic_fp64", "ic0", "fp64", "colour", "multicolour", 1)] + (
        [("ic0_fp64", "ic0", "fp64", "natural", "multicolour", 1)] if ic_natural else []) + [
        ("bco_natic_fp64", "bco", "fp64", "natural", "multicolour", max(1, min(k, 3))),
        ("bco_fp32", "bco", "fp32", "colour", "multicolour", k),
        ("amg_fp32", "amg", "fp32", "natural", "multicolour", k)]
    # 64 x 64 plane: the plain method
    p1 = inputs.lognormal_2d()
    csr = cpc.tpfa_assemble(p1.nx, p1.ny, p1.nz, torch.tensor(p1.logk, device=dev), p1.kz_ratio, p1.dirichlet)
    r = compare_matrix(cpc, csr, torch.tensor(p1.rhs(), device=dev), p1.rhs(), time_solves, three_way(args.steps),
                       args, bytes_fn=False)
    out["lognormal2d_64x64"] = dict(n=p1.n, results=r, verdict=verdict(r))
    # 256 x 256 x 128 channel field (natural-order IC(0) alone left out: 638 wavefronts per
    # triangular solve and thousands of iterations)
    p4 = inputs.channel_facies()
    csr = cpc.tpfa_assemble(p4.nx, p4.ny, p4.nz, torch.tensor(p4.logk, device=dev), p4.kz_ratio, p4.dirichlet)
    r = compare_matrix(cpc, csr, torch.tensor(p4.rhs(), device=dev), p4.rhs(), time_solves,
                       three_way(max(1, min(args.steps, 3)), ic_natural=False), args, bytes_fn=False)
    out["channels3d_256x256x128"] = dict(n=p4.n, results=r, verdict=verdict(r))
    del csr
    # mixed-hybrid (p, lambda) system of the 128 x 128 x 64 field, assembled on the device
    p2 = inputs.correlated_3d()
    lk = torch.tensor(p2.logk, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cpc.mhfem_assemble(p2.nx, p2.ny, p2.nz, lk, p2.kz_ratio, p2.dirichlet)
    torch.cuda.synchronize()
    e0.record()
    csr = cpc.mhfem_assemble(p2.nx, p2.ny, p2.nz, lk, p2.kz_ratio, p2.dirichlet)
    e1.record()
    torch.cuda.synchronize()
    nu = int(csr[0].shape[0]) - 1
    bh = np.zeros(nu)
    bh[:p2.n] = p2.rhs()
    r = compare_matrix(cpc, csr, torch.tensor(bh, device=dev), bh, time_solves,
                       three_way(max(1, min(args.steps, 3)), ic_natural=False), args, bytes_fn=False)
    out["correlated3d_128x128x64_mhfem"] = dict(n=nu, nnz=int(csr[1].shape[0]), assembly_ms=round(e0.elapsed_time(e1), 3),
                                                 results=r, verdict=verdict(r))
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


def oracle_time(p, openmp=False, tol=TOL):
    """The oracle (FP64) on the same matrix and with the same B_co as the headline (red-black IC(0)
    ordering): setup once, then one PCG solve.  openmp: the -fopenmp build on every host core."""
    import oracle as O
    A = O.tpfa_problem(p)
    t = time.perf_counter()
    orc = O.Oracle(A, ic_colour_order=True, openmp=openmp)
    setup_s = time.perf_counter() - t
    t = time.perf_counter()
    r = orc.pcg(p.rhs(), op=O.BCO, tol=tol, maxit=MAXIT)
    solve_s = time.perf_counter() - t
    return orc, r, setup_s, solve_s, O.threads(openmp)


def reference_arm(args, rank, world):
    """CPU oracle timed on the host cores (the reference arm: the paper has no code of its own):
    the headline's B_co (red-black IC(0) ordering), single-threaded.  Each step is one full PCG
    solve when warm-up plus timed steps fit in about two minutes; otherwise each step runs the
    number of PCG iterations that fits, and the time per iteration is scaled by the full
    iteration count."""
    import oracle as O
    if rank != 0:
        return
    p = inputs.workload(WORKLOAD)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, ic_colour_order=True)
    t = time.perf_counter()
    full_iters = orc.pcg(p.rhs(), op=O.BCO, tol=TOL, maxit=MAXIT)["iters"]     # untimed: the full count
    full_s = time.perf_counter() - t
    nsteps = args.warmup + max(1, args.steps)
    sample = full_iters if nsteps * full_s <= 120.0 else max(1, int(120.0 / (nsteps * full_s / full_iters)))
    times = []
    for k in range(nsteps):
        t = time.perf_counter()
        r = orc.pcg(p.rhs(), op=O.BCO, tol=TOL, maxit=sample)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt / r["iters"])
    per_it_ms = float(np.mean(times)) * 1e3
    value = per_it_ms * full_iters
    what = ("one full B_co PCG solve (%d iterations)" % full_iters if sample == full_iters else
            "%d B_co PCG iterations, scaled by the full iteration count (%d)" % (sample, full_iters))
    line = {"metric": METRIC, "value": round(value, 2), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(value, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": p.n, "nnz": A.nnz, "precond": "B_co",
                       "ic_order": "red-black (2-colour)", "tol": TOL, "l2": "cpu"},
            "cpu_baseline": {"value": round(value, 2), "unit": "ms", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "each step: %s of the oracle on the %s matrix, one host core"
                                       % (what, WORKLOAD)},
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
    """One preconditioner application plus one fine-level sweep and one fine SpMV between
    cudaProfilerStart/Stop
    (for `ncu --profile-from-start off`), after two untimed warm-up applications.  With
    name = "blockcg_fp32": one block PCG solve of the 64 right-hand sides of the batched workload
    (FP32 preconditioner) after one untimed warm-up solve.  With name = "sweeps_fp64": one
    forward Gauss-Seidel sweep of every coarse level, after two untimed ones.  With name =
    "setup_fp64": one setup of the benchmark's solver (the kernels of the AMG setup; the process
    does nothing else on the GPU besides the matrix assembly)."""
    import torch
    from paper_1205_6113_gb300 import cpc
    pre, prec = name.split("_")
    dev = torch.device("cuda:0")
    p = inputs.workload(WORKLOAD)
    logk = torch.tensor(p.logk, device=dev)
    rowptr, col, val = cpc.tpfa_assemble(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet)
    if pre == "setup":
        s = cpc.Solver(rowptr, col, val, precond="bco", precision=prec, ic_order="colour")
        torch.cuda.synchronize()
        print(json.dumps({"profiled": name, "setup_phases_ms": {k: round(v, 2) for k, v in s.setup_phases_ms().items()}}))
        return
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
    s = cpc.Solver(rowptr, col, val, precond=pre if pre != "sweeps" else "bco", precision=prec, ic_order="colour")
    if pre == "sweeps":     # one forward Gauss-Seidel sweep of every coarse level (k_gs launches only)
        xs = [torch.randn(s.level_info(l)["n"], dtype=torch.float64, device=dev) for l in range(s.nlevels - 1)]
        ys = [torch.zeros_like(x) for x in xs]
        for _ in range(2):
            for l in range(1, s.nlevels - 1):
                s.level_apply(l, 5, xs[l], ys[l])
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for l in range(1, s.nlevels - 1):
            s.level_apply(l, 5, xs[l], ys[l])
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profiled": name, "colours": [s.level_info(l)["ncolours"] for l in range(1, s.nlevels - 1)]}))
        return
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
        s.spmv(r, y)                # the fine SpMV of PCG (diagonal form)
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
    ap.add_argument("--no-matrices", action="store_true")
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
    arms = out["arms"]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world, "steps": k,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": p.n, "nnz": int(out["levels"][0]["nnz"]), "precond": "B_co",
                   "precision": "fp64", "ic_order": "red-black (2-colour)", "theta": 0.12, "tol": TOL,
                   "iters": iters, "levels": out["nlevels"],
                   "l2": "flushed (512 MiB write) before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": round(float(np.mean(out["e2e_ms"])), 3), "unit": "ms",
                "h2d_bytes_per_step": 8 * p.n, "d2h_bytes_per_step": 8 * p.n},
        "roofline": out["roofline"],
        "solve_hbm": {"bytes_per_iter": int(out["bytes_per_iter"]), "gbs": round(out["solve_gbs"], 1),
                      "frac": round(out["solve_gbs"] / out["roofline"]["peak"], 4)},
        "arms": arms,
        "setup_ms": out["setups"],
        "true_res": out["true_res"],
        "matrices": out.get("matrices"),
        "adjoint": out.get("adjoint"),
        "batched": out.get("batched"),
        "clocks": out["clocks"],
        "gpu_launches": launches,
        "launches_per_iteration": per_it,
        "hierarchy": {"n": [int(l["n"]) for l in out["levels"]], "nnz": [int(l["nnz"]) for l in out["levels"]],
                      "colours": [int(l["ncolours"]) for l in out["levels"][:-1]],
                      "operator_complexity": round(sum(l["nnz"] for l in out["levels"]) / out["levels"][0]["nnz"], 3),
                      "grid_complexity": round(sum(l["n"] for l in out["levels"]) / out["levels"][0]["n"], 3),
                      "coarse_inverse": {"method": ("fp32 cholesky + newton-schulz" if out["coarse_inverse"][0] == 1
                                                    else "fp64 cholesky"),
                                         "residual": float(out["coarse_inverse"][1])}},
    }
    headline_ms = round(value, 3)
    if arms:
        r = dict(arms)
        r["bco_fp64"] = dict(ms=headline_ms, iters=iters)
        line["verdict"] = verdict(r)
        line["fp32_vs_fp64"] = {"bco_fp32_ms": arms.get("bco_fp32", {}).get("ms"), "bco_fp64_ms": headline_ms,
                                "speedup": round(headline_ms / arms["bco_fp32"]["ms"], 3)
                                if arms.get("bco_fp32", {}).get("ms") else None}
    if not args.no_cpu_baseline and world == 1:
        import oracle as O
        orc, r, setup_s, solve_s, _ = oracle_time(p)
        line["cpu_baseline"] = {"value": round(solve_s * 1e3, 1), "unit": "ms", "cores": 1,
                                "host_cores": os.cpu_count(), "kind": "oracle",
                                "sample": "one full B_co PCG solve (%d iterations, red-black IC(0) ordering as on the "
                                          "GPU) of the %s matrix on one host core, solve phase only (oracle setup "
                                          "%.1f s excluded)" % (r["iters"], WORKLOAD, setup_s),
                                "iters": r["iters"]}
        _, r2, setup2, solve2, nthr = oracle_time(p, openmp=True)
        line["cpu_baseline"]["openmp"] = {"value": round(solve2 * 1e3, 1), "unit": "ms", "cores": nthr,
                                          "iters": r2["iters"], "setup_s": round(setup2, 2),
                                          "parallel": "sparse products, vector updates, dot products and the rows "
                                                      "of each Gauss-Seidel colour; IC(0) solves and the coarsest "
                                                      "solve sequential"}
        # error of the GPU solutions against the FP64 oracle's, all run to tol 1e-10
        ref = orc.pcg(p.rhs(), op=O.BCO, tol=1e-10, maxit=MAXIT)
        xo = ref["x"]
        line["error_vs_oracle"] = {"tol": 1e-10, "oracle_iters": ref["iters"]}
        for prec, v in out["xs"].items():
            line["error_vs_oracle"][prec] = {"rel_err": float(np.linalg.norm(v["x"] - xo) / np.linalg.norm(xo)),
                                             "iters": int(v["iters"]), "status": int(v["status"])}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
