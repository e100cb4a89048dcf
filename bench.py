#!/usr/bin/env python
"""Benchmark: additive-MG MPCG, DOFs/s to a 1e-8 relative residual.

Workload (one "step" = one complete solve to rtol 1e-8): 3D Poisson, Q1
hexahedral FE on the unit cube, 129^3 nodes (2,048,383 interior DOFs), zero
Dirichlet data, N(0,1) right-hand side (seed 2 + rank), 6 nested grids
(coarsest 5^3 nodes, Cholesky), damped Jacobi nu = 2, omega = 2/3, MPCG window
m = 5.  The headline value is the mixed-precision form (FP32 stencil, smoothing,
transfers and block updates; FP64 Gram reductions, pseudo-inverse, coarse
Cholesky and iterative refinement on the true FP64 residual); the plain FP64
form is measured in the same run and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own independent problem (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NODES, DIM, RHS_SEED, M_WINDOW, RTOL, MAXIT = 129, 3, 2, 5, 1e-8, 1000
WORKLOAD = (f"3D Poisson Q1 FE, unit cube, {NODES}^3 nodes ({(NODES - 2) ** 3:,} DOFs), N(0,1) RHS, "
            f"6 grids (5^3 coarsest, Cholesky), damped Jacobi nu=2 w=2/3, MPCG m={M_WINDOW}, rtol {RTOL:g}")
METRIC = "MPCG-AMG DOFs/s to 1e-8 rel. residual"


def _rank():
    from paper_2402_12833_gb300.multi import rank_env
    return rank_env()


# ---------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 50 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- algorithmic bytes / flops
# Stored stencil coefficients per unknown that a kernel streams: the full
# stencil (3^dim taps, 81 for 3D elasticity), or for the FP32 scalar kernels
# of the mixed precision its symmetric half (the diagonal and the couplings
# to the later neighbours: 14 of 27 in 3D, 5 of 9 in 2D).
def stencil_words(dim: int, w: int, vector: bool = False) -> int:
    if vector:
        return 81
    full = 3 ** dim
    return full // 2 + 1 if w == 4 else full


def kernel_work(cls: str, n: int, C: int, cnt: int, w: int, S: int = 27):
    """Algorithmic HBM bytes and flops of one launch on the fine grid (per
    unknown figures x n; cnt = blocks in the window at that launch; S =
    stored stencil coefficients per unknown, stencil_words).  The flops
    count the full stencil's products whatever is stored."""
    if cls == "orth_update":      # read Z, AZ, P_j, AP_j, r; write P, AP; sym Gram + P^T r
        return (2 * cnt * C + 4 * C + 1) * w * n, 2 * (2 * cnt * C * C + C * (C + 1) + C) * n
    if cls == "gram_window":      # read AP_j, Z
        return (cnt + 1) * C * w * n, 2 * cnt * C * C * n
    if cls == "spmm":             # read stencil, Z; write AZ (+ Z^T AZ)
        taps = 81 if S == 81 else (27 if S > 9 else 9)
        return (S + 2 * C) * w * n, 2 * (taps * C + C) * n
    if cls == "update_xr":        # read P, AP, x, r; write x, r
        return (2 * C + 4) * w * n, 2 * (2 * C + 1) * n
    if cls == "orth_gram":        # double-word: read the new P, AP and r; sym Gram + P^T r
        return (2 * C + 1) * w * n, 2 * (C * (C + 1) + C) * n
    return None, None


def level_dofs(nodes, dim, levels):
    """Interior unknowns of every grid, coarsest first."""
    return [((nodes - 1) // 2 ** (levels - 1 - j) - 1) ** dim for j in range(levels)]


def roofline(trace, ns, C, m, w, peaks, fp64_alu_peak_tflops, S=27, vector=False, s_fine=None):
    """Dominant kernel class by total time; achieved = algorithmic bytes
    (or flops) summed over its launches / summed CUDA-event durations.

    The grid of each multilevel launch follows the launch order of one MG
    chain: the smoothings of grids J, J-1, ..., 1 (nu = 2: one fused launch
    each; vector problems: the first sweep, then the second sweep's
    residual and block update -- one launch on the fine grid, two on the
    coarser ones), the
    restrictions from grids J, ..., 1, one composite prolongation."""
    J = len(ns) - 1
    jsub = 0
    tot = {}
    for cls, ms in trace:
        tot[cls] = tot.get(cls, 0.0) + ms
    dom = max(tot, key=tot.get)
    cnt = 0
    jj = jr = J
    jp = 1
    bytes_sum = flops_sum = 0.0
    launches = 0
    dur = 0.0
    for cls, ms in trace:
        b = f = None
        if cls == "init":
            cnt = 0
        if cls in ("init", "check"):
            jj, jr, jp, jsub = J, J, 1, 0
        if cls == "jacobi" and vector:
            fused = ns[jj] // 3 >= (1 << 17) * 0.9   # the fine grids whose last sweep is one launch
            if jsub == 0:     # s1 = D^-1 r: read r, 3 inverse-block planes; write s1
                b, f = 5 * w * ns[jj], 2 * 3 * ns[jj]
            elif fused:       # s = s1 + D^-1 (r - A s1) in one launch: read S planes, s1, r, 3 planes; write s
                b, f = (S + 6) * w * ns[jj], 2 * (S + 3) * ns[jj]
            elif jsub == 1:   # t = r - A s1: read S planes, s1, r; write t
                b, f = (S + 3) * w * ns[jj], 2 * S * ns[jj]
            else:             # s = s1 + D^-1 t: read t, s1, 3 planes; write s
                b, f = 6 * w * ns[jj], 2 * 3 * ns[jj]
            if jsub == 2 or (jsub == 1 and fused):
                jj -= 1
                jsub = 0
            else:
                jsub += 1
        elif cls == "jacobi":
            Sj = s_fine if (s_fine is not None and jj == J) else S   # matrix-free fine grid: kappa, not stencil
            taps = 27 if S > 9 else 9
            b, f = (Sj + 3) * w * ns[jj], (2 * taps + 4) * ns[jj]
            jj -= 1
        elif cls == "restrict":
            b, f = (ns[jr] + ns[jr - 1]) * w, 2 * 27 * ns[jr - 1]
            jr -= 1
        elif cls == "prolong":   # composite: write J fine columns, read every coarse correction once
            b, f = (J * ns[J] + sum(ns[:J])) * w, 2 * 8 * J * ns[J]
        elif cls in ("orth_update", "gram_window", "spmm", "update_xr", "orth_gram"):
            b, f = kernel_work(cls, ns[J], C, cnt, w, s_fine if (s_fine is not None and cls == "spmm") else S)
        if cls == dom:
            if b is not None:
                bytes_sum += b
                flops_sum += f
            dur += ms
            launches += 1
        if cls == "small_alpha":
            cnt = min(cnt + 1, m)
    share = tot[dom] / sum(tot.values())
    if bytes_sum == 0:
        return dom, None, share, tot
    if w == 8 and fp64_alu_peak_tflops:   # FP64 arithmetic on GB300 runs far below the HBM roofline: ALU bound
        ach = flops_sum / (dur * 1e-3) / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": fp64_alu_peak_tflops, "unit": "TFLOP/s",
               "frac": ach / fp64_alu_peak_tflops, "traffic": None,
               "hbm_GBps": bytes_sum / (dur * 1e-3) / 1e9}
    else:
        ach = bytes_sum / (dur * 1e-3) / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": ach / peaks["hbm_gbs"], "traffic": None}
    out.update({"kernel": dom, "launches": launches, "avg_launch_us": dur / launches * 1e3,
                "algorithmic_bytes_per_launch": bytes_sum / launches, "share_of_solve": share})
    return dom, out, share, tot


def profile_value(kind: str, key: str, field: str):
    """A figure recorded from an ncu capture in the summaries under profiles/
    (lines "<kind>: key=<key> <field>=<value> ... source=<file>[,<file>]
    sha256=<hash>[,<hash>]").  None unless every listed kernel source file is
    unchanged since the counters were taken."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                if not line.startswith(kind + ": "):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:])
                if kv.get("key") != key:
                    continue
                # source=a.cu[,b.cu] sha256=h_a[,h_b] (one digest per file) or
                # sha256=h (one digest of the files' contents in order):
                # every listed file unchanged, else look further
                names, digests = kv["source"].split(","), kv["sha256"].split(",")
                paths = [os.path.join(ROOT, "paper_2402_12833_gb300", "csrc", nm) for nm in names]
                if not all(os.path.exists(q) for q in paths):
                    continue
                blobs = []
                for q in paths:
                    with open(q, "rb") as g:
                        blobs.append(g.read())
                if len(digests) == len(names):
                    ok = all(hashlib.sha256(bl).hexdigest() == dg for bl, dg in zip(blobs, digests))
                else:
                    ok = hashlib.sha256(b"".join(blobs)).hexdigest() == digests[0]
                if ok:
                    return float(kv[field])
    return None


def measured_traffic(key: str):
    """DRAM bytes per launch of a kernel class ("traffic:" lines, key
    <leg>:<class>)."""
    return profile_value("traffic", key, "bytes_per_launch")


def bmin_per_iteration(iters: int, n: int, C: int, m: int, w: int, S: int) -> float:
    """Algorithmic bytes of one MPCG iteration on the fine grid (B_min, the
    least HBM traffic an iteration needs): read the stored window (P_j, A P_j),
    write the new block (P, A P), read and write x and r, read the operator
    once -- (2 cnt C + 2 C + 4) w + S w per unknown, with cnt the blocks in
    the window at that iteration (min(k - 1, m) for update k), averaged over
    the solve.  Coarse grids (at most 1/7 of the fine chain in 3D) are left
    out, so the fraction errs low."""
    tot = 0.0
    for k in range(1, iters + 1):
        cnt = min(k - 1, m)
        tot += ((2 * cnt * C + 2 * C + 4) * w + S * w) * n
    return tot / iters


def per_iteration(key: str, ms_per_step: float, iters: int, n: int, C: int, m: int, w: int, S: int, peaks):
    """Per-iteration HBM figures of one solve: the iteration time (the timed
    solve / its x updates, so per-solve work counts against it), the
    algorithmic B_min bandwidth and, where a committed ncu capture of one
    steady-state iteration of this leg exists for the current kernels, the
    measured DRAM bandwidth (dram__bytes_read + write of that iteration's
    launches / the iteration time)."""
    t = ms_per_step / iters * 1e-3
    bmin = bmin_per_iteration(iters, n, C, m, w, S)
    dram = profile_value("iteration", key, "dram_bytes")
    out = {"ms": t * 1e3, "iterations": iters, "bmin_bytes": bmin, "bmin_GBps": bmin / t / 1e9,
           "bmin_frac": bmin / t / 1e9 / peaks["hbm_gbs"], "dram_bytes": dram,
           "dram_GBps": dram / t / 1e9 if dram else None,
           "dram_frac": dram / t / 1e9 / peaks["hbm_gbs"] if dram else None,
           "peak_GBps": peaks["hbm_gbs"], "peak_source": peaks["source"]}
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# FP64 FMA issue rate of GB300: 2 per SM per clock (152 SMs, 2.07 GHz max) ->
# 152 * 2 * 2 flop * 2.07e9 = 1.26 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# ---------------------------------------------------------------------------- oracle (CPU) legs
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from paper_2402_12833_gb300 import problems as pb
from oracle import mg as omg, mpcg as ompcg
prob = pb.poisson_random({dim}, {nodes}, {seed})
t0 = time.perf_counter()
H = omg.Hierarchy(prob.dim, prob.n1, prob.stencil, prob.levels)
t1 = time.perf_counter()
times = []
for rep in range({warmup} + {steps}):
    ta = time.perf_counter()
    res = ompcg.mpcg(H.A[-1], prob.b, H.mg_columns, m={m}, rtol={rtol}, maxit={maxit})
    if rep >= {warmup}:
        times.append(time.perf_counter() - ta)
print(json.dumps({{"setup_s": t1 - t0, "solve_s": sum(times) / len(times), "iters": res.iters, "n": prob.n,
                  "res": res.res_hist[-1], "steps": len(times)}}))
"""


def usable_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_mem_available_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


ORACLE_GB_PER_PROCESS = 5.0   # one 129^3 oracle solve peaks at 4.1 GB resident; with margin


def oracle_baselines(n: int):
    """The FP64 oracle as it stands on the host cores, started after every GPU
    measurement so that it does not compete for them: one process on one
    core (one full solve), then one process per usable core, each solving the
    same workload at once (host throughput = processes x n / slowest solve;
    capped by the memory available).  Returns (all-cores, single-core)."""
    cmd, env = oracle_cmd(0, 1)
    single = None
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode == 0:
        o = json.loads(out.stdout.strip().splitlines()[-1])
        single = {"value": o["n"] / o["solve_s"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                  "sample": f"one full FP64 solve of the workload ({o['iters']} iterations, {o['solve_s']:.1f} s; "
                            f"hierarchy setup {o['setup_s']:.1f} s excluded)", "iters": o["iters"]}
    else:
        return ({"value": None, "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                 "sample": "failed: " + out.stderr[-300:]}, None)
    cores = usable_cores()
    nproc = max(1, min(cores, int(host_mem_available_gb() // ORACLE_GB_PER_PROCESS)))
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(nproc)]
    times, iters = [], None
    for p in procs:
        o_out, o_err = p.communicate(timeout=3600)
        if p.returncode != 0:
            return single, single
        o = json.loads(o_out.strip().splitlines()[-1])
        times.append(o["solve_s"])
        iters = o["iters"]
    allc = {"value": nproc * n / max(times), "unit": "DOFs/s", "cores": nproc, "kind": "oracle",
            "sample": f"{nproc} single-threaded oracle processes ({cores} usable cores), each one full FP64 solve "
                      f"of the workload at the same time ({iters} iterations; slowest {max(times):.1f} s, "
                      f"fastest {min(times):.1f} s; setup excluded)", "iters": iters,
            "single_core": single}
    return allc, single


def oracle_cmd(warmup: int, steps: int, seed: int = RHS_SEED):
    """The FP64 oracle as it stands, single-threaded, in a fresh process:
    hierarchy setup once, then warmup + steps full solves."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, dim=DIM, nodes=NODES, seed=seed, m=M_WINDOW, rtol=RTOL,
                                 maxit=MAXIT, warmup=warmup, steps=steps)
    return [sys.executable, "-c", code], env


def bench_reference(args):
    rank, world, _ = _rank()
    if rank != 0:
        return 0
    # each step is one full oracle solve of the workload (~10-20 s on one core);
    # a single untimed warm-up solve stands in for the W warm-up steps
    cmd, env = oracle_cmd(1, args.steps)
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + out.stderr[-200:]}))
        return 0
    o = json.loads(out.stdout.strip().splitlines()[-1])
    steps = [o]
    t = o["solve_s"]
    n = o["n"]
    v = n / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOFs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                             "sample": f"full solve of the workload per step ({steps[0]['iters']} iterations; "
                                       f"hierarchy setup {steps[0]['setup_s']:.1f} s excluded)"},
            "e2e": {"value": v, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- GPU leg
def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    M.load()

    from paper_2402_12833_gb300.multi import problem_seed
    prob = pb.poisson_random(DIM, NODES, problem_seed(RHS_SEED, rank))
    n = prob.n
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    st = torch.from_numpy(prob.stencil).cuda()
    ug = 0 if args.direct else 1
    legs = ("fp64", "fp64_dw", "mixed") if args.only is None else (args.only,)
    precs = {"mixed": M.MPCG_MIXED, "fp64": M.MPCG_FP64, "fp64_dw": M.MPCG_FP64_DW}
    H = {k: M.Hierarchy(st, DIM, NODES, prob.levels, m=M_WINDOW, precision=precs[k], stream=sptr, use_graph=ug)
         for k in legs}
    if args.matrix_free:   # the matrix-free fine operator (element coefficients kappa = 1) in the mixed solve
        M.mg_attach_q1_kappa(H["mixed"].h, torch.ones((NODES - 1) ** DIM, dtype=torch.float64, device="cuda"))
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    peaks = load_peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        from paper_2402_12833_gb300.multi import max_over_ranks as mor
        return mor(v, device="cuda")

    # launch shapes: the fixed rules first (timed below for comparison), then
    # the autotuner's choice for every leg, which the timed region uses
    fixed_ms = {}
    if not args.no_autotune:
        for key in legs:
            hk = H[key]
            for _ in range(args.warmup):
                x.zero_()
                hk.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)
            fixed_ms[key] = _timed(lambda: (x.zero_(), hk.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)),
                                   args.steps, 0, stream)
        tuned = {key: M.mg_autotune(H[key].h) for key in legs}
    res = {}
    clocks = None
    for key in legs:
        h = H[key]
        for _ in range(args.warmup):
            x.zero_()
            h.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)
        barrier()
        torch.cuda.synchronize()
        if key == "mixed" and rank == 0:
            clk = Clocks(local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = []
        torch.cuda.nvtx.range_push("timed_step")
        e0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            st_, k, _, _ = h.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)
            iters.append(k)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
        if key == "mixed" and rank == 0:
            clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        launches = M.mg_last_launches(h.h)
        # true FP64 residual of the last solution (one extra SpMV through the library)
        Ax = torch.empty_like(b)
        M.mg_apply_operator(h.h, prob.levels - 1, x, Ax, 1)
        true_res = float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b))
        res[key] = {"ms_per_step": ms, "value": world * n / (ms * 1e-3), "iters": iters[-1],
                    "launches_per_step": launches, "true_rel_residual": true_res,
                    "x": x.detach().clone() if key in ("fp64", "fp64_dw") else None}

    # the same mixed solve with the FP32 kernels on the full 27-plane stencil
    # (half_stencil = 0) instead of its symmetric half, same launch-shape table
    # and timing: the in-run comparison for the half-stencil layout
    full = None
    if args.only is None:
        Hf = M.Hierarchy(st, DIM, NODES, prob.levels, m=M_WINDOW, precision=M.MPCG_MIXED, stream=sptr,
                         use_graph=ug, half_stencil=0)
        kf = {}

        def full_step():
            x.zero_()
            _, kf["k"], _, _ = Hf.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

        full_ms = max_over_ranks(_timed(full_step, args.steps, args.warmup, stream))
        full = {"value": world * n / (full_ms * 1e-3), "ms_per_step": full_ms, "iterations": int(kf["k"]),
                "stencil_words_per_unknown": 27, "note": "FP32 SpMM and Jacobi on the full stencil (half_stencil=0)"}
        Hf.close()

    if args.only is not None:
        r = res[args.only]
        if rank == 0:
            print(json.dumps({"metric": METRIC, "only": args.only, "value": r["value"], "unit": "DOFs/s",
                              "ms_per_step": r["ms_per_step"], "iterations": r["iters"],
                              "true_rel_residual": r["true_rel_residual"], "launches_per_step": r["launches_per_step"],
                              "clocks": clocks}))
        for h in H.values():
            h.close()
        return 0

    # the single-block window (m = 1), reported beside the paper's m = 5
    Hm1 = M.Hierarchy(st, DIM, NODES, prob.levels, m=1, precision=M.MPCG_MIXED, stream=sptr, use_graph=ug)
    m1 = {}

    def m1_step():
        x.zero_()
        m1["st"], m1["k"], _, _ = Hm1.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

    m1_ms = max_over_ranks(_timed(m1_step, args.steps, args.warmup, stream))
    Hm1.close()

    # the same solve with the matrix-free fine operator (element coefficients
    # kappa = 1 of this Poisson problem; the FP32 fine kernels rebuild the rows)
    Hmf = M.Hierarchy(st, DIM, NODES, prob.levels, m=M_WINDOW, precision=M.MPCG_MIXED, stream=sptr, use_graph=ug)
    M.mg_attach_q1_kappa(Hmf.h, torch.ones((NODES - 1) ** DIM, dtype=torch.float64, device="cuda"))
    mf = {}

    def mf_step():
        x.zero_()
        mf["st"], mf["k"], _, _ = Hmf.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

    mf_ms = max_over_ranks(_timed(mf_step, args.steps, args.warmup, stream))
    Axm = torch.empty_like(b)
    M.mg_apply_operator(Hmf.h, prob.levels - 1, x, Axm, 1)
    mf["true_res"] = float(torch.linalg.norm(b - Axm) / torch.linalg.norm(b))
    x.zero_()
    _, _, _, trace_mf = M.mpcg_solve_profiled(Hmf.h, b, x, RTOL, MAXIT)
    _, mf["roofline"], _, tot_mf = roofline(trace_mf, level_dofs(NODES, DIM, prob.levels), prob.levels, M_WINDOW, 4,
                                            peaks, FP64_PEAK_TFLOPS, S=stencil_words(DIM, 4), s_fine=1)
    if mf["roofline"] is not None:
        mf["roofline"]["traffic"] = measured_traffic(f"poisson3d_mixed_mf:{mf['roofline']['kernel']}")
    mf["class_ms"] = {c: round(v, 4) for c, v in tot_mf.items()}
    Hmf.close()

    # per-kernel durations from a live profiled solve (CUDA events on the solve stream)
    prof = {}
    for key, w in (("mixed", 4), ("fp64", 8), ("fp64_dw", 8)):
        x.zero_()
        _, k, classes, trace = M.mpcg_solve_profiled(H[key].h, b, x, RTOL, MAXIT)
        # FP64 arithmetic is bound by the FP64 pipe; the double-word kernels
        # are reported against the HBM roofline they aim at
        dom, rl, share, tot = roofline(trace, level_dofs(NODES, DIM, prob.levels), prob.levels, M_WINDOW, w, peaks,
                                       FP64_PEAK_TFLOPS if key == "fp64" else None,
                                       S=stencil_words(DIM, 4 if key == "mixed" else 8))
        if rl is not None:
            rl["traffic"] = measured_traffic(f"poisson3d_{key}:{dom}")
        prof[key] = {"roofline": rl, "class_ms": {c: round(v, 4) for c, v in tot.items()}}
    # mixed vs fp64 solution difference
    x.zero_()
    H["mixed"].solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)
    mix_vs_fp64 = float(torch.linalg.norm(x - res["fp64"]["x"]) / torch.linalg.norm(res["fp64"]["x"]))
    dw_vs_fp64 = float(torch.linalg.norm(res["fp64_dw"]["x"] - res["fp64"]["x"]) / torch.linalg.norm(res["fp64"]["x"]))
    piter = {}
    for key, w in (("mixed", 4), ("fp64", 8), ("fp64_dw", 8)):
        piter[key] = per_iteration(f"poisson3d_{key}", res[key]["ms_per_step"], res[key]["iters"], n, prob.levels,
                                   M_WINDOW, w, stencil_words(DIM, w), peaks)

    # end to end through the C ABI with pinned host buffers
    bh = torch.from_numpy(prob.b).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    for _ in range(max(1, args.warmup // 2)):
        xh[:] = 0.0
        M.mpcg_solve(H["mixed"].h, bh, xh, RTOL, MAXIT, histories=False)
    barrier()
    # each step times the API call alone (H2D of b and x0, the solve, D2H of
    # x); resetting x0 to zero in the pinned host buffer is input preparation
    # and stays outside
    e2e_total = 0.0
    for _ in range(args.steps):
        xh[:] = 0.0
        t0 = time.perf_counter()
        M.mpcg_solve(H["mixed"].h, bh, xh, RTOL, MAXIT, histories=False)
        e2e_total += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_total / args.steps)
    barrier()

    for h in H.values():
        h.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _ = oracle_baselines(n)

    if rank == 0:
        mx = res["mixed"]
        line = {
            "metric": METRIC, "value": mx["value"], "unit": "DOFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed: FP32 bulk, FP64 Gram/pinv/Cholesky/refinement",
                       "dofs_per_rank": n, "parallelism": f"{world} independent problems (one per GPU)",
                       "l2": "working set ~1 GB per solve > 129 MB L2 (no flush needed)"},
            "iterations": mx["iters"], "true_rel_residual": mx["true_rel_residual"],
            "rel_diff_vs_fp64_solution": mix_vs_fp64,
            "m1": {"value": world * n / (m1_ms * 1e-3), "ms_per_step": m1_ms, "iterations": int(m1["k"])},
            "matrix_free": {"value": world * n / (mf_ms * 1e-3), "ms_per_step": mf_ms, "iterations": int(mf["k"]),
                            "true_rel_residual": mf["true_res"], "roofline": mf["roofline"],
                            "kernel_ms_per_solve": mf["class_ms"],
                            "operator": "fine grid rebuilt from the element coefficients (kappa = 1) in the FP32 "
                                        "SpMM and Jacobi kernels; stored stencils elsewhere"},
            "roofline": prof["mixed"]["roofline"],
            "per_iteration": piter["mixed"],
            "full_stencil": full,
            "autotune": None if args.no_autotune else {
                "candidates_timed": tuned, "fixed_rules_ms_per_step": fixed_ms,
                "note": "every leg timed with the autotuner's launch shapes; the fixed rules' times beside"},
            "fp64": {"value": res["fp64"]["value"], "unit": "DOFs/s", "ms_per_step": res["fp64"]["ms_per_step"],
                     "iterations": res["fp64"]["iters"], "true_rel_residual": res["fp64"]["true_rel_residual"],
                     "roofline": prof["fp64"]["roofline"], "per_iteration": piter["fp64"]},
            "fp64_dw": {"value": res["fp64_dw"]["value"], "unit": "DOFs/s",
                        "ms_per_step": res["fp64_dw"]["ms_per_step"], "iterations": res["fp64_dw"]["iters"],
                        "true_rel_residual": res["fp64_dw"]["true_rel_residual"],
                        "rel_diff_vs_fp64_solution": dw_vs_fp64, "roofline": prof["fp64_dw"]["roofline"],
                        "per_iteration": piter["fp64_dw"],
                        "arithmetic": "FP64 data; vectors and stencils as float pairs hi + lo (~48-bit "
                                      "significand) on the FP32 pipe; FP64 reductions, pseudo-inverse, coarse solve"},
            "kernel_ms_per_solve": {"mixed": prof["mixed"]["class_ms"], "fp64": prof["fp64"]["class_ms"],
                                    "fp64_dw": prof["fp64_dw"]["class_ms"]},
            "e2e": {"value": world * n / e2e_s, "unit": "DOFs/s", "h2d_bytes_per_step": 2 * 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": mx["launches_per_step"] * args.steps,
            "clocks": clocks,
            "peaks": peaks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------- extra workloads
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3) / steps


def bench_batched(args):
    """256 independent 2D high-contrast problems (sides drawn from 33..513, own
    kappa and N(0,1) RHS), mixed precision, rtol 1e-8 each: one batched
    hierarchy per side length, the classes solved concurrently."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import multi
    from paper_2402_12833_gb300 import problems as pb
    rank, world, local = multi.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    M.load()
    sizes = pb.batch_sizes(256, seed=4)
    # the 256 independent problems are dealt to the ranks by DOF count (no
    # communication on the data path)
    mine = multi.shard_batch([(s - 2) ** 2 for s in sizes], rank, world)
    by = {}
    for i in mine:
        by.setdefault(sizes[i], []).append(i)
    classes, bs, xs, ns = [], [], [], 0
    streams, kappas = [], []
    for nodes in sorted(by):
        ps = [pb.batch_problem(i, nodes) for i in by[nodes]]
        kappas.append(torch.from_numpy(np.concatenate([p.kappa.reshape(-1) for p in ps])).cuda())
        strm = torch.cuda.Stream()
        streams.append(strm)
        classes.append(M.BatchedHierarchy([torch.from_numpy(p.stencil).cuda() for p in ps], 2, nodes, ps[0].levels,
                                          m=M_WINDOW, precision=M.MPCG_MIXED, stream=strm.cuda_stream))
        bs.append(torch.from_numpy(np.stack([p.b for p in ps])).cuda())
        xs.append(torch.zeros_like(bs[-1]))
        ns += len(ps) * ps[0].n
    torch.cuda.synchronize()
    its = None

    def step():
        nonlocal its
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        _, its = M.mpcg_solve_batched(classes, bs, xs, rtol=RTOL, maxit=20000)

    if world > 1:
        dist.barrier()
    ms = multi.max_over_ranks(_timed(step, args.steps, max(1, args.warmup // 3), torch.cuda.current_stream()),
                              device="cuda")
    launches = sum(M.mg_last_launches(c.h) for c in classes)
    its_stored = its
    # the same batch with the matrix-free fine operators (each problem's kappa)
    for c, k in zip(classes, kappas):
        M.mg_attach_q1_kappa(c.h, k)
    ms_mf = multi.max_over_ranks(_timed(step, args.steps, max(1, args.warmup // 3), torch.cuda.current_stream()),
                                 device="cuda")
    its_mf, its = its, its_stored
    ns_all = multi.sum_over_ranks(ns, device="cuda")
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    # roofline of the dominant kernel class of the largest size class, over
    # its first five inner iterations: every problem of the class is still
    # running there, so a launch moves the class's problem count times the
    # per-problem algorithmic bytes (later launches skip converged problems)
    big = max(by)
    ci = sorted(by).index(big)
    cbig = classes[ci]
    p0 = pb.batch_problem(by[big][0], big)
    ns1 = [M.mg_level_size(cbig.h, j) for j in range(p0.levels)]
    M.mg_detach_q1_kappa(cbig.h)   # the stored stencils, as in the headline figure
    xs[ci].zero_()
    _, _, _, trace = M.mpcg_solve_profiled(cbig.h, bs[ci], xs[ci], RTOL, 20000)
    checks = [i for i, (c, _) in enumerate(trace) if c == "check"]
    head = trace[:checks[4] + 1] if len(checks) >= 5 else trace
    nprob = len(by[big])
    _, rl, _, tot1 = roofline(head, ns1, p0.levels, M_WINDOW, 4, load_peaks(), FP64_PEAK_TFLOPS,
                              S=stencil_words(2, 4))
    if rl is not None:
        for k in ("achieved", "frac", "algorithmic_bytes_per_launch"):
            rl[k] *= nprob
        rl["workload"] = (f"the {nprob} problems of {big}^2 nodes (the largest class), first five inner "
                          f"iterations of the profiled class solve (every problem running)")
    cpu = None
    if not args.no_cpu_baseline:   # after the GPU legs, one core: the oracle on one problem of each side <= 257
        sample = [(by[sd][0], sd) for sd in sorted(by) if sd <= 257]
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = BATCH_ORACLE.format(root=ROOT, sample=sample, m=M_WINDOW, rtol=RTOL)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode == 0:
            o = json.loads(r.stdout.strip().splitlines()[-1])
            cpu = {"value": o["n"] / o["solve_s"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                   "sample": f"FP64 oracle solves of problems {[i for i, _ in sample]} (sides "
                             f"{[sd for _, sd in sample]}, {o['iters']} iterations, {o['solve_s']:.1f} s, setup "
                             f"excluded); DOFs of the sample / its solve time"}
        else:
            cpu = {"value": None, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    print(json.dumps({
        "metric": METRIC, "workload": "batched", "value": ns_all / (ms * 1e-3), "unit": "DOFs/s", "n_gpus": world,
        "scaling": "strong", "steps": args.steps, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "256 x 2D diffusion, sides U{33,65,129,257,513}, log10 kappa U[-2,4] on 16x16 macro "
                               "cells, N(0,1) RHS, levels to 5x5, MPCG m=5, mixed precision, rtol 1e-8 each",
                   "problems_per_side_rank0": {str(k): len(v) for k, v in sorted(by.items())},
                   "total_dofs": int(ns_all)},
        "max_iterations_per_side": {str(k): int(i.max()) for k, i in zip(sorted(by), its)},
        "gpu_launches_per_step": launches, "one_graph_launch": True, "roofline": rl,
        "kernel_ms_first_five_iterations_of_largest_class": {c: round(v, 4) for c, v in tot1.items()},
        "cpu_baseline": cpu,
        "matrix_free": {"value": ns_all / (ms_mf * 1e-3), "ms_per_step": ms_mf,
                        "max_iterations_per_side": {str(k): int(i.max()) for k, i in zip(sorted(by), its_mf)}}}))
    return 0


BATCH_ORACLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from paper_2402_12833_gb300 import problems as pb
from oracle import mg as omg, mpcg as ompcg
n, t, its = 0, 0.0, []
for idx, nodes in {sample!r}:
    p = pb.batch_problem(idx, nodes)
    H = omg.Hierarchy(2, p.n1, p.stencil, p.levels)
    t0 = time.perf_counter()
    res = ompcg.mpcg(H.A[-1], p.b, H.mg_columns, m={m}, rtol={rtol}, maxit=20000)
    t += time.perf_counter() - t0
    n += p.n
    its.append(res.iters)
print(json.dumps({{"n": n, "solve_s": t, "iters": its}}))
"""


ELAST_ORACLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from paper_2402_12833_gb300 import problems as pb
from oracle import mg as omg, mpcg as ompcg
prob = pb.elasticity_cantilever({nodes})
t0 = time.perf_counter()
H = omg.Hierarchy(3, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces, ncomp=3)
t1 = time.perf_counter()
res = ompcg.mpcg(H.A[-1], prob.b, H.mg_columns, m={m}, rtol={rtol}, maxit={maxit})
t2 = time.perf_counter()
print(json.dumps({{"setup_s": t1 - t0, "solve_s": t2 - t1, "iters": res.iters, "n": prob.n}}))
"""


def bench_elasticity(args):
    """3D linear elasticity (Q1 hexahedra, E = 1, nu = 0.3) on the unit cube
    with 65^3 nodes, clamped at x = 0, body force (0, 0, -1): 811,200
    unknowns, 5 grids (coarsest 300 unknowns), 3 x 3 block Jacobi nu = 2,
    MPCG m = 5, rtol 1e-8; mixed precision (headline of this line) and FP64."""
    import torch
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    nodes = 65
    oracle_proc = None
    if not args.no_cpu_baseline:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ELAST_ORACLE.format(root=ROOT, nodes=nodes, m=M_WINDOW, rtol=RTOL, maxit=MAXIT)
        oracle_proc = subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                       text=True, env=env)
    _build.build()
    M.load()
    prob = pb.elasticity_cantilever(nodes)
    n = prob.n
    stream = torch.cuda.current_stream()
    st = torch.from_numpy(prob.stencil).cuda()
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    peaks = load_peaks()
    out = {}
    clocks = None
    legs = (("fp64", M.MPCG_FP64, 8), ("mixed", M.MPCG_MIXED, 4))
    m1 = {}
    if not args.only:
        Hm1 = M.Hierarchy(st, 3, nodes, prob.levels, dofs_per_node=3, faces=prob.faces, m=1,
                          precision=M.MPCG_MIXED, stream=stream.cuda_stream)

        def m1_step():
            x.zero_()
            m1["st"], m1["k"], _, _ = Hm1.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

        m1_ms = _timed(m1_step, args.steps, args.warmup, stream)
        m1 = {"value": n / (m1_ms * 1e-3), "ms_per_step": m1_ms, "iterations": int(m1["k"])}
        Hm1.close()
    if args.only:
        legs = tuple(l for l in legs if l[0] == args.only)
    for key, prec, w in legs:
        H = M.Hierarchy(st, 3, nodes, prob.levels, dofs_per_node=3, faces=prob.faces, m=M_WINDOW, precision=prec,
                        stream=stream.cuda_stream, use_graph=0 if args.direct else 1)
        ns = [M.mg_level_size(H.h, j) for j in range(prob.levels)]
        res = {}

        def step():
            x.zero_()
            res["st"], res["k"], _, _ = H.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if key == "mixed":
            clk = Clocks(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if key == "mixed":
            clocks = clk.stop()
        ms = e0.elapsed_time(e1) / args.steps
        launches = M.mg_last_launches(H.h)
        Ax = torch.empty_like(b)
        M.mg_apply_operator(H.h, prob.levels - 1, x, Ax, 1)
        true_res = float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b))
        if args.only:
            print(json.dumps({"workload": "elasticity", "only": key, "value": n / (ms * 1e-3), "ms_per_step": ms,
                              "iterations": int(res["k"]), "true_rel_residual": true_res}))
            H.close()
            continue
        x.zero_()
        _, _, classes, trace = M.mpcg_solve_profiled(H.h, b, x, RTOL, MAXIT)
        dom, rl, share, tot = roofline(trace, ns, prob.levels, M_WINDOW, w, peaks, FP64_PEAK_TFLOPS, S=81,
                                       vector=True)
        if rl is not None:
            rl["traffic"] = measured_traffic(f"elasticity_{key}:{dom}")
        out[key] = {"value": n / (ms * 1e-3), "ms_per_step": ms, "iterations": int(res["k"]),
                    "status": int(res["st"]), "true_rel_residual": true_res, "launches_per_step": launches,
                    "roofline": rl, "kernel_ms_per_solve": {c: round(v, 4) for c, v in tot.items()}}
        H.close()
    if args.only:
        if oracle_proc is not None:
            oracle_proc.kill()
        return 0
    learned = elasticity_learned(M, pb, prob, st, b, stream, args)
    cpu = None
    if oracle_proc is not None:
        o_out, o_err = oracle_proc.communicate(timeout=1800)
        if oracle_proc.returncode == 0:
            o = json.loads(o_out.strip().splitlines()[-1])
            cpu = {"value": o["n"] / o["solve_s"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                   "sample": f"one full FP64 solve of the same workload ({o['iters']} iterations, "
                             f"{o['solve_s']:.1f} s; hierarchy setup {o['setup_s']:.1f} s excluded)"}
        else:
            cpu = {"value": None, "kind": "oracle", "sample": "failed: " + o_err[-300:]}
    mx = out["mixed"]
    print(json.dumps({
        "metric": METRIC, "workload": "elasticity", "value": mx["value"], "unit": "DOFs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "3D linear elasticity, Q1 hexahedra, E=1, nu=0.3, unit cube 65^3 nodes clamped at "
                               "x=0, body force (0,0,-1): 811,200 unknowns, 5 grids (300-unknown coarsest, "
                               "Cholesky), 3x3 block Jacobi nu=2 w=2/3, MPCG m=5, rtol 1e-8",
                   "l2": "working set ~0.7 GB per solve > 129 MB L2 (no flush needed)"},
        "iterations": mx["iterations"], "true_rel_residual": mx["true_rel_residual"], "roofline": mx["roofline"],
        "fp64": out["fp64"], "m1": m1, "learned": learned, "kernel_ms_per_solve": mx["kernel_ms_per_solve"],
        "gpu_launches": mx["launches_per_step"] * args.steps, "clocks": clocks, "peaks": peaks,
        "cpu_baseline": cpu}))
    return 0


def elasticity_learned(M, pb, prob, st, b, stream, args):
    """The learned column on the elasticity workload: the 3x3x3 network is
    trained on the GPU on (residual, error) pairs that the FP64 solver makes
    for the same body under two other loads, (1, 0, 0) and (0, 1, 1) (the
    first 24 iterates of each), then the mixed-precision solve of the
    workload's load (0, 0, -1) runs with the trained column."""
    import torch
    t0 = time.perf_counter()
    R, E = [], []
    H = M.Hierarchy(st, 3, prob.nodes, prob.levels, dofs_per_node=3, faces=prob.faces, m=M_WINDOW)
    Ax = torch.empty_like(b)
    for force in ((1.0, 0.0, 0.0), (0.0, 1.0, 1.0)):
        bf = torch.from_numpy(pb.elasticity_body_force(prob.nodes, force)).cuda()
        xs = torch.zeros_like(bf)
        H.solve(bf, xs, rtol=1e-13, maxit=MAXIT, histories=False)
        for k in range(1, 25):
            xk = torch.zeros_like(bf)
            H.solve(bf, xk, rtol=1e-30, maxit=k, histories=False)
            M.mg_apply_operator(H.h, prob.levels - 1, xk, Ax, 1)
            r = bf - Ax
            nr = torch.linalg.norm(r)
            R.append((r / nr).float())
            E.append(((xs - xk) / nr).float())
    gen_s = time.perf_counter() - t0
    params = pb.net_init_params(7, (3, 16, 16, 16, 3), taps=27)
    epochs = 20
    t0 = time.perf_counter()
    loss = M.mg_learned_train([H.h], [0] * len(R), torch.stack(R).contiguous(), torch.stack(E).contiguous(), params,
                              epochs=epochs, batch=8, lr=1e-3)
    train_s = time.perf_counter() - t0
    H.close()
    H = M.Hierarchy(st, 3, prob.nodes, prob.levels, dofs_per_node=3, faces=prob.faces, m=M_WINDOW,
                    precision=M.MPCG_MIXED, stream=stream.cuda_stream)
    M.mg_learned_attach(H.h, params)
    x = torch.zeros_like(b)
    res = {}

    def step():
        x.zero_()
        res["st"], res["k"], _, _ = H.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

    ms = _timed(step, args.steps, args.warmup, stream)
    M.mg_apply_operator(H.h, prob.levels - 1, x, Ax, 1)
    out = {"value": prob.n / (ms * 1e-3), "ms_per_step": ms, "iterations": int(res["k"]), "status": int(res["st"]),
           "true_rel_residual": float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b)),
           "training": {"pairs": len(R), "epochs": epochs, "loss_first": float(loss[0]),
                        "loss_last": float(loss[-1]), "pair_generation_s": gen_s, "train_s": train_s}}
    x.zero_()
    _, _, _, trace = M.mpcg_solve_profiled(H.h, b, x, RTOL, MAXIT)
    net = [t for c, t in trace if c == "net"]
    if net:   # the four layer launches of one application, CUDA-event time
        out["net_us_per_application"] = 1e3 * sum(net) / len(net)
    H.close()
    return out


def bench_example1(args):
    """Section 3, Example 1 on the GPU: anisotropic diffusion, 160 x 160
    elements, 4 grids (20 x 20 coarsest), k_xx = 10^-n (n = 0..7), k_yy = 1,
    f = 1, zero Dirichlet data, FP64, rtol 1e-8: iterations and time of
    additive MG-MPCG (one column per grid, m = 5 and m = 1) and additive MG-PCG
    (the summed correction B r as a single direction, m = 1) with the damped
    Jacobi smoother, and the paper's comparison with SSOR: additive MG-MPCG
    (m = 5) and MG-PCG with 6 SSOR steps per grid, and PCG preconditioned by
    the multiplicative V(3,3) cycle; the oracle's iteration counts beside them."""
    import torch
    from oracle import mg as omg
    from oracle import mpcg as ompcg
    from oracle import pcg as opcg
    from oracle import ssor as oss
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    _build.build()
    M.load()
    rows = []
    for n in range(8):
        kxx = 10.0 ** (-n)
        prob = pb.example1(kxx)
        st = torch.from_numpy(prob.stencil).cuda()
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        row = {"kxx": kxx}
        ssor = dict(smoother=M.MPCG_SMOOTHER_SSOR)
        series = (("mpcg_m5", dict(m=5)), ("mpcg_m1", dict(m=1)), ("pcg", dict(m=1, sum_columns=1)),
                  ("ssor_mpcg_m5", dict(ssor, nu=6, m=5)), ("ssor_pcg", dict(ssor, nu=6, m=1, sum_columns=1)),
                  ("v33_pcg", dict(ssor, nu=3, m=1, vcycle=1)))
        for key, opts in series:
            H = M.Hierarchy(st, 2, prob.nodes, prob.levels, **opts)
            res = {}

            def step():
                x.zero_()
                res["st"], res["k"], _, _ = H.solve(b, x, rtol=RTOL, maxit=20000, histories=False)

            ms = _timed(step, args.steps, 1, torch.cuda.current_stream())
            row[key] = {"iterations": int(res["k"]), "ms": ms, "status": int(res["st"])}
            H.close()
        O = omg.Hierarchy(2, prob.n1, prob.stencil, prob.levels)
        A, Ss = O.A[-1], oss.level_smoothers(O)
        row["oracle_iterations"] = {
            "mpcg_m5": ompcg.mpcg(A, prob.b, O.mg_columns, m=5, rtol=RTOL, maxit=20000).iters,
            "pcg": ompcg.mpcg(A, prob.b, lambda r: O.additive_mg(r)[:, None], m=1, rtol=RTOL,
                              maxit=20000).iters,
            "ssor_mpcg_m5": ompcg.mpcg(A, prob.b, lambda r: oss.additive_columns(O, Ss, r, 6), m=5, rtol=RTOL,
                                       maxit=20000).iters,
            "ssor_pcg": opcg.pcg(A, prob.b, lambda r: oss.additive_columns(O, Ss, r, 6).sum(axis=1), rtol=RTOL,
                                 maxit=20000)[1],
            "v33_pcg": opcg.pcg(A, prob.b, lambda r: oss.vcycle(O, Ss, r, 3), rtol=RTOL, maxit=20000)[1]}
        rows.append(row)
    print(json.dumps({"metric": "iterations to 1e-8 rel. residual", "workload": "example1",
                      "config": {"workload": "Section 3 Example 1: (0,1)^2, 160x160 Q1 elements, 4 grids (20x20 "
                                             "coarsest), K = diag(k_xx, 1), f = 1, zero Dirichlet, FP64, rtol 1e-8; "
                                             "mpcg_m5/mpcg_m1/pcg: damped Jacobi nu=2 w=2/3; ssor_*: 6 "
                                             "multicoloured SSOR steps per grid (w=1); v33_pcg: V(3,3) SSOR "
                                             "cycle, exact coarsest solve"},
                      "rows": rows}))
    return 0


def amg_roofline(trace, ns, nnzA, nnzP, C, m, w, peaks):
    """Dominant kernel class of a profiled solve on an algebraic hierarchy
    and its achieved rate: algorithmic bytes per launch are the CSR content
    of the matrix it streams (4-byte column + w-byte value per entry; ELL
    padding excluded) plus the vectors it reads and writes once.  Launch
    order per iteration (one stream): Jacobi J, restriction J, Jacobi J-1,
    restriction J-1, ..., Jacobi 1, restriction 1, coarse solve,
    prolongations P_1 .. P_J (k columns each), then the block kernels."""
    J = len(ns) - 1
    tot = {}
    for cls, ms in trace:
        tot[cls] = tot.get(cls, 0.0) + ms
    dom = max(tot, key=tot.get)
    cnt, jj, jr, jp = 0, J, J, 1
    bytes_sum = dur = 0.0
    launches = 0
    for cls, ms in trace:
        b = None
        if cls == "init":
            cnt = 0
        if cls in ("init", "check"):
            jj, jr, jp = J, J, 1
        if cls == "jacobi":
            b = nnzA[jj] * (4 + w) + 3 * ns[jj] * w
            jj -= 1
        elif cls == "restrict":
            b = nnzP[jr] * (4 + w) + (ns[jr] + ns[jr - 1]) * w
            jr -= 1
        elif cls == "prolong":
            b = nnzP[jp] * (4 + w) + jp * (ns[jp - 1] + ns[jp]) * w
            jp += 1
        elif cls == "spmm":
            b = nnzA[J] * (4 + w) + 2 * C * ns[J] * w
        elif cls in ("orth_update", "gram_window", "update_xr"):
            b, _ = kernel_work(cls, ns[J], C, cnt, w)
        if cls == dom:
            if b is not None:
                bytes_sum += b
            dur += ms
            launches += 1
        if cls == "small_alpha":
            cnt = min(cnt + 1, m)
    share = tot[dom] / sum(tot.values())
    if bytes_sum == 0:
        return dom, None, tot
    ach = bytes_sum / (dur * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": dom, "launches": launches,
           "avg_launch_us": dur / launches * 1e3, "algorithmic_bytes_per_launch": bytes_sum / launches,
           "share_of_solve": share}
    return dom, out, tot


def _timed_flushed(fn, steps, warmup, stream, nvtx=False):
    """Mean CUDA-event time of fn over `steps` calls, each preceded (outside
    its event pair) by a 256 MB write that evicts the 129 MB L2; with nvtx
    every timed call sits in an NVTX range "timed_step"."""
    import torch
    scratch = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        fn()
    total = 0.0
    for _ in range(steps):
        scratch.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if nvtx:
            torch.cuda.nvtx.range_push("timed_step")
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if nvtx:
            torch.cuda.nvtx.range_pop()
        total += e0.elapsed_time(e1)
    return total / steps


def bench_algebraic(args):
    """Algebraic hierarchies (smoothed aggregation, Section 2.1's
    agglomeration; the stand-in for Section 3's BoomerAMG setup).  Headline:
    the Example 2 stand-in, a seeded network of 24 fractures (thickness 1e-4)
    on (0,1)^2 with 545^2 nodes (296,480 unknowns), p = 1 on the right edge,
    unit inflow on the left, conducting fractures k_f = 1e4, k_m = 1; mixed
    precision additive MG-MPCG (m = 5) to rtol 1e-8 on the algebraic
    hierarchy.  Beside it: k_f = 10^-4 .. 10^4 with FP64 MPCG (m = 5 and the
    longest window, m = 16), PCG and MG(V)-PCG (V(3,3) with damped Jacobi) on
    the algebraic hierarchy and mixed MPCG on the geometric one, and Section 3's
    Example 1 (160^2 elements) across k_xx on both hierarchies; the oracle's
    iteration counts at the two extreme k_f and at k_xx = 1e-6."""
    import time
    import torch
    from oracle import amg as oa
    from oracle import mg as omg
    from oracle import mpcg as ompcg
    from oracle import pcg as opcg
    from oracle import ssor as oss
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    _build.build()
    M.load()
    stream = torch.cuda.current_stream()
    peaks = load_peaks()

    def solve_timed(H, b, x, steps, warmup, nvtx=False):
        res = {}

        def step():
            x.zero_()
            res["st"], res["k"], _, _ = H.solve(b, x, rtol=RTOL, maxit=MAXIT, histories=False)

        ms = _timed_flushed(step, steps, warmup, stream, nvtx)
        return ms, int(res["k"]), int(res["st"])

    rows = []
    head = None
    for kf in ((1e4,) if args.headline_only else (1e-4, 1e-2, 1.0, 1e2, 1e4)):
        prob = pb.fracture_network(kf)
        A = pb.stencil_csr(prob)
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        row = {"kf": kf}
        t0 = time.perf_counter()
        Hm = M.AlgebraicHierarchy(A, precision=M.MPCG_MIXED, stream=stream.cuda_stream,
                                  use_graph=0 if args.direct else 1)
        row["setup_s"] = time.perf_counter() - t0
        ns = [M.mg_level_size(Hm.h, j) for j in range(Hm.levels)]
        row["grids"] = ns
        steps = args.steps if kf == 1e4 else 1
        clk = Clocks(0) if kf == 1e4 else None
        ms, k, st = solve_timed(Hm, b, x, steps, args.warmup if kf == 1e4 else 1, nvtx=kf == 1e4)
        clocks = clk.stop() if clk else None
        Ax = torch.empty_like(b)
        M.mg_apply_operator(Hm.h, Hm.levels - 1, x, Ax, 1)
        tr = float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b))
        row["mixed_mpcg"] = {"iterations": k, "ms": ms, "status": st, "true_rel_residual": tr}
        if kf == 1e4:
            x.zero_()
            _, _, _, trace = M.mpcg_solve_profiled(Hm.h, b, x, RTOL, MAXIT)
            nnzA = [M.mg_amg_nnz(Hm.h, j, M.MPCG_AMG_A) for j in range(Hm.levels)]
            nnzP = [0] + [M.mg_amg_nnz(Hm.h, j, M.MPCG_AMG_P) for j in range(1, Hm.levels)]
            dom, rl, tot = amg_roofline(trace, ns, nnzA, nnzP, Hm.levels, M_WINDOW, 4, peaks)
            if rl is not None:
                rl["traffic"] = measured_traffic(f"fracture_mixed:{dom}")
            head = {"value": prob.n / (ms * 1e-3), "ms_per_step": ms, "iterations": k, "true_rel_residual": tr,
                    "roofline": rl, "clocks": clocks, "launches": M.mg_last_launches(Hm.h),
                    "kernel_ms_per_solve": {c: round(v, 4) for c, v in tot.items()}}
            x.zero_()
            ms_steps, _, _ = solve_timed(Hm, b, x, 1, 0)
            head["launches"] = M.mg_last_launches(Hm.h)
        Hm.close()
        if args.headline_only:
            rows.append(row)
            continue
        for key, opts in (("fp64_mpcg", dict(m=M_WINDOW)), ("fp64_mpcg_m16", dict(m=16)),
                          ("fp64_pcg", dict(m=1, sum_columns=1)), ("fp64_vpcg", dict(m=1, vcycle=1, nu=3))):
            H = M.AlgebraicHierarchy(A, stream=stream.cuda_stream, **opts)
            ms, k, st = solve_timed(H, b, x, 1, 1)
            row[key] = {"iterations": k, "ms": ms, "status": st}
            H.close()
        st_dev = torch.from_numpy(prob.stencil).cuda()
        Hg = M.Hierarchy(st_dev, 2, prob.nodes, prob.levels, faces=prob.faces, precision=M.MPCG_MIXED,
                         stream=stream.cuda_stream)
        ms, k, st = solve_timed(Hg, b, x, 1, 1)
        row["geometric_mixed_mpcg"] = {"iterations": k, "ms": ms, "status": st, "grids": prob.levels}
        Hg.close()
        if kf in (1e-4, 1e4) and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            O = oa.AlgebraicHierarchy(A)
            t1 = time.perf_counter()
            r5 = ompcg.mpcg(A, prob.b, O.mg_columns, m=M_WINDOW, rtol=RTOL, maxit=MAXIT)
            t2 = time.perf_counter()
            r1 = ompcg.mpcg(A, prob.b, lambda v: O.additive_mg(v)[:, None], m=1, rtol=RTOL, maxit=MAXIT)
            r16 = ompcg.mpcg(A, prob.b, O.mg_columns, m=16, rtol=RTOL, maxit=MAXIT)
            O3 = oa.AlgebraicHierarchy(A, nu=3)
            Sm = oss.jacobi_smoothers(O3)
            rv = opcg.pcg(A, prob.b, lambda v: oss.vcycle(O3, Sm, v, 3), rtol=RTOL, maxit=MAXIT)
            row["oracle"] = {"mpcg": r5.iters, "mpcg_m16": r16.iters, "pcg": r1.iters, "vpcg": rv[1],
                             "setup_s": t1 - t0, "mpcg_solve_s": t2 - t1}
        rows.append(row)
    ex1 = []
    for n_ in (() if args.headline_only else range(0, 8)):
        kxx = 10.0 ** (-n_)
        prob = pb.example1(kxx)
        A = pb.stencil_csr(prob)
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        H = M.AlgebraicHierarchy(A, stream=stream.cuda_stream)
        ms, k, st = solve_timed(H, b, x, 1, 1)
        r = {"kxx": kxx, "algebraic_mpcg": {"iterations": k, "ms": ms, "grids": H.levels}}
        H.close()
        H = M.AlgebraicHierarchy(A, stream=stream.cuda_stream, m=1, sum_columns=1)
        ms, k, st = solve_timed(H, b, x, 1, 1)
        r["algebraic_pcg"] = {"iterations": k, "ms": ms}
        H.close()
        H = M.AlgebraicHierarchy(A, stream=stream.cuda_stream, m=1, vcycle=1, nu=3)
        ms, k, st = solve_timed(H, b, x, 1, 1)
        r["algebraic_vpcg"] = {"iterations": k, "ms": ms}
        H.close()
        if kxx == 1e-6 and not args.no_cpu_baseline:
            O = oa.AlgebraicHierarchy(A)
            r["oracle"] = {"mpcg": ompcg.mpcg(A, prob.b, O.mg_columns, m=M_WINDOW, rtol=RTOL, maxit=MAXIT).iters,
                           "pcg": ompcg.mpcg(A, prob.b, lambda v: O.additive_mg(v)[:, None], m=1, rtol=RTOL,
                                             maxit=MAXIT).iters}
        ex1.append(r)
    last = rows[-1]
    cpu = None
    if "oracle" in last:
        o = last["oracle"]
        cpu = {"value": 296480 / o["mpcg_solve_s"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
               "sample": f"one full FP64 oracle solve of the headline problem ({o['mpcg']} iterations, "
                         f"{o['mpcg_solve_s']:.1f} s; hierarchy setup {o['setup_s']:.1f} s excluded)"}
    print(json.dumps({
        "metric": METRIC, "workload": "algebraic", "value": head["value"], "unit": "DOFs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "Example 2 stand-in: seeded network of 24 fractures (delta 1e-4) in (0,1)^2, 545^2 "
                               "Q1 nodes, 296,480 unknowns, p=1 right edge, unit inflow left, k_m=1, k_f=1e4; "
                               "smoothed-aggregation hierarchy (theta 0.4, w 4/3, coarse <= 256), damped "
                               "Jacobi nu=2, MPCG m=5, mixed precision, rtol 1e-8",
                   "l2": "working set ~130 MB per solve, about the L2 size: L2 flushed (256 MB write) before "
                         "every timed solve, outside its events"},
        "iterations": head["iterations"], "true_rel_residual": head["true_rel_residual"],
        "roofline": head["roofline"], "kernel_ms_per_solve": head["kernel_ms_per_solve"],
        "gpu_launches": head["launches"] * args.steps, "clocks": head["clocks"], "peaks": peaks,
        "fracture_sweep": rows, "example1": ex1, "cpu_baseline": cpu}))
    return 0


def bench_learned(args):
    """2D high-contrast diffusion, 1025^2 nodes, 9 grids, f = 1, kappa seed 3:
    the mixed-precision solver without and with the learned column; the
    network is trained on the GPU on (residual, error) pairs made by the
    solver itself: by default 4096 pairs of 129^2 problems with kappa seeds
    1000..1015 (FP64 iterates 1..256); --train-nodes 1025 trains on pairs of
    the evaluation size instead (--train-seeds problems, mixed-precision
    iterates 1, 1 + stride, ... below 257)."""
    import numpy as np
    import torch
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    _build.build()
    M.load()
    t0 = time.perf_counter()
    hs, R, E, owner = [], [], [], []
    tn = args.train_nodes
    prec = M.MPCG_FP64 if tn <= 129 else M.MPCG_MIXED   # iterates of the evaluation size: the mixed solver
    for i, sd in enumerate(range(1000, 1000 + args.train_seeds) if args.epochs > 0 else ()):
        prob = pb.diffusion_macro(2, tn, sd)
        H = M.Hierarchy(torch.from_numpy(prob.stencil).cuda(), 2, tn, prob.levels, m=M_WINDOW, precision=prec)
        b = torch.from_numpy(prob.b).cuda()
        xs = torch.zeros_like(b)
        H.solve(b, xs, rtol=1e-12, maxit=20000, histories=False)
        Ax = torch.empty_like(b)
        for k in range(1, 257, args.train_stride):
            x = torch.zeros_like(b)
            H.solve(b, x, rtol=1e-30, maxit=k, histories=False)
            M.mg_apply_operator(H.h, prob.levels - 1, x, Ax, 1)
            r = b - Ax
            nr = torch.linalg.norm(r)
            R.append((r / nr).float())
            E.append(((xs - x) / nr).float())
            owner.append(i)
        hs.append(H)
    gen_s = time.perf_counter() - t0
    print(f"learned workload: {len(R)} training pairs in {gen_s:.1f} s", file=sys.stderr, flush=True)
    params = pb.net_init_params(7)
    t0 = time.perf_counter()
    loss = [float("nan")]
    if args.epochs > 0:   # --epochs 0: the initial (untrained) weights, inference cost only
        loss = M.mg_learned_train([h.h for h in hs], owner, torch.stack(R).contiguous(),
                                  torch.stack(E).contiguous(), params, epochs=args.epochs, batch=8, lr=1e-3)
    train_s = time.perf_counter() - t0
    print(f"learned workload: trained {args.epochs} epochs in {train_s:.1f} s", file=sys.stderr, flush=True)
    prob = pb.diffusion_macro(2, 1025, 3)
    st = torch.from_numpy(prob.stencil).cuda()
    b = torch.from_numpy(prob.b).cuda()
    out = {}
    kap = torch.from_numpy(np.ascontiguousarray(prob.kappa).reshape(-1)).cuda()
    legs = {"plain": M.MPCG_MIXED, "learned": M.MPCG_MIXED, "plain_matrix_free": M.MPCG_MIXED,
            "learned_matrix_free": M.MPCG_MIXED, "plain_fp64": M.MPCG_FP64, "plain_fp64_dw": M.MPCG_FP64_DW,
            "learned_fp64_dw": M.MPCG_FP64_DW, "plain_full_stencil": M.MPCG_MIXED}
    for key, prec in legs.items():
        print(f"learned workload: leg {key}", file=sys.stderr, flush=True)
        # plain_full_stencil: the FP32 kernels on the full 9-plane stencil instead of its symmetric half
        H = M.Hierarchy(st, 2, 1025, prob.levels, m=M_WINDOW, precision=prec,
                        half_stencil=0 if key == "plain_full_stencil" else 1)
        if key.startswith("learned"):
            M.mg_learned_attach(H.h, params)
        if key.endswith("matrix_free"):   # fine operator rebuilt from the element coefficients
            M.mg_attach_q1_kappa(H.h, kap)
        x = torch.zeros_like(b)
        res = {}

        def step():
            x.zero_()
            res["st"], res["k"], _, _ = H.solve(b, x, rtol=RTOL, maxit=50000, histories=False)

        ms = _timed(step, args.steps, 1, torch.cuda.current_stream())
        Ax = torch.empty_like(b)
        M.mg_apply_operator(H.h, prob.levels - 1, x, Ax, 1)
        out[key] = {"ms_per_solve": ms, "iterations": int(res["k"]), "status": int(res["st"]),
                    "dofs_per_s": prob.n / (ms * 1e-3),
                    "true_rel_residual": float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b))}
        if key == "learned":  # live CUDA-event time of the fused tensor-core network kernel
            x.zero_()
            _, _, _, trace = M.mpcg_solve_profiled(H.h, b, x, RTOL, 50000)
            net = [t for c, t in trace if c == "net"]
            if net:
                out[key]["net_us_per_application"] = 1e3 * sum(net) / len(net)
        H.close()
    print(json.dumps({
        "metric": METRIC, "workload": "learned", "value": out["learned"]["dofs_per_s"], "unit": "DOFs/s",
        "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64+bf16", "data": "synthetic",
        "config": {"workload": "2D diffusion 1025^2, 9 grids, log10 kappa U[-2,4] on 16x16 macro cells (seed 3), "
                               "f = 1, MPCG m=5, mixed precision, rtol 1e-8; network 2-16-16-16-1 trained on "
                               f"{len(R)} pairs from {args.train_nodes}^2 problems (kappa seeds 1000-"
                               f"{999 + args.train_seeds})"},
        "plain": out["plain"], "learned": out["learned"],
        "plain_matrix_free": out["plain_matrix_free"], "learned_matrix_free": out["learned_matrix_free"],
        "plain_fp64": out["plain_fp64"], "plain_fp64_dw": out["plain_fp64_dw"],
        "learned_fp64_dw": out["learned_fp64_dw"], "plain_full_stencil": out["plain_full_stencil"],
        # wall time of the plain FP64 solve over that of mixed precision + the learned column
        "speedup_learned_mixed_vs_plain_fp64": out["plain_fp64"]["ms_per_solve"] / out["learned"]["ms_per_solve"],
        "speedup_learned_mixed_vs_plain_mixed": out["plain"]["ms_per_solve"] / out["learned"]["ms_per_solve"],
        "training": {"pairs": len(R), "grid": f"{args.train_nodes}^2", "problems": args.train_seeds,
                     "iterate_stride": args.train_stride, "epochs": args.epochs, "loss_first": float(loss[0]),
                     "loss_last": float(loss[-1]), "pair_generation_s": gen_s, "train_s": train_s}}))
    return 0


def bench_net_kernels(args):
    """Throughput of the learned column's tensor-core kernels on their own:
    inference (mg_learned_forward, 4 images of the 1025^2 field) and one
    training forward + backward pass (mg_learned_grad, 8 pairs of a 257^2
    field; --nodes sets the training grid), then the same for the 3D network
    on the 65^3 elasticity grid (--nodes3 sets its training grid).  The ncu
    captures of these kernels run this workload."""
    import numpy as np
    import torch
    from paper_2402_12833_gb300 import build as _build
    from paper_2402_12833_gb300 import mpcg as M
    from paper_2402_12833_gb300 import problems as pb
    _build.build()
    M.load()
    out = {}
    theta = pb.net_init_params(7)
    theta3 = pb.net_init_params(7, (3, 16, 16, 16, 3), taps=27)
    cases = (("inference", 2, 1025, 4), ("training_pass", 2, args.nodes or 257, 8),
             ("inference3", 3, 65, 4), ("training_pass3", 3, args.nodes3 or 65, 8))
    for key, dim, nodes, nimg in cases:
        if dim == 2:
            prob = pb.diffusion_macro(2, nodes, 21)
            H = M.Hierarchy(torch.from_numpy(prob.stencil).cuda(), 2, nodes, prob.levels)
            th = theta
        else:   # the 3x3x3 network of the elasticity cantilever
            prob = pb.elasticity_cantilever(nodes)
            H = M.Hierarchy(torch.from_numpy(prob.stencil).cuda(), 3, nodes, prob.levels, dofs_per_node=3,
                            faces=prob.faces)
            th = theta3
        R = np.stack([pb.normal(40 + k, prob.n) for k in range(nimg)])
        R /= np.linalg.norm(R, axis=1, keepdims=True)
        Rd = torch.from_numpy(R.astype(np.float32)).cuda()
        if key.startswith("inference"):
            M.mg_learned_attach(H.h, th)
            Y = torch.zeros_like(Rd)
            fn = lambda: M.mg_learned_forward(H.h, Rd, Y, nimg)
        else:
            Ed = torch.from_numpy(np.stack([pb.normal(50 + k, prob.n) for k in range(nimg)]).astype(np.float32)).cuda()
            fn = lambda: M.mg_learned_grad(H.h, th, Rd, Ed, nimg)
        ms = _timed(fn, args.steps, args.warmup, torch.cuda.current_stream())
        out[key] = {"grid": f"{nodes}^{dim}", "images": nimg, "ms_per_call": ms, "us_per_image": 1e3 * ms / nimg}
        H.close()
    print(json.dumps({"metric": "learned-column kernel throughput", "workload": "net_kernels", "unit": "us/image",
                      **out, "note": "each call is synchronous through the C ABI (includes its host round trip "
                                     "and, for the 3D calls, the allocation of the activations)"}))
    return 0


def main():
    faulthandler.enable()   # a native crash prints the Python stack of the call that made it
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["poisson3d", "batched", "learned", "elasticity", "example1", "algebraic",
                                           "net_kernels"],
                    default="poisson3d",
                    help="poisson3d: the headline line; batched / learned / elasticity: the other workloads")
    ap.add_argument("--epochs", type=int, default=20, help="training epochs of the learned workload")
    ap.add_argument("--train-nodes", type=int, default=129, help="learned workload: nodes per side of the training problems")
    ap.add_argument("--train-seeds", type=int, default=16, help="learned workload: number of training problems")
    ap.add_argument("--train-stride", type=int, default=1, help="learned workload: stride of the iterates 1..256 used as pairs")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="algebraic workload: the headline solve only (no sweeps, no oracle)")
    ap.add_argument("--matrix-free", action="store_true",
                    help="with --only mixed: the matrix-free fine operator in the timed solve")
    ap.add_argument("--direct", action="store_true",
                    help="launch kernels directly instead of one graph per solve (for ncu launch lists)")
    ap.add_argument("--only", choices=["mixed", "fp64", "fp64_dw"], default=None,
                    help="time one precision only and print its figures (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the fixed launch-shape rules only (no autotuning)")
    ap.add_argument("--nodes", type=int, default=None,
                    help="with --only: nodes per side of the 3D Poisson grid (smaller cases for profiling)")
    ap.add_argument("--nodes3", type=int, default=None,
                    help="with --workload net_kernels: nodes per side of the 3D training-pass grid")
    args = ap.parse_args()
    if args.nodes is not None:
        if args.only is None and args.workload != "net_kernels":
            ap.error("--nodes goes with --only or --workload net_kernels")
        global NODES
        NODES = args.nodes
    if args.warmup < 3 and args.impl == "ours" and args.only is None and args.workload != "net_kernels":
        print("note: warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)
    if args.workload == "batched":
        return bench_batched(args)
    if args.workload == "elasticity":
        return bench_elasticity(args)
    if args.workload == "example1":
        return bench_example1(args)
    if args.workload == "algebraic":
        return bench_algebraic(args)
    if args.workload == "learned":
        return bench_learned(args)
    if args.workload == "net_kernels":
        return bench_net_kernels(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
