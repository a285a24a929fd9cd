#!/usr/bin/env python
"""Benchmark: 2D deflated, CSLP-multigrid-preconditioned GMRES solve to 1e-7
on the GB300 (one solve = one step), plus operator / V-cycle bandwidth.

Workload (one step): MP 2-A, unit square, constant k = 200, p = 3, 320 x 320
elements (n = 103 041 complex128 dofs), unit point source at the centre,
CSLP shift (1, 0.5), one V-cycle (nu = 1/1), ADP deflation, FP64 throughout,
tol 1e-7, maxit 100.  Inputs are resident on the device before the timed
region; L2 is flushed (a 512 MiB buffer is written) before every timed solve.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# dram__bytes_read.sum + dram__bytes_write.sum of k_kron2d<3, double, EPI_Y, 32, 8> applying A
# at n = 321^2 (one ncu capture, L2 cold); the algorithmic bytes are 16 B in + 16 B out per dof
APPLY_DRAM_BYTES = 1695232
K_WAVE, P_DEG, N_EL = 200.0, 3, 320
METRIC = "2D solve time to 1e-7 rel. residual + iterations; apply/V-cycle HBM GB/s vs peak"
WORKLOAD = f"MP2-A constant k={int(K_WAVE)}, p={P_DEG}, {N_EL}x{N_EL} elements, centre point source"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time(ms: float, ws: int, dist=None, device="cuda"):
    """Replicas: every rank solves its own instance each step, so one step of
    the job takes the slowest rank's time and retires ws solves.  Returns
    (max over ranks of the per-step time, job-level time per solve).  The
    reduction is a MAX all-reduce on `device` followed by a barrier; with one
    rank (or no process group) it is the identity."""
    if dist is not None and ws > 1:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    return ms, ms / ws


# ---------------------------------------------------------------------------- CPU oracle legs
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle.solver import Solver
pr = W.config2(k={k}, p={p})
t0 = time.perf_counter(); s = Solver(pr); f = s.load(); t1 = time.perf_counter()
times, iters = [], None
for _ in range({reps}):
    a = time.perf_counter(); r = s.solve(f, tol=1e-7, maxit=100); times.append(time.perf_counter() - a); iters = r.iters
print(json.dumps({{"setup_s": t1 - t0, "solve_s": times, "iters": iters, "true_res": r.true_res}}))
"""


def run_oracle(reps: int, threads: int = 1) -> dict:
    """FP64 oracle on the host cores: `threads` BLAS/OpenMP threads (1 =
    single-threaded, the paper's serial setting)."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, k=K_WAVE, p=P_DEG, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cpu() -> dict:
    """Core count and model of the host the oracle runs on."""
    info = {"nproc": os.cpu_count(), "machine": platform.machine(), "model": None}
    try:
        with open("/proc/cpuinfo") as fh:
            fields = {}
            for line in fh:
                if ":" in line:
                    k_, v_ = (x.strip() for x in line.split(":", 1))
                    fields.setdefault(k_, v_)
        if "model name" in fields:
            info["model"] = fields["model name"]
        elif "CPU part" in fields:
            info["model"] = f"implementer {fields.get('CPU implementer')} part {fields['CPU part']}"
    except OSError:
        pass
    return info


def cpu_baseline_record(reps: int = 3) -> dict:
    """The oracle timed on this host: `reps` solves single-threaded (the
    reported value, median) and `reps` with every core, setup and solve
    reported separately."""
    one = run_oracle(reps, 1)
    med = lambda xs: sorted(xs)[len(xs) // 2]
    rec = {"value": 1000.0 * med(one["solve_s"]), "unit": "ms", "cores": 1, "kind": "oracle",
           "sample": f"{reps} full FP64 oracle solves of the bench problem, single-threaded, median, setup excluded",
           "iters": one["iters"], "setup_s": one["setup_s"],
           "solve_ms_runs": [1000.0 * x for x in one["solve_s"]], "host": host_cpu()}
    ncores = os.cpu_count() or 1
    if ncores > 1:
        try:
            allc = run_oracle(reps, ncores)
            rec["all_cores"] = {"cores": ncores, "solve_ms_median": 1000.0 * med(allc["solve_s"]),
                                "setup_s": allc["setup_s"], "iters": allc["iters"]}
        except Exception as e:       # report, do not hide
            rec["all_cores"] = {"cores": ncores, "error": str(e)[:200]}
    return rec


def reference_arm(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    r = run_oracle(args.warmup + args.steps)
    times = r["solve_s"][args.warmup:]
    ms = 1000.0 * sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "iterations": r["iters"],
        "config": {"workload": WORKLOAD, "n_dof": (N_EL + P_DEG - 2) ** 2, "tol": 1e-7},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full FP64 oracle solves of the same problem (setup excluded)"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------- GPU arm
def gpu_arm(args):
    import numpy as np
    import torch
    import workloads as W
    from paper_2010_10232_gb300 import _ffi
    from paper_2010_10232_gb300.solver import Helmholtz, from_problem
    import ctypes as C

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lib = _ffi.lib()
    stream = torch.cuda.current_stream()
    pr = W.config2(k=K_WAVE, p=P_DEG)
    h = from_problem(pr)
    f = h.point_source(*pr.sources[0])
    x = h.vec()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        _, iters, hist, tr, st = h.solve(f, x=x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = lib.iga_launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
            _, iters, hist, tr, st = h.solve(f, x=x)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = lib.iga_launch_count() - launches0 - 0   # fill_ is torch's, not counted
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms, value = job_time(ms, ws, dist)     # job-level time per solve: N replicas solve N instances per step

    # ---- end to end through the public API with host buffers (copies inside the timed region)
    fh = f.cpu().numpy()
    h.solve_host(fh)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_t = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 255)
        torch.cuda.synchronize()
        a = time.perf_counter()
        xh, it2, *_ = h.solve_host(fh)
        e2e_t.append(time.perf_counter() - a)
    e2e_ms = 1000.0 * sum(e2e_t) / len(e2e_t)
    _, e2e_ms = job_time(e2e_ms, ws, dist)

    # ---- dominant kernel: FP64 operator apply (constant-k banded tile kernel), timed alone
    peaks, src = _peaks()
    reps = 200
    xr = torch.randn(h.n, dtype=torch.complex128, device="cuda")
    yr = h.vec()
    for _ in range(10):
        h.apply_A(xr, yr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        h.apply_A(xr, yr)
    e1.record(stream)
    torch.cuda.synchronize()
    t_apply = e0.elapsed_time(e1) / reps * 1e-3
    W_ = 2 * P_DEG + 1
    flops_dof = 16 * W_ + 8                      # x-pass 2 bands, y-pass 2 bands, complex scale
    apply_flops = flops_dof * h.n
    apply_bytes = 32 * h.n
    # FP64 / FP32 FMA ceilings from the probe kernel
    sink = torch.zeros(2, dtype=torch.float64, device="cuda")
    import measure
    from measure import build as mbuild
    mbuild.build()
    mlib = measure.lib()
    probe = {}
    for prec, name in ((0, "fp64"), (1, "fp32")):
        fl = C.c_double(0.0)
        its = 4096 if prec == 0 else 65536
        mlib.measure_probe_fma(prec, 64, C.c_void_p(sink.data_ptr()), C.c_void_p(stream.cuda_stream), C.byref(fl))
        e0.record(stream)
        mlib.measure_probe_fma(prec, its, C.c_void_p(sink.data_ptr()), C.c_void_p(stream.cuda_stream), C.byref(fl))
        e1.record(stream)
        torch.cuda.synchronize()
        probe[name] = fl.value / (e0.elapsed_time(e1) * 1e-3) / 1e12
    fp64_nominal = 1.25                            # TFLOP/s, GB300 FP64 (profiling recipe)
    achieved_gflops = apply_flops / t_apply / 1e9

    # ---- out-of-L2 operator / V-cycle bandwidth (n = 4097^2, 268 MB per complex128 vector)
    big = {}
    try:
        hb64 = Helmholtz(dim=2, p=P_DEG, n_el=4096, kfield=K_WAVE * 4096 / N_EL, skip_deflation=1)
        nb = hb64.n
        xb = torch.randn(nb, dtype=torch.complex128, device="cuda")
        yb = hb64.vec()
        for _ in range(3):
            hb64.apply_A(xb, yb)
        e0.record(stream)
        for _ in range(10):
            hb64.apply_A(xb, yb)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 10 * 1e-3
        big["apply_fp64_n"] = nb
        big["apply_fp64_gbs"] = 32 * nb / tb / 1e9
        big["apply_fp64_tflops"] = flops_dof * nb / tb / 1e12
        del hb64, yb
        hb32 = Helmholtz(dim=2, p=P_DEG, n_el=4096, kfield=K_WAVE * 4096 / N_EL, skip_deflation=1, precision=1)
        zb = hb32.vec()
        for _ in range(2):
            hb32.vcycle(xb, zb)
        e0.record(stream)
        for _ in range(5):
            hb32.vcycle(xb, zb)
        e1.record(stream)
        torch.cuda.synchronize()
        tv = e0.elapsed_time(e1) / 5 * 1e-3
        # algorithmic bytes of one FP32 V-cycle (nu = 1/1) with complex64 storage:
        # per level n_l*(16 jacobi0 + 24 residual + 8 restrict-read + 16 prolong rmw + 24 post)
        # + n_{l+1}*(8 restrict-write + 8 prolong-read); plus the c128<->c64 conversions at level 0.
        ns = [hb32.level_n(l) for l in range(hb32.levels)]
        vb = sum(ns[l] * 88 + ns[l + 1] * 16 for l in range(len(ns) - 1)) + 48 * ns[0]
        big["vcycle_fp32_gbs"] = vb / tv / 1e9
        big["vcycle_fp32_ms"] = tv * 1e3
        big["vcycle_fp32_bytes"] = vb
        del hb32, zb, xb
    except Exception as e:       # report, do not hide
        big["error"] = str(e)[:200]

    forms = {} if (args.no_forms or ws > 1) else other_forms(h, f, x, stream, flush, ws)
    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline_record(3)
        except Exception as e:
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:200]}
    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_dof": h.n, "coarse_dof": h.m, "levels": h.levels, "tol": 1e-7,
                   "precision": "fp64", "l2": "flushed (512 MiB write) before every timed solve",
                   "parallelism": f"replicas x{ws}"},
        "iterations": iters, "true_res": tr,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 16 * h.n, "d2h_bytes_per_step": 16 * h.n},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_kron2d<3,double,EPI_Y> (apply A)", "bound": "alu",
                     "achieved": achieved_gflops / 1e3, "peak": fp64_nominal, "unit": "TFLOP/s",
                     "frac": achieved_gflops / 1e3 / fp64_nominal, "traffic": APPLY_DRAM_BYTES,
                     "traffic_note": "DRAM bytes read + written per launch, one ncu capture at this size "
                                     "(cold L2; the output stays in L2, so about the x read)",
                     "algorithmic": f"{flops_dof} flop/dof x {h.n} dofs per launch",
                     "peak_source": "nominal FP64 of the profiling recipe",
                     "probe_fma_tflops": probe, "launch_us": t_apply * 1e6,
                     "hbm_gbs": apply_bytes / t_apply / 1e9},
        "out_of_l2": dict(big, hbm_peak_gbs=peaks.get("hbm_gbs"), peak_source=src),
        "forms": forms,
        "clocks": clk.summary(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))


def _time_solves(h, f, x, stream, flush, reps):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        _, it, hist, tr, st = h.solve(f, x=x)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / reps, it, tr


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def other_forms(h64, f, x, stream, flush, ws):
    """Mixed precision, learned correction and the batched 64-instance launch,
    each with its error against the oracle's direct FP64 solution."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2010_10232_gb300.solver import from_problem, solve_batched
    out = {}
    pr = W.config2(k=K_WAVE, p=P_DEG)
    ref = None
    try:
        from oracle.solver import Solver, rel_err      # error report only (CPU, untimed)
        s_or = Solver(pr)
        ref = s_or.direct(s_or.load())
    except Exception as e:
        out["oracle_error"] = str(e)[:200]
    err = (lambda u: float(np.linalg.norm(u - ref) / np.linalg.norm(ref))) if ref is not None else (lambda u: None)
    def tight(h):
        """error of the same form solved to a relative residual of 1e-10"""
        xt = h.vec()
        _, it_t, _, tr_t, st_t = h.solve(f, x=xt, tol=1e-10, maxit=300)
        return {"rel_err_vs_oracle_direct": err(xt.cpu().numpy()), "iterations": it_t, "status": st_t}

    out["plain_fp64"] = {"rel_err_vs_oracle_direct": err(x.cpu().numpy()), "tol_1e-10": tight(h64)}
    try:
        hm = from_problem(pr, precision=1)
        xm = hm.vec()
        hm.solve(f, x=xm)
        ms, it, tr = _time_solves(hm, f, xm, stream, flush, 5)
        out["mixed_fp32_vcycle"] = {"ms": ms, "iterations": it, "true_res": tr,
                                    "rel_err_vs_oracle_direct": err(xm.cpu().numpy()), "tol_1e-10": tight(hm)}
        wpath = os.path.join(ROOT, "paper_2010_10232_gb300", "weights", "cslp_correction.npz")
        if os.path.exists(wpath):
            from paper_2010_10232_gb300.learned import Net
            d = np.load(wpath)
            net = Net(seed=0)
            net.set_params(d["params"])
            hm.attach(net, float(d["gamma"]))
            hm.solve(f, x=xm)
            ms, it, tr = _time_solves(hm, f, xm, stream, flush, 5)
            out["learned_correction"] = {"ms": ms, "iterations": it, "true_res": tr,
                                         "rel_err_vs_oracle_direct": err(xm.cpu().numpy()), "tol_1e-10": tight(hm)}
            # the network alone on the bench grid (one correction's inference)
            nx = hm.level_nx(0)
            xin = torch.zeros(1, nx, nx, 16, dtype=torch.bfloat16, device="cuda")
            xin[..., :3] = torch.randn(1, nx, nx, 3, device="cuda").to(torch.bfloat16)
            for _ in range(3):
                net.forward(xin)
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            for _ in range(20):
                net.forward(xin)
            b_.record()
            torch.cuda.synchronize()
            us = a_.elapsed_time(b_) / 20 * 1e3
            flop = 2 * 9 * (3 * 32 + 32 * 32 + 32 * 32 + 32 * 2) * nx * nx     # algorithmic, unpadded channels
            bf16_peak = _measured_peaks().get("bf16_tflops")
            out["learned_correction"]["cnn_forward"] = {
                "us": us, "pixels": nx * nx, "tflops": flop / us / 1e6,
                "frac_of_bf16_peak": (flop / us / 1e6 / bf16_peak) if bf16_peak else None,
                "note": "3x3 convs 3-32-32-32-2, bf16 mma.sync with FP32 accumulation; bound by launches "
                        "and the pack/epilogue traffic at this size, not by the tensor pipe"}
            hm.attach(None)
        del hm
    except Exception as e:
        out["mixed_error"] = str(e)[:200]
    try:
        inst = W.config4(64)
        ctxs, rhs = [], []
        for prb, nr in inst:
            c = from_problem(prb, precision=1)
            ctxs.append(c)
            rhs.append(torch.stack([c.point_source(*s_) for s_ in prb.sources]))
        solve_batched(ctxs, rhs)                    # warm-up (also builds every workspace)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        e0.record(stream)
        xs, its, sts, rc = solve_batched(ctxs, rhs)
        e1.record(stream)
        torch.cuda.synchronize()
        tot = sum(len(r) for r in rhs)
        ms = e0.elapsed_time(e1)
        allit = np.concatenate(its)
        out["batched_cfg4"] = {"instances": len(ctxs), "rhs": int(tot), "ms_total": ms,
                               "ms_per_solve": ms / tot, "dofs": int(sum(c.n for c in ctxs)),
                               "iterations_mean": float(allit.mean()), "iterations_max": int(allit.max()),
                               "status": int(rc), "note": "one CUDA-graph launch, FP32 V-cycle, FP64 FGMRES"}
        del ctxs, rhs, xs
        # the same method unbatched, and the plain FP64 form, on every 8th
        # instance (all its right-hand sides): one solve call after another
        sub = inst[::8]
        ctxs32 = [from_problem(prb, precision=1) for prb, _ in sub]
        ctxs64 = [from_problem(prb, precision=0) for prb, _ in sub]
        rhs = [torch.stack([c.point_source(*s_) for s_ in prb.sources]) for c, (prb, _) in zip(ctxs32, sub)]
        nsub = sum(len(r) for r in rhs)

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        def seq(cs):
            def run():
                for c, r in zip(cs, rhs):
                    x_ = c.vec()
                    for j in range(r.shape[0]):
                        c.solve(r[j], x=x_)
            return run
        out["batched_vs_sequential"] = {
            "instances": len(sub), "rhs": int(nsub),
            "batched_ms": timed(lambda: solve_batched(ctxs32, rhs)),
            "sequential_same_method_ms": timed(seq(ctxs32)),
            "sequential_plain_fp64_ms": timed(seq(ctxs64)),
            "note": "every 8th instance of the 64, all of its right-hand sides"}
        del ctxs32, ctxs64, rhs
    except Exception as e:
        out["batched_error"] = str(e)[:200]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
