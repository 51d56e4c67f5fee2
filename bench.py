#!/usr/bin/env python
"""Benchmark: nonlocal P1 stiffness assembly on GB300 (one JSON line on rank 0).

Workload (default): regular 32-gon ball, delta = 0.1, (-0.1, 1.1)^2 split into
96 x 96 squares (18432 triangles) with vertices jittered by U[-0.2h, 0.2h]
(seed 1077502), psi = 4/(pi delta^4), 16-point outer and 7-point inner rules,
FP64 geometry with FP32-compensated quadrature.  One step = one full assembly
(cell list, pair geometry + quadrature, symbolic CSR pattern, numeric scatter)
from a mesh already in HBM to the finished CSR.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torchrun: every rank assembles its own copy of the workload
(independent problems, no data-path collective: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "assembly qp-pairs/s & ms/matrix, FP32-comp vs FP64 GPU at rel err <=1e-6"
UNIT = "qp-pairs/s"
# algorithmic work per unit, counted from the quadrature of Secs. 5-6 and the local
# blocks of Sec. 7.2: the inner-point
# evaluation (map, phi_b, omega, s0, s1, S2) and the per-(T_a, q, T_b) outer combination
FLOP_PER_QP = 37.0
FLOP_PER_INTER = 48.0
SMS, FP32_LANES = 152, 128
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate (nominal); the measured one comes from nl_fma_peak
# DRAM bytes (read + write) of the numeric phase (k_interior + k_boundary + k_deferred) of
# one assembly, from one ncu capture of the current kernels (profiles/k_boundary_<workload>.md)
NCU_TRAFFIC = {"ngon32_96": (380.4e6, "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_interior + k_boundary "
                                      "+ k_deferred + k_defer_merge, profiles/numeric_traffic_ngon32_96.md")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ngon32_96")
    ap.add_argument("--prec", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--solve", action="store_true",
                    help="after the assembly, extract A, form F and solve A U = F by CG (u = |x|^2)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other benchmark configurations (barycenter_32, singular_128, solve_220, "
                         "batch64, paper Table 1 balls) reported under 'configs'")
    ap.add_argument("--peaks-only", action="store_true",
                    help="print the measured FP32 / FP64 FMA throughput of the GPU and exit")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, dev, dist=None):
    """The largest value of x over the ranks (every rank gets it): the job's time is
    that of its slowest rank.  x is a float; dev the device of the reduction buffer."""
    import torch
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_local, world, dev, dist=None):
    """Whole-job throughput of N replicas: the units all ranks processed divided by the
    slowest rank's time (weak scaling: every rank does the same work)."""
    return units_per_rank * world / max_over_ranks(seconds_local, dev, dist)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(problem, seconds, steps=1):
    """The FP64 oracle as it stands, on a bounded sample of outer triangles of the same
    workload (evenly spaced, each against every triangle), timed on the host cores."""
    import numpy as np

    from oracle import oracle as O
    cores = os.cpu_count() or 1
    K = problem.mesh.nt
    cfg = dict(delta=problem.delta, ball=problem.ball, outer=problem.outer, inner=problem.inner,
               kernel=problem.kernel, kernel_c=problem.kernel_c, ngon_off=problem.ngon_off, cap_m=problem.cap_m)
    # calibrate on a small sample, then size the sample to about `seconds`
    probe = np.linspace(0, K - 1, num=max(cores, 4)).astype(np.int32)
    t0 = time.perf_counter()
    O.assemble(problem.mesh, cfg, a_list=probe, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    m = int(min(K, max(cores, len(probe) * seconds / dt)))
    res = []
    for s in range(steps):
        a_list = ((np.arange(m) * (K / m) + s * 0.37 * K / m) % K).astype(np.int32)
        t0 = time.perf_counter()
        out = O.assemble(problem.mesh, cfg, a_list=a_list, nthreads=cores)
        res.append((out["n_qp_pairs"], time.perf_counter() - t0, m))
    qp = sum(r[0] for r in res)
    tt = sum(r[1] for r in res)
    return {"value": qp / tt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} of {K} outer triangles (evenly spaced) x all {K} inner triangles, "
                      f"{qp // max(steps, 1)} qp-pairs per step, FP64"}, tt / steps


def cpu_baseline_batch(problems, seconds):
    """The FP64 oracle on a bounded sample of the batched workload: a few evenly spaced
    outer triangles of every problem (each against every triangle of its mesh)."""
    import numpy as np

    from oracle import oracle as O
    cores = os.cpu_count() or 1

    def cfg(p):
        return dict(delta=p.delta, ball=p.ball, outer=p.outer, inner=p.inner, kernel=p.kernel,
                    kernel_c=p.kernel_c, ngon_off=p.ngon_off, cap_m=p.cap_m)
    p0 = problems[0]
    probe = np.linspace(0, p0.mesh.nt - 1, num=max(cores, 4)).astype(np.int32)
    t0 = time.perf_counter()
    O.assemble(p0.mesh, cfg(p0), a_list=probe, nthreads=cores)
    per_a = max(time.perf_counter() - t0, 1e-3) / len(probe) / p0.mesh.nt   # seconds per outer triangle per K
    per_round = per_a * sum(p.mesh.nt for p in problems)
    k = max(1, int(seconds / per_round))
    qp, tt, na = 0, 0.0, 0
    for p in problems:
        K = p.mesh.nt
        a_list = np.linspace(0, K - 1, num=min(k * max(cores, 1), K)).astype(np.int32)
        t0 = time.perf_counter()
        out = O.assemble(p.mesh, cfg(p), a_list=a_list, nthreads=cores)
        tt += time.perf_counter() - t0
        qp += out["n_qp_pairs"]
        na += len(a_list)
        if tt > 2.0 * seconds:
            break
    return {"value": qp / tt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{na} outer triangles spread evenly over the problems of the batch, each against every "
                      f"triangle of its mesh, {qp} qp-pairs, FP64"}, tt


def batch_bench(args, nl, ctx, stream, dev, world, dist, rank, cpu_seconds=None):
    """The batched workload: 64 independent assemblies (delta 0.05 .. 0.2, K 2450 .. 38088,
    nocaps / approxcaps) in one nl_assemble_batch, against 64 sequential nl_assemble calls;
    re-assembly by the captured graph (nl_batch_run) against 64 nl_assemble_numeric calls."""
    import numpy as np
    import torch

    from paper_2005_10775_gb300 import inputs as I
    probs = I.batch_problems()
    keep = nl._Keep()

    def dev_mesh(m):
        return nl.make_mesh(type("DevMesh", (), dict(vx=torch.tensor(m.vx, device=dev),
                                                     vy=torch.tensor(m.vy, device=dev),
                                                     tri=torch.tensor(m.tri, device=dev))), keep)
    meshes = [dev_mesh(p.mesh) for p in probs]

    def cfgs_for(prec):
        return [nl.config_of(p, keep, prec=prec) for p in probs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return max_over_ranks(tot, dev, dist) / steps

    state = {}

    def batch_once(cfgs, keep_out=False):
        outs = nl.nl_assemble_batch(ctx, meshes, cfgs)
        state["stats"] = [(o.n_pairs, o.n_qp_pairs, o.n_inter, o.nnz) for o in outs]
        if keep_out:
            return outs
        for o in outs:
            nl.nl_csr_free(ctx, o)

    def seq_once(cfgs):
        for mh, c in zip(meshes, cfgs):
            o = nl.nl_assemble(ctx, mh, c)
            nl.nl_csr_free(ctx, o)

    cfgs = cfgs_for(args.prec)
    # first batch of this shape: the autotuner picks the schedule (kept in the context)
    h, outs = nl.nl_batch_create(ctx, meshes, cfgs)
    tune = nl.nl_batch_get_info(h)
    # the staged path once more (schedule from the cache): its phases, one numeric phase of all
    # problems for the roofline (nl_assemble_batch pipelines the phases, which then overlap)
    h2, outs2 = nl.nl_batch_create(ctx, meshes, cfgs)
    phases = np.array(nl.nl_last_timings(ctx), dtype=np.float64)
    nl.nl_batch_destroy(ctx, h2)
    for o in outs2:
        nl.nl_csr_free(ctx, o)
    for _ in range(args.warmup):
        batch_once(cfgs)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    l0 = nl.nl_launch_count(ctx)
    ms_batch = timed(lambda: batch_once(cfgs), args.steps, 0)
    launches = nl.nl_launch_count(ctx) - l0
    ck = clocks.stop()
    stats = np.array(state["stats"], dtype=np.int64)
    n_qp = int(stats[:, 1].sum())
    n_inter = int(stats[:, 2].sum())
    ms_seq = timed(lambda: seq_once(cfgs), max(1, args.steps // 2), 1)
    # re-assembly of the values: one graph launch against 64 numeric calls
    ms_replay = timed(lambda: nl.nl_batch_run(ctx, h), args.steps, 1)

    def seq_numeric():
        for o in outs:
            nl.nl_assemble_numeric(ctx, o)
    ms_seq_num = timed(seq_numeric, args.steps, 1)
    nl.nl_batch_destroy(ctx, h)
    for o in outs:
        nl.nl_csr_free(ctx, o)
    fp64 = None
    if args.fp64_steps > 0 and args.prec != "fp64":
        c64 = cfgs_for("fp64")
        ms64 = timed(lambda: batch_once(c64), args.fp64_steps, 1)
        fp64 = {"ms_per_step": ms64, "value": n_qp * world / (ms64 / 1e3)}
    e2e = None
    if not args.no_e2e:
        hmeshes = [nl.make_mesh(p.mesh, keep) for p in probs]
        hcfgs = [nl.config_of(p, keep, prec=args.prec) for p in probs]
        nnzs = [int(s[3]) for s in state["stats"]] if state.get("stats") else [1] * len(probs)
        bufs = [(torch.empty(p.mesh.nv + 1, dtype=torch.int64).pin_memory(),
                 torch.empty(max(z, 1), dtype=torch.int32).pin_memory(),
                 torch.empty(max(z, 1), dtype=torch.float64).pin_memory()) for p, z in zip(probs, nnzs)]

        def e2e_once():
            os_ = nl.nl_assemble_batch(ctx, hmeshes, hcfgs)
            for o, (rp, ci, va) in zip(os_, bufs):
                nl._check(ctx, nl.LIB.nl_csr_download(ctx, nl.ctypes.byref(o), rp.data_ptr(), ci.data_ptr(),
                                                      va.data_ptr()))
                nl.nl_csr_free(ctx, o)
        e2e_once()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_once()
        torch.cuda.synchronize()
        e2e_value = job_throughput(n_qp, (time.perf_counter() - t0) / args.steps, world, dev, dist)
        h2d = sum(p.mesh.vx.nbytes + p.mesh.vy.nbytes + p.mesh.tri.nbytes for p in probs)
        d2h = sum(8 * (p.mesh.nv + 1) + 12 * z for p, z in zip(probs, nnzs))
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    peaks, src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = (FLOP_PER_QP * n_qp + FLOP_PER_INTER * n_inter) / (phases[1] / 1e3) / 1e12
    Ks = [p.mesh.nt for p in probs]
    line = {
        "metric": METRIC, "value": n_qp * world / (ms_batch / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32c" if args.prec == "fp32c" else "f64",
        "data": "synthetic",
        "config": {"workload": "batch64", "problems": len(probs), "K_total": int(sum(Ks)), "K_min": min(Ks),
                   "K_max": max(Ks), "deltas": list(I.BATCH_DELTAS), "balls": "nocaps / approxcaps (m=2)",
                   "outer": "dunavant7", "inner": "dunavant7", "kernel": "const",
                   "parallelism": f"replica x{world}", "l2": "flushed (512 MB write) before every step",
                   "n_qp_pairs": n_qp, "n_inter": n_inter, "nnz_total": int(stats[:, 3].sum()),
                   "phase_ms_staged": {"prepare": phases[0], "numeric": phases[1], "symbolic": phases[2],
                                       "scatter": phases[3],
                                       "what": "nl_batch_create (phases one after the other, numeric phase "
                                               "in the tuned schedule); nl_assemble_batch, timed here, "
                                               "pipelines them per problem"},
                   "schedule": tune},
        "sequential": {"ms_per_step": ms_seq, "value": n_qp * world / (ms_seq / 1e3),
                       "what": "64 nl_assemble calls, one after the other"},
        "speedup_batch_vs_sequential": ms_seq / ms_batch,
        "reassembly": {"graph_ms": ms_replay, "sequential_numeric_ms": ms_seq_num,
                       "speedup": ms_seq_num / ms_replay,
                       "what": "values on unchanged meshes: one nl_batch_run graph launch vs 64 "
                               "nl_assemble_numeric calls"},
        "fp64": fp64,
        "speedup_fp32c_vs_fp64": (fp64["ms_per_step"] / ms_batch) if fp64 else None,
        "roofline": {"bound": "alu",
                     "kernel": "k_interior_batch + k_boundary_batch + k_deferred_batch (pair geometry + quadrature, "
                               "all problems)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"FP32 FMA: {SMS} SMs x {FP32_LANES} lanes x 2 x {sm_mhz:.0f} MHz "
                                    f"(clock from MEASURED_PEAKS.json, {src})",
                     "traffic": None},
        "clocks": ck,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_baseline_batch(probs, args.cpu_seconds if cpu_seconds is None else cpu_seconds)
    return line


def solve_phase(nl, ctx, m, p, prec, stream, dev, keep):
    """A = D[Omega, Omega], F = G - D[Omega, Omega_I] g and the CG solve to 1e-10 for u = |x|^2
    (f = -4), timed with CUDA events on the library's stream; one FP32 SpMV timed for GB/s."""
    import numpy as np
    import torch
    hmesh = nl.make_mesh(m, keep)
    dcfg = nl.make_config(keep, p.delta, p.ball, p.outer, p.inner, p.kernel, p.kernel_c, p.ngon_off, p.cap_m, prec)
    D = nl.nl_assemble(ctx, hmesh, dcfg)
    u = m.vx ** 2 + m.vy ** 2
    f = np.full_like(u, -4.0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    A, B = nl.nl_extract(ctx, D, hmesh)
    F = torch.tensor(nl.nl_rhs(ctx, B, hmesh, f, u), device=dev)
    ev[1].record(stream)
    x = torch.zeros_like(F)
    it, rel = nl.nl_cg(ctx, A, F, x, rtol=1e-10, max_it=20000)
    ev[2].record(stream)
    torch.cuda.synchronize()
    om = m.node_in_omega.astype(bool)
    err = float(np.abs(x.cpu().numpy() - u[om]).max())
    # one FP32 matrix-vector product (the CG inner loop's kernel): bytes = values + columns + x + y.
    # The calls are captured in a CUDA graph so that the host side of each call is not timed.
    y = torch.empty_like(F)
    nl.nl_matvec(ctx, A, x, y, prec="fp32c")
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    spmv_timing = "CUDA graph of %d calls" % reps
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            for _ in range(reps):
                nl.nl_matvec(ctx, A, x, y, prec="fp32c")
        g.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        g.replay()
        e1.record(stream)
    except Exception:   # capture refused: time the calls themselves (host time included)
        torch.cuda.synchronize()
        spmv_timing = "%d calls in a row (host time included)" % reps
        e0.record(stream)
        for _ in range(reps):
            nl.nl_matvec(ctx, A, x, y, prec="fp32c")
        e1.record(stream)
    e1.synchronize()
    spmv_ms = e0.elapsed_time(e1) / reps
    spmv_bytes = A.nnz * 8 + (A.n + 1) * 8 + 2 * A.n * 8
    out = {"J_omega": int(A.n), "nnz_A": int(A.nnz), "extract_rhs_ms": ev[0].elapsed_time(ev[1]),
           "cg_ms": ev[1].elapsed_time(ev[2]), "cg_inner_iterations": it, "relres": rel,
           "max_nodal_error_vs_u": err, "spmv_fp32_ms": spmv_ms, "spmv_timing": spmv_timing,
           "spmv_fp32_GBps": spmv_bytes / (spmv_ms * 1e-3) / 1e9,
           "spmv_frac_of_hbm": spmv_bytes / (spmv_ms * 1e-3) / 1e9 / float(measured_peaks()[0].get("hbm_gbs", 6800.0)),
           "spmv_bytes": int(spmv_bytes)}
    for z in (D, A, B):
        nl.nl_csr_free(ctx, z)
    return out


def reference_arm(args, rank, world):
    from paper_2005_10775_gb300 import inputs as I
    if rank != 0:
        return
    per_step = max(2.0, min(20.0, 60.0 / max(args.steps, 1)))
    if args.workload == "batch64":
        probs = I.batch_problems()
        tt = 0.0
        for _ in range(args.steps):
            base, t = cpu_baseline_batch(probs, per_step)
            tt += t
        ms = tt / args.steps
        conf = {"workload": "batch64", "problems": len(probs), "K_total": sum(q.mesh.nt for q in probs)}
    else:
        p = I.problem(args.workload)
        cpu_baseline(p, per_step / 4, steps=1) if args.warmup else None
        base, ms = cpu_baseline(p, per_step, steps=args.steps)
        conf = {"workload": args.workload, "K": p.mesh.nt, "ball": p.ball, "outer": p.outer, "inner": p.inner,
                "delta": p.delta}
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": conf,
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def device_mesh(nl, m, dev, keep):
    import torch
    dmesh = type("DevMesh", (), dict(vx=torch.tensor(m.vx, device=dev), vy=torch.tensor(m.vy, device=dev),
                                     tri=torch.tensor(m.tri, device=dev)))
    return nl.make_mesh(dmesh, keep)


def time_assembly(nl, ctx, mesh, cfg, steps, warmup, stream, flush, dev, dist):
    """`steps` nl_assemble calls from a mesh in HBM to the finished CSR, each bracketed by CUDA
    events on the library's stream (L2 flushed before each); the max over ranks of the total."""
    import numpy as np
    import torch
    for _ in range(warmup):
        out = nl.nl_assemble(ctx, mesh, cfg)
        nl.nl_csr_free(ctx, out)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tot = 0.0
    phase = np.zeros(4)
    stats = None
    l0 = nl.nl_launch_count(ctx)
    wall0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = nl.nl_assemble(ctx, mesh, cfg)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        phase += nl.nl_last_timings(ctx)
        stats = (out.n_pairs, out.n_qp_pairs, out.n_inter, out.nnz, nl.nl_last_fp64_items(ctx))
        nl.nl_csr_free(ctx, out)
    launches = nl.nl_launch_count(ctx) - l0
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    return max_over_ranks(tot, dev, dist), phase / steps, stats, launches, wall


def fp32c_vs_fp64_error(nl, ctx, mesh, cfg32, cfg64):
    """max |D_fp32c - D_fp64| / max |D_fp64| over all entries (the two share their pattern)."""
    import numpy as np
    res = []
    for cfg in (cfg32, cfg64):
        out = nl.nl_assemble(ctx, mesh, cfg)
        try:
            res.append(nl.nl_csr_download(ctx, out))
        finally:
            nl.nl_csr_free(ctx, out)
    (rp32, ci32, v32), (rp64, ci64, v64) = res
    if not (np.array_equal(rp32, rp64) and np.array_equal(ci32, ci64)):
        return None
    return float(np.abs(v32 - v64).max() / np.abs(v64).max())


def alu_peaks(nl, ctx):
    """Derived FP32 FMA peak (the roofline denominator: SMs x lanes x 2 x the maximum SM clock of
    MEASURED_PEAKS.json), and the FP32 / FP64 FMA throughput measured on this GPU by nl_fma_peak."""
    peaks, src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    derived = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    meas32 = nl.nl_fma_peak(ctx, "fp32c")
    meas64 = nl.nl_fma_peak(ctx, "fp64")
    return {"fp32_derived_tflops": derived, "fp32_measured_tflops": meas32, "fp64_measured_tflops": meas64,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS, "sm_max_mhz": sm_mhz, "clock_source": src,
            "how": "nl_fma_peak: 8 independent FMA chains a thread, 2048 threads a SM, best of 3 launches"}


def config_entry(args, nl, ctx, name, stream, dev, dist, flush, world, rank, peaks, steps=5, fp64_steps=2,
                 cpu_seconds=3.0, solve=False):
    """One more benchmark configuration, measured like the headline: FP32-compensated and FP64
    assembly times, qp-pairs/s, the FP32c/FP64 speedup and error, the numeric phase against the
    FP32 and FP64 FMA rooflines, and a short oracle sample on the host cores."""
    from paper_2005_10775_gb300 import inputs as I
    p = I.problem(name)
    keep = nl._Keep()
    mesh = device_mesh(nl, p.mesh, dev, keep)

    def cfg_for(prec):
        return nl.make_config(keep, p.delta, p.ball, p.outer, p.inner, p.kernel, p.kernel_c, p.ngon_off, p.cap_m,
                              prec)
    t32, ph32, st32, l32, _ = time_assembly(nl, ctx, mesh, cfg_for("fp32c"), steps, 2, stream, flush, dev, dist)
    t64, ph64, st64, _, _ = time_assembly(nl, ctx, mesh, cfg_for("fp64"), fp64_steps, 1, stream, flush, dev, dist)
    n_pairs, n_qp, n_inter, nnz, n_fp64 = st32
    ms32, ms64 = t32 / steps, t64 / fp64_steps
    flop = FLOP_PER_QP * n_qp + FLOP_PER_INTER * n_inter
    a32 = flop / (ph32[1] / 1e3) / 1e12
    a64 = flop / (ph64[1] / 1e3) / 1e12
    e = {"workload": name, "K": p.mesh.nt, "ball": f"{p.ball}{p.ngon_n or ''}", "delta": p.delta,
         "outer": p.outer, "inner": p.inner, "kernel": p.kernel,
         "n_pairs": n_pairs, "n_qp_pairs": n_qp, "n_inter": n_inter, "nnz": nnz, "fp64_items": n_fp64,
         "ms_per_matrix": {"fp32c": ms32, "fp64": ms64},
         "value": {"fp32c": n_qp * world / (ms32 / 1e3), "fp64": n_qp * world / (ms64 / 1e3), "unit": UNIT},
         "speedup_fp32c_vs_fp64": ms64 / ms32,
         "phase_ms_fp32c": {"prepare": ph32[0], "numeric": ph32[1], "symbolic": ph32[2], "scatter": ph32[3]},
         "numeric_ms_fp64": ph64[1],
         "roofline": {"bound": "alu", "unit": "TFLOP/s",
                      "achieved_fp32c": a32, "peak_fp32": peaks["fp32_derived_tflops"],
                      "frac_fp32c": a32 / peaks["fp32_derived_tflops"],
                      "achieved_fp64": a64, "peak_fp64_measured": peaks["fp64_measured_tflops"],
                      "frac_fp64_of_measured_fp64": a64 / peaks["fp64_measured_tflops"]},
         "fp32c_vs_fp64_max_rel_err": fp32c_vs_fp64_error(nl, ctx, mesh, cfg_for("fp32c"), cfg_for("fp64")),
         "gpu_launches_per_matrix": l32 / steps}
    if solve:
        e["solve"] = solve_phase(nl, ctx, p.mesh, p, "fp32c", stream, dev, keep)
    if rank == 0 and not args.no_cpu_baseline:
        e["cpu_baseline"], _ = cpu_baseline(p, cpu_seconds)
    return e


def table1_times(nl, ctx, stream, dev, dist, flush, h=0.0125, steps=3):
    """Assembly time of each ball of the paper's Table 1 on grid (a) with cell size h (K = 18432 at
    h = 0.0125), with the paper's rule protocol, FP32-compensated, relative to the slowest
    (exactcaps in the paper, whose times are relative to it too: context only)."""
    from paper_2005_10775_gb300 import inputs as I
    m = I.paper_grid(h)
    keep = nl._Keep()
    mesh = device_mesh(nl, m, dev, keep)
    d = 0.1
    ms, n64 = {}, {}
    for ball in ("exactcaps", "approxcaps", "nocaps", "barycenter", "overlap"):
        cfg = nl.make_config(keep, d, ball, "switch47", "gauss3", "const", I.const_kernel_c(d), None, 2, "fp32c",
                             cap_printed=1 if ball == "exactcaps" else 0)
        t, _, _, _, _ = time_assembly(nl, ctx, mesh, cfg, steps, 1, stream, flush, dev, dist)
        ms[ball] = t / steps
        n64[ball] = nl.nl_last_fp64_items(ctx)
    slow = max(ms.values())
    paper = {"exactcaps": 10.31, "approxcaps": 8.36, "nocaps": 7.76, "barycenter": 4.24, "overlap": 5.23}
    return {"h": h, "K": m.nt, "ms_per_matrix": ms, "fp64_items": n64,
            "relative_to_slowest_pct": {b: 100 * v / slow for b, v in ms.items()},
            "paper_pct_of_its_slowest_run": paper,
            "note": "paper Table 1 times at h = 0.0125 as a percentage of its slowest run (exactcaps, h = 0.00625); "
                    "hardware unstated"}


def main():
    args = parse()
    rank, local, world = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch

    from paper_2005_10775_gb300 import inputs as I
    from paper_2005_10775_gb300 import nlfem as nl

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    # a dedicated stream shared by the library and the timing events (the legacy default
    # stream has handle 0, which the C ABI reads as "create a private stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = nl.nl_create(local, stream.cuda_stream)
    if args.peaks_only:
        if rank == 0:
            print(json.dumps({"fma_peaks": alu_peaks(nl, ctx), "gpu": torch.cuda.get_device_name(dev)}), flush=True)
        nl.nl_destroy(ctx)
        return
    if args.workload == "batch64":
        line = batch_bench(args, nl, ctx, stream, dev, world, dist, rank)
        nl.nl_destroy(ctx)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    p = I.problem(args.workload)
    m = p.mesh
    keep = nl._Keep()
    mesh = device_mesh(nl, m, dev, keep)
    off = None if p.ngon_off is None else torch.tensor(p.ngon_off, device=dev)

    def cfg_for(prec):
        return nl.make_config(keep, p.delta, p.ball, p.outer, p.inner, p.kernel, p.kernel_c, off, p.cap_m, prec)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def run(prec, steps, warmup):
        return time_assembly(nl, ctx, mesh, cfg_for(prec), steps, warmup, stream, flush, dev, dist)

    clocks = ClockSampler(local)
    clocks.start()
    tot_ms, phase, stats, launches, wall = run(args.prec, args.steps, args.warmup)
    ck = clocks.stop()
    n_pairs, n_qp, n_inter, nnz, n_fp64 = stats
    ms_step = tot_ms / args.steps
    value = n_qp * world * args.steps / (tot_ms / 1e3)

    # FP64 path for the FP32-comp vs FP64 comparison, and the error of the timed FP32c matrix
    # against it (both assembled once more, compared entry by entry)
    fp64 = None
    err32 = None
    if args.fp64_steps > 0 and args.prec != "fp64":
        t64, ph64, _, _, _ = run("fp64", args.fp64_steps, 1)
        fp64 = {"ms_per_step": t64 / args.fp64_steps, "value": n_qp * world * args.fp64_steps / (t64 / 1e3),
                "numeric_ms": ph64[1]}
        err32 = fp32c_vs_fp64_error(nl, ctx, mesh, cfg_for("fp32c"), cfg_for("fp64"))

    # end to end through the C ABI with host buffers: H2D of the mesh inside, D2H of the CSR
    e2e = None
    if not args.no_e2e:
        hmesh = nl.make_mesh(m, keep)
        hoff = p.ngon_off
        hcfg = nl.make_config(keep, p.delta, p.ball, p.outer, p.inner, p.kernel, p.kernel_c, hoff, p.cap_m,
                              args.prec)
        rp = torch.empty(m.nv + 1, dtype=torch.int64).pin_memory()
        ci = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
        va = torch.empty(max(nnz, 1), dtype=torch.float64).pin_memory()
        out = nl.nl_assemble(ctx, hmesh, hcfg)
        nl.nl_csr_free(ctx, out)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            out = nl.nl_assemble(ctx, hmesh, hcfg)
            nl._check(ctx, nl.LIB.nl_csr_download(ctx, nl.ctypes.byref(out), rp.data_ptr(), ci.data_ptr(),
                                                  va.data_ptr()))
            nl.nl_csr_free(ctx, out)
        torch.cuda.synchronize()
        e2e_value = job_throughput(n_qp * args.steps, time.perf_counter() - t0, world, dev, dist)
        h2d = m.vx.nbytes + m.vy.nbytes + m.tri.nbytes + (0 if hoff is None else hoff.nbytes)
        d2h = 8 * (m.nv + 1) + 12 * nnz
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    solve = None
    if args.solve:
        solve = solve_phase(nl, ctx, m, p, args.prec, stream, dev, keep)

    peaks = alu_peaks(nl, ctx)
    peak = peaks["fp32_derived_tflops"]
    numeric_ms = phase[1]
    achieved = (FLOP_PER_QP * n_qp + FLOP_PER_INTER * n_inter) / (numeric_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32c" if args.prec == "fp32c" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "K": m.nt, "J": m.nv, "ball": f"{p.ball}{p.ngon_n or ''}",
                   "delta": p.delta, "outer": p.outer, "inner": p.inner, "kernel": p.kernel,
                   "parallelism": f"replica x{world}", "l2": "flushed (512 MB write) before every step",
                   "n_pairs": n_pairs, "n_qp_pairs": n_qp, "n_inter": n_inter, "nnz": nnz,
                   "fp64_items": n_fp64,
                   "phase_ms": {"prepare": phase[0], "numeric": phase[1], "symbolic": phase[2],
                                "scatter": phase[3]},
                   "wall_s_timed": wall},
        "fp64": fp64,
        "speedup_fp32c_vs_fp64": (fp64["ms_per_step"] / ms_step) if fp64 else None,
        "fp32c_vs_fp64_max_rel_err": err32,
        "roofline": {"bound": "alu", "kernel": "k_interior + k_boundary + k_deferred + k_defer_merge (+ k_near for the "
                               "singular kernel): pair geometry + quadrature",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"FP32 FMA: {SMS} SMs x {FP32_LANES} lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz "
                                    f"(clock from MEASURED_PEAKS.json, {peaks['clock_source']})",
                     "frac_of_measured_fp32": achieved / peaks["fp32_measured_tflops"],
                     "traffic": NCU_TRAFFIC[args.workload][0] if args.workload in NCU_TRAFFIC else None,
                     "traffic_source": NCU_TRAFFIC[args.workload][1] if args.workload in NCU_TRAFFIC else None},
        "fma_peaks": peaks,
        "clocks": ck,
        "solve": solve,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if fp64:
        a64 = (FLOP_PER_QP * n_qp + FLOP_PER_INTER * n_inter) / (fp64["numeric_ms"] / 1e3) / 1e12
        line["roofline"]["fp64_path"] = {"achieved": a64, "peak_fp64_measured": peaks["fp64_measured_tflops"],
                                         "frac": a64 / peaks["fp64_measured_tflops"]}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_baseline(p, args.cpu_seconds)
    if not args.no_configs and args.workload == "ngon32_96":
        # the other benchmark configurations, measured the same way (not the headline)
        cfgs = {}
        ck2 = ClockSampler(local)
        ck2.start()
        for name, solve_it in (("barycenter_32", False), ("singular_128", False), ("solve_220", True)):
            cfgs[name] = config_entry(args, nl, ctx, name, stream, dev, dist, flush, world, rank, peaks,
                                      solve=solve_it)
        cfgs["paper_table1_times"] = table1_times(nl, ctx, stream, dev, dist, flush)
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup, bargs.fp64_steps, bargs.no_e2e = 3, 1, 1, True
        bargs.no_cpu_baseline = args.no_cpu_baseline
        bl = batch_bench(bargs, nl, ctx, stream, dev, world, dist, rank, cpu_seconds=4.0)
        cfgs["batch64"] = {k: bl[k] for k in ("value", "ms_per_step", "config", "sequential",
                                              "speedup_batch_vs_sequential", "reassembly", "fp64",
                                              "speedup_fp32c_vs_fp64", "roofline", "gpu_launches")
                           if k in bl}
        if "cpu_baseline" in bl:
            cfgs["batch64"]["cpu_baseline"] = bl["cpu_baseline"]
        cfgs["clocks"] = ck2.stop()
        line["configs"] = cfgs
    nl.nl_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
