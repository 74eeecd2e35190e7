#!/usr/bin/env python
"""Throughput benchmark of the confined-TTSH solver on GB300: grid-point-steps per second.

One timed step = one segment of `--solver-steps` steps of Algorithm 1 on the workload's
domain (default: the 512 x 512 circular domain, R = 5.4, dx = 0.04, uniform noise 0.01 from
seed 2, 20000 solver steps).  The float32 path is the headline value; the float64 path is
measured alongside under "fp64".  Multi-GPU (torchrun): every rank advances its own
independent domain (seed + rank), no data-path collective; value = all ranks' grid-point-
steps / the slowest rank's time.

--impl reference times the FP64 CPU oracle (the method written from the paper in numpy) on
the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ttsh_inputs as ti  # noqa: E402
from paper_2304_03306_gb300 import sharding as shd  # noqa: E402

METRIC = "grid-point-steps/s FP32 vs FP64 on 1 GB300; surrogate speedup at ≤2% error"
UNIT = "grid-point-steps/s"
DEFAULT_SOLVER_STEPS = {"circle512": 20000, "circle64_fp64": 2000, "circle2048_turbulent": 2000,
                        "circle4096_turbulent": 400, "circle8192_paper_grid": 100}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="circle512", choices=sorted(ti.WORKLOADS))
    ap.add_argument("--solver-steps", type=int, default=None)
    ap.add_argument("--record-every", type=int, default=10,
                    help="time-series sample interval in solver steps (0: plain stepping)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-lyap", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 2048^2 and 8192^2 legs")
    ap.add_argument("--plan", default=None, metavar="ROW,COL[,MODE]",
                    help="float32 step-kernel variants and launch mode instead of the autotuner's choice")
    return ap.parse_args()


def workload_desc(name, w, S):
    return (f"{name}: one circular domain R={w['radius']} on a {w['n']}x{w['n']} periodic grid, "
            f"dx={w['dx']}, Table I constants, dt=0.01, uniform noise 0.01 inside the mask "
            f"(seed {w['seed']}), {S} solver steps per timed step")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_id)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("ttsh_fft.cuh", "ttsh_wait.cuh", "ttsh_kernels.cuh", "ttsh_ops_impl.cuh")


def csrc_hash():
    """Hash of the sources that define the step kernels (ncu counters go stale when it changes)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2304_03306_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def plan_variant(kernel, plan):
    if kernel == "row_pass":
        cl = plan.get("row_cluster", 1)
        return [plan["rows_per_block"], plan["row_points_per_thread"]] + ([cl] if cl > 1 else []) + \
            (["compact"] if plan.get("row_compact", 0) else [])
    return [plan["col_points_per_thread"]]


def profile_record(fname, key, kernel, n, precision, plan):
    """A per-launch counter from a committed ncu summary, if it was taken on the current
    kernel sources and on the tile variant the autotuner chose."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", fname)))["records"]
        for e in t[f"{kernel}:{n}:{precision}"]:
            if e.get("csrc_hash") == csrc_hash() and list(e["variant"]) == plan_variant(kernel, plan):
                return float(e[key])
    except Exception:
        pass
    return None


def ncu_traffic(kernel, n, precision, plan):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)."""
    return profile_record("traffic.json", "dram_bytes_per_launch", kernel, n, precision, plan)


def algorithmic_bytes(n, elt):
    """Bytes one launch of each pass must move (inputs read once, outputs written once):
    the row pass reads the three column-transformed fields (omega, v_x, v_y) on the H = n/4 + 1
    stored columns and the mask, and writes the three right-hand-side fields on the same
    columns; the column pass reads those, reads and writes the state column, and writes the
    three column-transformed fields."""
    H = n // 4 + 1
    NK = n // 2 + 1
    c = 2 * elt
    row = 3 * H * n * c + n * n * elt + 3 * H * n * c
    col = 3 * H * n * c + 2 * H * NK * c + 3 * H * n * c
    return {"row_pass": row, "col_pass": col}


def algorithmic_flops(n):
    """Nominal flops of one launch of each pass: an m-point complex transform counts
    5 m log2 m (the radix-2 convention); a real row transform of length n is an n/2-point
    complex transform plus a 12-flop (inverse) or 14-flop (forward, kept outputs only)
    twiddle pass; 14 flops per point of real-space terms; 30 flops per stored mode of
    spectral update and multipliers.  Three inverse and three forward transforms per row and
    per column."""
    L, H, NK = n // 2, n // 4 + 1, n // 2 + 1
    fft = lambda m: 5.0 * m * np.log2(m)
    row = n * (3 * (fft(L) + 12 * L) + 3 * fft(L) + 3 * 14 * H + 14 * n)
    col = H * (6 * fft(n) + 30 * NK)
    return {"row_pass": row, "col_pass": col}


# one DFMA per clock per SM partition pair: 2 DFMA/clk/SM x 2 flops x 152 SMs x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# 128 FP32 lanes/SM x 2 flops x 152 SMs x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def ncu_executed(kernel, n, precision, plan):
    """Executed floating-point operations per launch (ncu FMA x 2 + ADD + MUL instruction counts)."""
    return profile_record("flops.json", "executed_flops_per_launch", kernel, n, precision, plan)


# ----------------------------------------------------------------------- CPU oracle leg

def _oracle_replica(wname, record_every, warm_steps, timed_steps, budget_s, barrier, out):
    """One single-threaded oracle process stepping its own copy of the workload: set-up and
    warm-up, then (after every replica is ready) `timed_steps` steps, or as many as fit in
    `budget_s` seconds when timed_steps is 0.  Puts (steps, seconds) on `out`."""
    from oracle import ttsh_oracle as O
    w = ti.WORKLOADS[wname]
    n, dx = w["n"], w["dx"]
    mask = ti.circle_mask(n, dx, w["radius"])
    vx, vy = ti.noise_velocity(mask, w["seed"], 0.01)
    p = O.Params(n=n, dx=dx)
    K = O.process_mask(mask)
    s = O.project_velocity(vx, vy, p)
    count = 0

    def one(s, count):
        if record_every > 0 and count % record_every == 0:
            O.diagnostics(s, p)
        return O.step(s, K, p), count + 1

    for _ in range(max(1, warm_steps)):
        s, count = one(s, count)
    barrier.wait()
    t0 = time.perf_counter()
    steps = 0
    while (timed_steps > 0 and steps < timed_steps) or \
            (timed_steps == 0 and (steps < 3 or time.perf_counter() - t0 < budget_s)):
        s, count = one(s, count)
        steps += 1
    out.put((steps, time.perf_counter() - t0))


def oracle_replicas(wname, record_every, procs=None, warm_steps=1, timed_steps=0, budget_s=10.0):
    """The FP64 oracle as it stands on every host core: `procs` (default: all cores)
    independent single-threaded processes, each stepping its own copy of the workload, started
    with the spawn method (no fork after CUDA).  Returns (aggregate grid-point-steps/s, procs,
    steps per process, wall seconds of the slowest)."""
    import multiprocessing as mp
    P = procs or os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(P), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(wname, record_every, warm_steps, timed_steps, budget_s,
                                                       barrier, out)) for _ in range(P)]
    for q in ps:
        q.start()
    res = [out.get() for _ in range(P)]
    for q in ps:
        q.join()
    n = ti.WORKLOADS[wname]["n"]
    rate = sum(n * n * st / dt for st, dt in res)
    return rate, P, [st for st, _ in res], max(dt for _, dt in res)


# ------------------------------------------------------------------------ GPU leg

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2304_03306_gb300 import build, ttsh

    build.build()
    ttsh.load_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)

    def barrier():
        shd.barrier(dev)

    w = ti.WORKLOADS[args.workload]
    n, dx = w["n"], w["dx"]
    S = args.solver_steps or DEFAULT_SOLVER_STEPS.get(args.workload, 1000)
    K, W = args.steps, args.warmup
    mask = ti.circle_mask(n, dx, w["radius"])
    vx0, vy0 = ti.noise_velocity(mask, w["seed"] + rank, 0.01)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    RE = args.record_every
    cap = -(-S // RE) if RE > 0 else 0
    series = torch.zeros(max(cap, 1) * 5, dtype=torch.float64, device=dev)

    def advance(dom, steps_per, record=True):
        """One timed step's work: steps_per solver steps, recording energy, enstrophy and the
        order parameter every RE steps on the device (the workload's time series)."""
        if record and RE > 0:
            dom.step_record(steps_per, RE, series.data_ptr(), cap)
        else:
            dom.step(steps_per)

    def timed_segments(dom, nseg, steps_per, record=True):
        evs = []
        for i in range(nseg):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            advance(dom, steps_per, record)
            e1.record(stream)
            evs.append((e0, e1))
        stream.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3

    def max_over_ranks(x):
        return shd.max_over_ranks(x, device=dev)

    # ---- float32 (headline) ----
    dom = ttsh.Domain(mask, n, dx, precision=32, stream=stream.cuda_stream)
    dom.set_velocity(vx0, vy0)
    if args.plan:
        pv = [int(x) for x in args.plan.split(",")]
        dom.set_plan(pv[0], pv[1], pv[2] if len(pv) > 2 else 0)
        plan32 = dom.plan()
    else:
        plan32 = dom.autotune(iters=max(20, min(400, int(4e7 // (n * n)))))   # untimed
    for _ in range(W):
        advance(dom, S)
    dom.synchronize()
    torch.cuda.synchronize()
    barrier()
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    clocks = ClockSampler(vis[local_rank].strip() if local_rank < len(vis) else local_rank)
    clocks.start()
    t32 = timed_segments(dom, K, S)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t32 = max_over_ranks(t32)
    value = world * n * n * S * K / t32
    series_last = series[: cap * 5].view(-1, 5)[-1].tolist() if cap > 0 else None
    # the same steps without the time series, for context (untimed by the headline)
    t_plain = max_over_ranks(timed_segments(dom, K, S, record=False))

    # kernel-level timing for the roofline (same domain, same stream; state restored)
    iters = max(50, min(2000, int(2e7 // (n * n))))
    row_ms, col_ms = dom.time_kernels(iters)
    diag = dom.diagnostics()

    # measured FMA throughput of this GPU: the denominators of the ALU rooflines
    fma_peak = {"fp32_tflops": ttsh.ttsh_fma_peak(32, 1 << 17), "fp64_tflops": ttsh.ttsh_fma_peak(64, 1 << 12),
                "how": "ttsh_fma_peak: 8 blocks of 256 threads per SM, 8 independent FMA chains per thread, "
                       "CUDA events"}

    # ---- float64 alongside ----
    fp64 = None
    if not args.no_fp64:
        d64 = ttsh.Domain(mask, n, dx, precision=64, stream=stream.cuda_stream)
        d64.set_velocity(vx0, vy0)
        plan64 = d64.autotune(iters=max(10, min(100, int(1e7 // (n * n)))))
        S64 = max(1, S // 4)
        advance(d64, S64)
        d64.synchronize()
        barrier()
        t64 = max_over_ranks(timed_segments(d64, K, S64))
        r64, c64 = d64.time_kernels(max(20, iters // 4))
        d64.close()
        v64 = world * n * n * S64 * K / t64
        fl = algorithmic_flops(n)
        k64 = "row_pass" if r64 >= c64 else "col_pass"
        ms64 = max(r64, c64)
        ach64 = fl[k64] / (ms64 * 1e-3) / 1e12
        ex64 = ncu_executed(k64, n, 64, plan64)
        fp64 = {"value": v64, "unit": UNIT, "solver_steps_per_step": S64,
                "ms_per_solver_step": 1e3 * t64 / (S64 * K), "row_pass_ms": r64, "col_pass_ms": c64,
                "fp32_over_fp64": value / v64, "plan": plan64,
                "roofline": {"bound": "alu", "achieved": ach64, "peak": fma_peak["fp64_tflops"], "unit": "TFLOP/s",
                             "frac": ach64 / fma_peak["fp64_tflops"], "traffic": ncu_traffic(k64, n, 64, plan64),
                             "kernel": k64, "kernel_ms": ms64, "algorithmic_flops": fl[k64],
                             "executed_flops": ex64,
                             "executed_tflops": None if ex64 is None else ex64 / (ms64 * 1e-3) / 1e12,
                             "peak_source": "measured (ttsh_fma_peak, FP64 FMA chains on every SM)",
                             "nominal_peak": FP64_PEAK_TFLOPS}}

    # ---- batched sweep: 48 domains (128^2..512^2 circles and dumbbells) in lock step ----
    batched = None
    if not args.no_batch:
        sweep = ti.sweep_domains()
        # the 48 domains are split over the ranks (cost-balanced, no collective); each rank
        # steps its share as one batch
        mine = shd.shard([d["n"] ** 2 for d in sweep], rank, world)
        objs = []
        for dspec in (sweep[i] for i in mine):
            o = ttsh.Domain(dspec["mask"], dspec["n"], dspec["dx"], precision=32, stream=stream.cuda_stream)
            bvx, bvy = ti.noise_velocity(dspec["mask"], dspec["seed"], 0.01)
            o.set_velocity(bvx, bvy)
            objs.append(o)
        bt = ttsh.Batch(objs, stream=stream.cuda_stream)
        Sb = max(32, S // 20)
        persistent = bt.persistent
        grouped_ms = None
        if persistent:   # the grouped launches (one per pass per group of equal domains), for comparison
            bt.set_persistent(False)
            bt.step(Sb)
            bt.synchronize()
            grouped_ms = 1e3 * max_over_ranks(timed_segments(bt, K, Sb, record=False)) / (Sb * K)
            bt.set_persistent(True)
        bt.step(Sb)
        bt.synchronize()
        barrier()
        tb = max_over_ranks(timed_segments(bt, K, Sb, record=False))
        pts = sum(dspec["n"] ** 2 for dspec in sweep)
        batched = {"value": pts * Sb * K / tb, "unit": UNIT, "domains": len(sweep),
                   "grouped_value": pts / (grouped_ms * 1e-3) if grouped_ms else None,
                   "grid_points": pts, "solver_steps_per_step": Sb, "launch_groups": bt.groups,
                   "persistent": persistent,
                   "launches_per_call": 1 if persistent else 2 * bt.groups * Sb,
                   "grouped_ms_per_solver_step": grouped_ms,
                   "scaling": "strong (the 48 domains are split across the ranks)",
                   "ms_per_solver_step": 1e3 * tb / (Sb * K),
                   "workload": "24 circles (R 5.0-8.0, forward and backward members) + 24 dumbbells "
                               "(R in {2.8, pi, 3.5} x D/R 1.0-1.9) on 128^2-512^2 grids, noise 0.01"}
        bt.close()
        for o in objs:
            o.close()

    # ---- the HBM-bound grids: 2048^2 turbulent circle (FP32 and FP64) and the paper's 8192^2 ----
    def large_leg(wname, prec, S_l):
        wl = ti.WORKLOADS[wname]
        nl, dxl = wl["n"], wl["dx"]
        ml = ti.circle_mask(nl, dxl, wl["radius"])
        dl = ttsh.Domain(ml, nl, dxl, precision=prec, stream=stream.cuda_stream)
        dl.init_noise(wl["seed"] + rank, 0.01)
        planl = dl.autotune(iters=max(20, min(400, int(4e7 // (nl * nl)))))
        for _ in range(W):
            dl.step(S_l)
        dl.synchronize()
        barrier()
        tl = max_over_ranks(timed_segments(dl, K, S_l, record=False))
        rms, cms = dl.time_kernels(max(20, min(2000, int(2e7 // (nl * nl)))))
        dl.close()
        elt_l = 4 if prec == 32 else 8
        abl = algorithmic_bytes(nl, elt_l)
        kl = "row_pass" if rms >= cms else "col_pass"
        msl = max(rms, cms)
        pk, pk_src = peaks()
        ach = abl[kl] / (msl * 1e-3) / 1e9
        vl = world * nl * nl * S_l * K / tl
        step_bytes = abl["row_pass"] + abl["col_pass"]
        out = {"workload": workload_desc(wname, wl, S_l), "precision": prec, "value": vl, "unit": UNIT,
               "ms_per_solver_step": 1e3 * tl / (S_l * K), "plan": planl,
               "roofline": {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                            "traffic": ncu_traffic(kl, nl, prec, planl), "kernel": kl, "kernel_ms": msl,
                            "algorithmic_bytes": abl[kl], "peak_source": f"{pk_src} (copy bandwidth)",
                            "passes_ms": {"row_pass": rms, "col_pass": cms}},
               "step_roofline": {"bytes_per_point": step_bytes / (nl * nl),
                                 "achieved_gbs": step_bytes * vl / (world * nl * nl) / 1e9,
                                 "frac": step_bytes * vl / (world * nl * nl) / 1e9 / pk,
                                 "note": "whole step (both passes and the launch gaps) at the algorithmic bytes"}}
        if prec == 64:
            fl = algorithmic_flops(nl)
            out["alu_roofline"] = {"bound": "alu", "achieved": fl[kl] / (msl * 1e-3) / 1e12,
                                   "peak": fma_peak["fp64_tflops"], "unit": "TFLOP/s",
                                   "frac": fl[kl] / (msl * 1e-3) / 1e12 / fma_peak["fp64_tflops"],
                                   "peak_source": "measured (ttsh_fma_peak)"}
        return out

    large = None
    if not args.no_large:
        large = {"circle2048_fp32": large_leg("circle2048_turbulent", 32, 2000),
                 "circle8192_fp32": large_leg("circle8192_paper_grid", 32, 100)}
        if not args.no_fp64:
            large["circle2048_fp64"] = large_leg("circle2048_turbulent", 64, 100)

    # ---- Lyapunov analysis: the workload's domain with 8 perturbed copies ----
    lyap = None
    if not args.no_lyap and rank == 0:
        kl, il = 8, 10
        dl = ttsh.Domain(mask, n, dx, precision=32, stream=stream.cuda_stream)
        dl.set_velocity(vx0, vy0)
        dl.set_plan(plan32["row_variant"], plan32["col_variant"], plan32["launch_mode"])
        dl.step(200)
        w0, m0 = dl.spectral_state()
        u0 = np.concatenate([np.stack([w0.real, w0.imag], axis=-1).reshape(-1), m0])
        L = ttsh.Lyapunov(dl, ti.perturbation_directions(n, kl, 11), 1e-3 * np.linalg.norm(u0))
        L.step(10 * il, il)   # warm-up (graphs, attributes)
        dl.synchronize()
        Sl = max(il, (S // 40) // il * il)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.step(Sl, il)
        e1.record(stream)
        stream.synchronize()
        tl = e0.elapsed_time(e1) / 1e3
        ex, last = L.result()
        lyap = {"perturbations": kl, "interval": il, "solver_steps": Sl,
                "ms_per_solver_step": 1e3 * tl / Sl,
                "grid_point_steps_per_s": (kl + 1) * n * n * Sl / tl,
                "exponents": [float(x) for x in ex],
                "note": "FP32 domain, eps = 1e-3 of the state norm; exponents over a short run (not converged)"}
        L.close()
        dl.close()

    # ---- learned corrector (the corrector configuration as written): trained on 200
    # trajectories of the batched 512^2 solver, evaluated on the held-out radii for 1e4 coarse
    # steps against the plain FP32 512^2 solver ----
    surrogate = None
    if not args.no_surrogate and rank == 0:
        from paper_2304_03306_gb300 import corrector as Cr
        t0 = time.perf_counter()
        ntraj, nsamp, iters_tr, coarse_steps = 200, 16, 1000, 10000
        net = ttsh.FNO(n=256, width=32, modes=16, layers=4, max_batch=8, seed=0)
        X, Y = Cr.generate(net, ntraj=ntraj, samples=nsamp, spacing=40, transient=3000, amplitude=0.3, seed=0)
        Cr.normalise(net, X, Y)
        torch.cuda.synchronize()
        t_gen = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = Cr.train(net, X, Y, iters=iters_tr, batch=8, lr=1e-3, log_every=iters_tr - 1)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del X, Y
        evs = {}
        for radius in Cr.HELD_OUT:
            ev = Cr.evaluate(net, radius, coarse_steps=coarse_steps, sample_every=50, correct_every=1)
            evs[str(radius)] = {k: ev[k] for k in ("speedup_fno", "speedup_plain", "spectrum_error_fno",
                                                   "spectrum_error_plain", "psi_fine", "psi_fno", "psi_plain",
                                                   "t_fine", "t_plain", "t_fno", "nonfinite")}
        net.close()
        mean = lambda k: float(np.mean([e[k] for e in evs.values()]))
        surrogate = {
            "metric": "wall-clock speedup of the coarse (256^2, 4 dt) solver + FNO corrector over the fine "
                      "FP32 512^2 solver for the same physical time, and time-averaged E(k) error (s <= 64)",
            "speedup": mean("speedup_fno"), "spectrum_error": mean("spectrum_error_fno"),
            "spectrum_error_without_corrector": mean("spectrum_error_plain"),
            "speedup_without_corrector": mean("speedup_plain"),
            "held_out": evs, "coarse_steps": coarse_steps,
            "train": {"trajectories": ntraj, "samples": ntraj * nsamp, "iters": iters_tr, "batch": 8,
                      "loss_first_last": [losses[0][1], losses[-1][1]], "t_generate_s": t_gen, "t_train_s": t_train},
            "network": "FNO 4 layers, width 32, 16 modes, BF16 weights, FP32 accumulate"}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        hx, hy = pin((n, n)), pin((n, n))
        hx[:], hy[:] = vx0, vy0
        ox, oy, ow = pin((n, n)), pin((n, n)), pin((n, n))
        # the headline's own domain: the same plan, and the same placement of its workspace
        # in device memory (the step time depends on it at the 1 % level)
        de = dom
        lib = ttsh.load_library()
        P = lambda a: a.ctypes.data_as(ttsh._D)

        hser = torch.empty(max(cap, 1) * 5, dtype=torch.float64, pin_memory=True)

        def e2e_step():
            ttsh._check(lib.ttsh_set_velocity(de.h, P(hx), P(hy)))
            if RE > 0:
                ttsh._check(lib.ttsh_step_record(de.h, S, RE, series.data_ptr(), cap, None))
                with torch.cuda.stream(stream):
                    hser.copy_(series, non_blocking=True)
            else:
                ttsh._check(lib.ttsh_step(de.h, S))
            ttsh._check(lib.ttsh_get_fields(de.h, P(ox), P(oy), P(ow)))

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        te = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * n * n * S * K / te, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * n * 8,
               "d2h_bytes_per_step": 3 * n * n * 8 + (cap * 5 * 8 if RE > 0 else 0),
               "path": "ttsh_set_velocity (pinned host) + ttsh_step_record + time series and "
                       "ttsh_get_fields to pinned host, wall clock, on the headline's domain"}
    dom.close()

    if dist:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return None

    # ---- roofline of the dominant kernel ----
    elt = 4
    ab = algorithmic_bytes(n, elt)
    dom_k = "row_pass" if row_ms >= col_ms else "col_pass"
    dom_ms = max(row_ms, col_ms)
    peak, peak_src = peaks()
    achieved = ab[dom_k] / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom_k, n, 32, plan32),
                "kernel": dom_k, "kernel_ms": dom_ms, "algorithmic_bytes": ab[dom_k],
                "peak_source": f"{peak_src} (copy bandwidth)",
                "passes_ms": {"row_pass": row_ms, "col_pass": col_ms},
                "share": {"row_pass": row_ms / (row_ms + col_ms), "col_pass": col_ms / (row_ms + col_ms)},
                "step_bytes_per_point": (ab["row_pass"] + ab["col_pass"]) / (n * n)}
    fl32 = algorithmic_flops(n)
    roofline["alu_context"] = {"achieved_tflops": fl32[dom_k] / (dom_ms * 1e-3) / 1e12,
                               "peak_tflops": fma_peak["fp32_tflops"],
                               "frac": fl32[dom_k] / (dom_ms * 1e-3) / 1e12 / fma_peak["fp32_tflops"],
                               "algorithmic_flops": fl32[dom_k],
                               "executed_flops": ncu_executed(dom_k, n, 32, plan32),
                               "peak_source": "measured (ttsh_fma_peak, FP32 FMA chains on every SM)",
                               "nominal_peak_tflops": FP32_PEAK_TFLOPS}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, P, steps, dt = oracle_replicas(args.workload, RE)
        cpu = {"value": v, "unit": UNIT, "cores": P, "kind": "oracle",
               "sample": f"{P} independent single-threaded oracle processes (numpy FP64, one per host core, "
                         f"nproc = {os.cpu_count()}), each stepping its own copy of the {n}x{n} workload for "
                         f"~{dt:.0f} s ({min(steps)}-{max(steps)} steps each), oracle diagnostics every {RE} "
                         f"steps; value = the sum of the processes' grid-point-steps/s"}

    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * t32 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, w, S), "n": n, "dx": dx,
                   "radius": w["radius"], "solver_steps_per_step": S, "plan": plan32,
                   "l2": "flushed (256 MiB write) before every timed step; the state stays L2-resident within a step",
                   "time_series": (f"energy, enstrophy, psi recorded on the device every {RE} solver steps "
                                   f"({cap} samples per timed step, ttsh_step_record)") if RE > 0 else "none",
                   "parallelism": "replicas" if world == 1 else f"independent domains x{world}"},
        "e2e": e2e, "gpu_launches": K * (2 * S + (1 if RE > 0 else 0)), "clocks": clk, "roofline": roofline,
        "value_without_time_series": world * n * n * S * K / t_plain,
        "time_series_last_sample": series_last,
        "cpu_baseline": cpu, "fp64": fp64, "batched": batched, "large_grids": large, "fma_peak": fma_peak,
        "surrogate": surrogate, "lyapunov": lyap,
        "diagnostics_after": {"energy": diag["energy"], "psi": diag["psi"], "nonfinite": diag["nonfinite"]},
        "ms_per_solver_step": 1e3 * t32 / (K * S),
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = ti.WORKLOADS[args.workload]
    n = w["n"]
    S_ref = max(1, int(1.0e6 // (n * n)))   # oracle steps per timed step and process (~0.3 s at 512^2)
    RE = args.record_every
    # every process warms up for W steps' worth, then all run the K timed steps' worth at once
    v, P, steps, wall = oracle_replicas(args.workload, RE, warm_steps=S_ref * max(1, args.warmup),
                                        timed_steps=S_ref * args.steps)
    v = P * n * n * S_ref * args.steps / wall   # whole job: all processes' points over the slowest's time
    sample = (f"{P} independent single-threaded oracle processes (one per host core, nproc = {os.cpu_count()}), "
              f"each {S_ref * args.steps} timed oracle steps of its own copy of the {n}x{n} workload")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, w, S_ref), "n": n,
                       "solver_steps_per_step": S_ref, "parallelism": f"{P} CPU processes (replicas)",
                       "time_series": f"oracle diagnostics every {RE} solver steps" if RE > 0 else "none"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": P, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
