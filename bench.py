"""Benchmark of the angle-dependent CT operator path on GB300.

One step = one pass of the whole operator path over one batch of the
256 x 256 / 180-view / 363-bin workload (random-ellipse phantom, 1-degree
angle errors):
    Y  = H(theta) X      for a Krylov block of K = 8 images
    X' = H(theta)^T Y'   for a block of K = 8 sinograms
    dy = J_theta dtheta  for one image
    g  = J_theta^T r     for one image and one residual
The metric is sinogram samples produced or consumed per second (GSamples/s),
counted as V*B*(K + K + 1 + 1) per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank runs its own
replica of the workload (the operators shard by views without any exchange;
this build runs replicas only) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "A/Aᵀ/Jθ GSamples/s + NL-RMM-GKS iter time vs FP64 GPU form at equal error"
WORKLOAD = "C2"
KBLOCK = 8
# DRAM bytes per launch of the dominant kernels, from ncu captures of
# `python bench.py --steps 3 --warmup 3 --no-cpu-baseline --no-solver --tuning <shape>`
# (4,4,1,8,2,2,1,0,0,0, 4,4,1,8,4,2,2,0,0,16 and 4,4,1,8,4,4,1,0,0,8), keyed by the launch shape
# that selects the kernel; a shape that was not profiled reports null.
PROFILED_DRAM_BYTES = {
    ("forward_K8", (4, 4, 1, 0)): 8.56e6,   # k_ray<float, 0, 0, 4, 4>: fwd kb, split, views/CTA, staging
    ("adjoint_K8", (8, 2, 0)): 3.95e6,      # k_adjoint<float, 8, 2>: adj kb, view groups, staging
    ("adjoint_K8", (8, 4, 16)): 4.04e6,     # k_adj_band<8, 16>, 4 CTAs per tile
    ("adjoint_K8", (8, 4, 8)): 4.04e6,      # k_adj_band<8, 8>, 4 CTAs per tile
}


def launches_per_step(t):
    """Kernels of one bench step at launch shapes t (the 10 ct_get_tuning values):
    forward, J and J^T lay out their image and the transpose its sinograms
    (1 each; the same launch brings the view table up to date); the forward
    ray kernel(s) over the 8-image block, the transpose, the JVP, the VJP and
    its per-view reduction; staged shapes with several CTAs per ray / tile
    add a combining kernel."""
    fkb, fsplit, _, akb, asplit, _, _, fstage, _, astage = t
    fwd = 0
    k = 0
    for width in (8, 4, 2, 1):
        if width <= fkb and (KBLOCK - k) // width > 0:
            fwd += 1
            k += (KBLOCK - k) // width * width
    fwd += 1 if (fstage > 0 and fsplit > 1) else 0
    adj = 0
    k = 0
    for width in (8, 4, 2, 1):
        if width <= akb and (KBLOCK - k) // width > 0:
            adj += 1
            k += (KBLOCK - k) // width * width
    adj += 1 if (astage > 0 and asplit > 1) else 0
    return 3 + 1 + fwd + adj + 1 + 1 + 1


L2_FLUSH_BYTES = 512 * 1024 * 1024
LSU_BYTES_PER_CLK_SM = 128          # L1/shared data path per SM per clock
NUM_SMS = 152
SM_MAX_MHZ_NOMINAL = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solver", action="store_true", help="skip the NL-RMM-GKS comparison")
    ap.add_argument("--solver-iters", type=int, default=30)
    ap.add_argument("--stream-passes", type=int, default=2,
                    help="passes of the streaming solve on the 2048^2 / 1440-view workload (0: skip)")
    ap.add_argument("--solver-only", action="store_true",
                    help="run only the FP32 NL-RMM-GKS solve of the workload (--solver-iters outer iterations) "
                         "and print its timing: the command the solver's profiles are taken with")
    ap.add_argument("--varpro", action="store_true", help="with --solver-only: the VarPro parameter update")
    ap.add_argument("--solver-workload", default=WORKLOAD, choices=["C1", "C2", "C3", "C4"],
                    help="with --solver-only: the workload (C4: the 16-frame dynamic problem, with ANISO-TV)")
    ap.add_argument("--stream-only", action="store_true",
                    help="run only the streaming solve on the 2048^2 / 1440-view workload (--stream-passes passes) "
                         "and print its timing: the command the streaming profiles are taken with")
    ap.add_argument("--fan-only", action="store_true",
                    help="run only the fan-beam operator step (--steps replays) and print its timing")
    ap.add_argument("--stream-scale", type=float, default=1.0,
                    help="with --stream-only: shrink the streaming workload (image side, bins, views)")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shapes 'fkb,fsplit,fvw,akb,asplit,jsplit,jvw,fstage,jstage,astage' "
                         "(the ct_set_tuning values) instead of autotuning")
    return ap.parse_args()


def max_over_ranks(ms, world, device):
    """The job's time for a timed region: the slowest replica's (all_reduce MAX)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ms, world):
    """Whole-job throughput in G units/s: the units of every replica over the job's time."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def interp_steps_per_image(w):
    """Algorithmic work: number of (ray, sample) pairs with -1 < q < N (exact, FP64)."""
    N, B = w.N, w.B
    th = w.theta_true
    c, s = np.cos(th), np.sin(th)
    h = 0.5 * (N - 1)
    sb = np.arange(B)[None, :] - 0.5 * (B - 1)
    rows = np.abs(c) >= np.abs(s)
    r = np.arange(N)[:, None, None]
    total = 0
    for sel, cc, ss in ((rows, c, s), (~rows, c, s)):
        if not sel.any():
            continue
        cv, sv = cc[sel][None, :, None], ss[sel][None, :, None]
        if sel is rows:
            q = (sb[None] - (h - r) * sv) / cv + h
        else:
            q = h - (sb[None] - (r - h) * cv) / sv
        total += int(np.count_nonzero((q > -1) & (q < N)))
    return total


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clk_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_reference(args):
    """The FP64 CPU oracle as it stands, on the host cores, bounded sample of the same step."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    from paper_2605_06336_gb300 import synth
    w = synth.make_workload(WORKLOAD)
    g = oracle.Geometry(w.N, w.B, w.V)
    rng = np.random.default_rng(1)
    X = np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(KBLOCK - 1, w.N * w.N))])
    Ys = oracle.forward(g, w.theta_true, X[:1])
    dth = rng.standard_normal(w.V)
    # a bounded sample: the step restricted to one image / one sinogram per operator
    def step():
        oracle.forward(g, w.theta_true, X[0])
        oracle.adjoint(g, w.theta_true, Ys[0])
        oracle.jac(g, w.theta_true, X[0], dth)
        oracle.jacT(g, w.theta_true, X[0], Ys[0])
    for _ in range(min(args.warmup, 1)):
        step()
    t0 = time.perf_counter()
    n = 0
    while n < args.steps and (time.perf_counter() - t0) < args.cpu_seconds:
        step()
        n += 1
    dt = time.perf_counter() - t0
    samples = w.V * w.B * 4 * n
    val = samples / dt / 1e9
    line = {"metric": METRIC, "value": val, "unit": "GSamples/s", "n_gpus": args.gpus, "steps": n,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(n, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "C2: 256x256 random-ellipse phantom, 180 views, 363 bins",
                       "sample": "one image per operator (H, H^T, J, J^T) per step", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "GSamples/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} steps of H, H^T, J, J^T on one 256^2 image, 180x363 sinogram"},
            "e2e": {"value": val, "unit": "GSamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def solver_comparison(w, dev, outer_iters, **extra):
    """NL-RMM-GKS on the workload: FP32 operators + FP64 small algebra + batched
    basis projection against the plain FP64 GPU form, same data, same options
    (`extra`: further solver options, e.g. temporal=1 for ANISO-TV)."""
    import torch
    from paper_2605_06336_gb300 import ct
    N, B, V = w.N, w.B, w.V
    u_true = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device=dev)
    th_true = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    op64 = ct.CTOperator(N, B, V, w.views_per_frame, max_batch=8, dtype=torch.float64)
    b_true = op64.forward(u_true, th_true)
    e = torch.tensor(w.noise_dir, dtype=torch.float64, device=dev)
    e *= w.noise_level * b_true.norm() / e.norm()
    b64 = b_true + e
    nn = float(e.norm())
    th0 = torch.tensor(w.theta_nominal, dtype=torch.float64, device=dev)
    out = {}
    for name, dt in (("fp64_plain", torch.float64), ("fp32_batched", torch.float32)):
        op = op64 if dt == torch.float64 else ct.CTOperator(N, B, V, w.views_per_frame, max_batch=8, dtype=dt)
        op.autotune()
        bb = b64.to(dt)
        xt = u_true.to(dt)
        op.solve(bb, th0, x_true=xt, noise_norm=nn, outer_iters=2, stop_on_convergence=0, **extra)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, th, st = op.solve(bb, th0, x_true=xt, noise_norm=nn, outer_iters=outer_iters, stop_on_convergence=0,
                             **extra)
        e1.record()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        ang = float((th - th_true).norm() / th_true.norm())
        it_ms = np.asarray(st["ms"], dtype=float)   # host wall time of each outer iteration
        spread = [float(np.percentile(it_ms, q)) for q in (10, 50, 90)] if it_ms.size else None
        out[name] = {"total_ms": total_ms, "ms_per_outer_iter": total_ms / outer_iters,
                     "outer_iter_ms_p10_p50_p90": spread,
                     "final_rre": st["rre"][-1], "rel_angle_err": ang,
                     "max_abs_angle_err_deg": float((th - th_true).abs().max()) * 180 / math.pi,
                     "enlarge_steps": sum(st["enlarge_steps"])}
    a, b_ = out["fp64_plain"], out["fp32_batched"]
    out["equal_error"] = abs(b_["final_rre"] - a["final_rre"]) <= 1e-3 * a["final_rre"]
    out["speedup_fp32_vs_fp64"] = a["total_ms"] / b_["total_ms"]
    out["outer_iters"] = outer_iters
    out["initial_max_abs_angle_err_deg"] = float(np.abs(w.theta_nominal - w.theta_true).max()) * 180 / math.pi
    if extra.get("temporal"):
        # the same FP32 solve with spatial differences only, for the effect of the temporal coupling
        op = ct.CTOperator(N, B, V, w.views_per_frame, max_batch=8, dtype=torch.float32)
        op.autotune()
        _, _, st = op.solve(b64.float(), th0, x_true=u_true.float(), noise_norm=nn, outer_iters=outer_iters,
                            stop_on_convergence=0)
        out["fp32_spatial_only_final_rre"] = st["rre"][-1]
    return out


def solver_only(w, dev, outer_iters, tuning=None, **extra):
    """The FP32 NL-RMM-GKS solve of solver_comparison alone (for profiling):
    autotune (or the given launch shapes), one 2-iteration warm-up solve, then
    the timed solve."""
    import torch
    from paper_2605_06336_gb300 import ct
    u_true = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device=dev)
    th_true = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    op64 = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=8, dtype=torch.float64)
    b_true = op64.forward(u_true, th_true)
    e = torch.tensor(w.noise_dir, dtype=torch.float64, device=dev)
    e *= w.noise_level * b_true.norm() / e.norm()
    b = (b_true + e).float()
    nn = float(e.norm())
    th0 = torch.tensor(w.theta_nominal, dtype=torch.float64, device=dev)
    op = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=8, dtype=torch.float32)
    if tuning:
        op.tuning = tuning
    else:
        op.autotune()
    op.solve(b, th0, x_true=u_true.float(), noise_norm=nn, outer_iters=2, stop_on_convergence=0, **extra)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, _, st = op.solve(b, th0, x_true=u_true.float(), noise_norm=nn, outer_iters=outer_iters, stop_on_convergence=0,
                        **extra)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"ms_per_outer_iter": ms / outer_iters, "enlarge_steps": sum(st["enlarge_steps"]),
            "final_rre": st["rre"][-1], "outer_iters": outer_iters, "tuning": dict(zip(ct.TUNING_FIELDS, op.tuning))}


def streaming_c5(dev, passes, scale=1.0):
    """Streaming NL-RMM-GKS (FP32 operators, FP64 small algebra) on the 2048^2 /
    1440-view workload in its 12 random chunks of 120 views: one handle per
    chunk, `passes` passes.  The data are H(theta_true) u_true from the FP64
    GPU forward plus 0.5 % noise.  `scale` < 1 shrinks the same recipe (for
    profiler captures of a smaller case)."""
    import torch
    from paper_2605_06336_gb300 import ct, synth
    w = synth.make_workload("C5", scale=scale)
    N, B = w.N, w.B
    chunks = w.extra["chunks"]
    u64 = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device=dev)
    bt = []
    for ch in chunks:
        op64 = ct.CTOperator(N, B, len(ch), max_batch=1, dtype=torch.float64)
        bt.append(op64.forward(u64, torch.tensor(w.theta_true[ch], device=dev)).cpu().numpy())
        op64.close()
    nd = w.noise_dir.reshape(w.V, B)
    scale = w.noise_level * math.sqrt(sum(float((x * x).sum()) for x in bt)) / np.linalg.norm(nd)
    ops, bs, th0, nns, tuning = [], [], [], [], None
    for j, ch in enumerate(chunks):
        op = ct.CTOperator(N, B, len(ch), max_batch=4, dtype=torch.float32)
        if tuning is None:
            tuning = op.autotune()  # one geometry for every chunk
        else:
            op.tuning = tuning
        e = scale * nd[ch].ravel()
        bs.append(torch.tensor(bt[j] + e, dtype=torch.float32, device=dev))
        th0.append(torch.tensor(w.theta_nominal[ch], device=dev))
        nns.append(float(np.linalg.norm(e)))
        ops.append(op)
    k_min, k_max = 20, 60
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, th, st = ct.stream_solve(ops, bs, th0, nns, x_true=u64.float(), k_min=k_min, k_max=k_max,
                                outer_iters=passes, stop_on_convergence=0)
    wall = time.perf_counter() - t0
    tht = np.concatenate([w.theta_true[ch] for ch in chunks])
    thn = np.concatenate([w.theta_nominal[ch] for ch in chunks])
    the = np.concatenate([t.cpu().numpy() for t in th])
    rel = lambda a: float(np.linalg.norm(a - tht) / np.linalg.norm(tht))
    out = {"workload": f"C5: {N}x{N}, {w.V} views in {len(chunks)} streamed chunks of {len(chunks[0])}, {B} bins, "
                       f"{w.noise_level * 100:.1f}% noise",
           "passes": st["passes"], "k_min": k_min, "k_max": k_max, "wall_s": wall, "ms_per_pass": st["ms"],
           "enlarge_steps_per_pass": st["enlarge_steps"], "rre_per_pass": st["rre"], "lambda_last_block": st["lambda"],
           "rel_angle_err_initial": rel(thn), "rel_angle_err_final": rel(the),
           "tuning": dict(zip(ct.TUNING_FIELDS, tuning)),
           "note": "basis capped at k_max = 60 (the FP64 small algebra holds at most 64 columns); "
                   "data from the FP64 GPU forward"}
    for op in ops:
        op.close()
    return out


def graph_op_timing(op, calls, reps, flush):
    """Device time of each operator call alone: every call captured in its own
    CUDA graph and replayed `reps` times (L2 flushed before each replay,
    outside the events).  Returns mean ms per call, one per entry of `calls`."""
    import torch
    out = []
    for call in calls:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            op.set_stream(side)
            call()
        torch.cuda.current_stream().wait_stream(side)
        with torch.cuda.graph(g):
            op.set_stream(torch.cuda.current_stream())
            call()
        op.set_stream(torch.cuda.current_stream())
        cur = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        g.replay()
        for a, b in evs:
            flush.zero_()
            a.record(cur)
            g.replay()
            b.record(cur)
        torch.cuda.synchronize()
        out.append(float(np.mean([a.elapsed_time(b) for a, b in evs])))
    return out


def graph_step_timing(op, step, steps, flush, stream_ctx):
    """Capture `step` (a sequence of C-ABI calls) in a CUDA graph and time replays,
    flushing L2 between replays outside the events.  Returns ms per step."""
    import torch
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        op.set_stream(side)
        step()
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        op.set_stream(torch.cuda.current_stream())
        step()
    op.set_stream(torch.cuda.current_stream())
    for _ in range(3):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    cur = torch.cuda.current_stream()
    for a, b in evs:
        flush.zero_()
        a.record(cur)
        g.replay()
        b.record(cur)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def batched_frames(dev, steps, flush):
    """16 frames of 256^2 with 30-120 golden-angle views each (uneven), Krylov
    block 8, one persistent launch per operator, replayed from a CUDA graph."""
    import torch
    from paper_2605_06336_gb300 import ct, synth
    w = synth.make_workload("C4")
    K = 8
    op = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=K, dtype=torch.float32)
    tuning = op.autotune()
    rng = np.random.default_rng(4)
    th = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    dth = torch.tensor(rng.standard_normal(w.V), dtype=torch.float64, device=dev)
    X = torch.tensor(rng.uniform(size=(K, op.n)), dtype=torch.float32, device=dev)
    Ys = torch.tensor(rng.standard_normal((K, op.m)), dtype=torch.float32, device=dev)
    Y, Xa = torch.empty_like(Ys), torch.empty_like(X)
    dy = torch.empty(op.m, device=dev)
    gt = torch.empty(w.V, dtype=torch.float64, device=dev)

    def step():
        ct.ct_forward(op.h, th, None, X, Y, K)
        ct.ct_adjoint(op.h, th, None, Ys, Xa, K)
        ct.ct_jac(op.h, th, None, X[0], dth, None, dy)
        ct.ct_jacT(op.h, th, None, X[0], Ys[0], gt, None)

    ms = graph_step_timing(op, step, steps, flush, None)
    samples = w.V * w.B * (K + K + 1 + 1)
    return {"workload": f"C4: {w.F} frames of {w.N}x{w.N}, {w.V} views in total "
                        f"({min(w.views_per_frame)}-{max(w.views_per_frame)} per frame), {w.B} bins, Krylov block {K}",
            "ms_per_step": ms, "value": samples / (ms * 1e-3) / 1e9, "unit": "GSamples/s",
            "tuning": dict(zip(ct.TUNING_FIELDS, tuning)), "launch": "CUDA graph replay"}


def fan_beam_step(dev, steps, flush):
    """The headline step (H on an 8-image block, H^T on 8 sinograms, J dtheta,
    J^T r) on the 256^2 / 180-view / 363-bin workload in fan-beam geometry
    (source at 2N from the rotation centre), replayed from a CUDA graph; the
    fan-beam kernels take only the images-per-lane shapes (kb) of the tuning."""
    import torch
    from paper_2605_06336_gb300 import ct, synth
    w = synth.make_workload(WORKLOAD)
    K = KBLOCK
    D = 2.0 * w.N
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=K, dtype=torch.float32, source_distance=D)
    rng = np.random.default_rng(6)
    th = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    dth = torch.tensor(rng.standard_normal(w.V), dtype=torch.float64, device=dev)
    X = torch.tensor(np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(K - 1, op.n))]),
                     dtype=torch.float32, device=dev)
    Ys = torch.tensor(rng.standard_normal((K, op.m)), dtype=torch.float32, device=dev)
    Y, Xa = torch.empty_like(Ys), torch.empty_like(X)
    dy = torch.empty(op.m, device=dev)
    gt = torch.empty(w.V, dtype=torch.float64, device=dev)

    def step():
        ct.ct_forward(op.h, th, None, X, Y, K)
        ct.ct_adjoint(op.h, th, None, Ys, Xa, K)
        ct.ct_jac(op.h, th, None, X[0], dth, None, dy)
        ct.ct_jacT(op.h, th, None, X[0], Ys[0], gt, None)

    ms = graph_step_timing(op, step, steps, flush, None)
    samples = w.V * w.B * (K + K + 1 + 1)
    return {"workload": f"fan beam, source at {D:.0f} px: {w.N}x{w.N}, {w.V} views, {w.B} bins, Krylov block {K}",
            "ms_per_step": ms, "value": samples / (ms * 1e-3) / 1e9, "unit": "GSamples/s",
            "tuning": dict(zip(ct.TUNING_FIELDS, op.tuning)), "launch": "CUDA graph replay"}


def cpu_baseline(w, seconds):
    import oracle
    g = oracle.Geometry(w.N, w.B, w.V)
    x = w.images.reshape(-1)
    y = oracle.forward(g, w.theta_true, x)
    dth = np.ones(w.V)
    t0 = time.perf_counter()
    n = 0
    while n == 0 or (time.perf_counter() - t0) < seconds:
        oracle.forward(g, w.theta_true, x)
        oracle.adjoint(g, w.theta_true, y)
        oracle.jac(g, w.theta_true, x, dth)
        oracle.jacT(g, w.theta_true, x, y)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": w.V * w.B * 4 * n / dt / 1e9, "unit": "GSamples/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} passes of H, H^T, J, J^T on one 256^2 image (not the 8-image block), FP64, "
                      f"single thread, {dt:.1f} s"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2605_06336_gb300 import ct, synth
    ct.load_library()  # fails loudly if the CUDA library is missing

    if args.fan_only:
        import torch
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"fan_beam": fan_beam_step(dev, max(args.steps, 1), flush)}), flush=True)
        return
    if args.stream_only:
        print(json.dumps({"streaming": streaming_c5(dev, max(args.stream_passes, 1), args.stream_scale)}), flush=True)
        return
    w = synth.make_workload(WORKLOAD)
    if args.solver_only:
        tun = [int(x) for x in args.tuning.split(",")] if args.tuning else None
        ws = synth.make_workload(args.solver_workload)
        extra = {"varpro": int(args.varpro)}
        if ws.F > 1:
            extra["temporal"] = 1
        out = solver_only(ws, dev, args.solver_iters, tun, **extra)
        print(json.dumps({"solver_only": out}), flush=True)
        return
    N, B, V, K = w.N, w.B, w.V, KBLOCK
    rng = np.random.default_rng(100 + rank)
    Xh = np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(K - 1, N * N))]).astype(np.float32)
    Ysh = rng.standard_normal((K, V * B)).astype(np.float32)
    dth_h = rng.standard_normal(V)
    op = ct.CTOperator(N, B, V, max_batch=K, dtype=torch.float32)
    if args.tuning:
        op.tuning = [int(x) for x in args.tuning.split(",")]
        tuning = op.tuning
    else:
        tuning = op.autotune()
    stream = torch.cuda.current_stream()
    theta = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    X = torch.tensor(Xh, device=dev)
    Ys = torch.tensor(Ysh, device=dev)
    dth = torch.tensor(dth_h, dtype=torch.float64, device=dev)
    Y = torch.empty(K, V * B, device=dev)
    Xa = torch.empty(K, N * N, device=dev)
    dy = torch.empty(V * B, device=dev)
    gt = torch.empty(V, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(ev=None):
        if ev: ev[0].record(stream)
        ct.ct_forward(op.h, theta, None, X, Y, K)
        if ev: ev[1].record(stream)
        ct.ct_adjoint(op.h, theta, None, Ys, Xa, K)
        if ev: ev[2].record(stream)
        ct.ct_jac(op.h, theta, None, X[0], dth, None, dy)
        if ev: ev[3].record(stream)
        ct.ct_jacT(op.h, theta, None, X[0], Y[0], gt, None)
        if ev: ev[4].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if op.status() != ct.CT_OK:
        raise RuntimeError("device status not OK after warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clk = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()              # evict L2 between timed steps (outside the events)
        step(evs[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    per_op = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(args.steps)])
    step_ms = per_op.sum(axis=1)
    total_ms = float(step_ms.sum())
    total_ms = max_over_ranks(total_ms, world, dev)
    samples_per_step = V * B * (K + K + 1 + 1)
    value_eager = job_rate(samples_per_step * args.steps, total_ms, world)
    # the same step replayed from a CUDA graph (what the solver and a serving loop run)
    if world > 1:
        dist.barrier()
    graph_ms = graph_step_timing(op, step, args.steps, flush, None)
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    graph_ms = max_over_ranks(graph_ms, world, dev)
    value = job_rate(samples_per_step, graph_ms, world)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region.
    # Every step uploads its inputs from pinned host memory and downloads all its results.  Serial:
    # the copies and the calls on one stream.  Pipelined (the reported e2e): two device slots for the
    # inputs and outputs; step k+1's upload (one copy stream) and step k-1's download (another) run
    # while step k's kernels run on the handle's stream.
    Xp = torch.tensor(Xh).pin_memory()
    Ysp = torch.tensor(Ysh).pin_memory()
    thp = torch.tensor(w.theta_true, dtype=torch.float64).pin_memory()
    dthp = torch.tensor(dth_h, dtype=torch.float64).pin_memory()
    Yp = torch.empty(K, V * B).pin_memory()
    Xap = torch.empty(K, N * N).pin_memory()
    dyp = torch.empty(V * B).pin_memory()
    gtp = torch.empty(V, dtype=torch.float64).pin_memory()
    h2d = Xp.numel() * 4 + Ysp.numel() * 4 + thp.numel() * 8 + dthp.numel() * 8
    d2h = Yp.numel() * 4 + Xap.numel() * 4 + dyp.numel() * 4 + gtp.numel() * 8

    def e2e_step():
        theta.copy_(thp, non_blocking=True)
        X.copy_(Xp, non_blocking=True)
        Ys.copy_(Ysp, non_blocking=True)
        dth.copy_(dthp, non_blocking=True)
        step()
        Yp.copy_(Y, non_blocking=True)
        Xap.copy_(Xa, non_blocking=True)
        dyp.copy_(dy, non_blocking=True)
        gtp.copy_(gt, non_blocking=True)

    slots = [{"theta": torch.empty_like(theta), "X": torch.empty_like(X), "Ys": torch.empty_like(Ys),
              "dth": torch.empty_like(dth), "Y": torch.empty_like(Y), "Xa": torch.empty_like(Xa),
              "dy": torch.empty_like(dy), "gt": torch.empty_like(gt)} for _ in range(2)]
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]

    def e2e_pipelined(n, start):
        s_up.wait_event(start)
        for k in range(n):
            j = k % 2
            sl = slots[j]
            with torch.cuda.stream(s_up):
                if k >= 2:
                    s_up.wait_event(ev_done[j])       # step k-2 has read this slot's inputs
                sl["theta"].copy_(thp, non_blocking=True)
                sl["X"].copy_(Xp, non_blocking=True)
                sl["Ys"].copy_(Ysp, non_blocking=True)
                sl["dth"].copy_(dthp, non_blocking=True)
                ev_up[j].record(s_up)
            stream.wait_event(ev_up[j])
            if k >= 2:
                stream.wait_event(ev_down[j])         # step k-2's results have left this slot
            ct.ct_forward(op.h, sl["theta"], None, sl["X"], sl["Y"], K)
            ct.ct_adjoint(op.h, sl["theta"], None, sl["Ys"], sl["Xa"], K)
            ct.ct_jac(op.h, sl["theta"], None, sl["X"][0], sl["dth"], None, sl["dy"])
            ct.ct_jacT(op.h, sl["theta"], None, sl["X"][0], sl["Y"][0], sl["gt"], None)
            ev_done[j].record(stream)
            with torch.cuda.stream(s_down):
                s_down.wait_event(ev_done[j])
                Yp.copy_(sl["Y"], non_blocking=True)
                Xap.copy_(sl["Xa"], non_blocking=True)
                dyp.copy_(sl["dy"], non_blocking=True)
                gtp.copy_(sl["gt"], non_blocking=True)
                ev_down[j].record(s_down)
        stream.wait_event(ev_down[(n - 1) % 2])

    def timed(run):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        run(e0)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world, dev)

    for _ in range(3):
        e2e_step()
    e2e_serial_ms = timed(lambda e0: [e2e_step() for _ in range(args.steps)])
    ref_out = [t.clone() for t in (Yp, Xap, dyp, gtp)]
    w0 = torch.cuda.Event()
    w0.record(stream)
    e2e_pipelined(3, w0)
    torch.cuda.synchronize()
    e2e_ms = timed(lambda e0: e2e_pipelined(args.steps, e0))
    # the pipelined results must be those of the serial form (same inputs, deterministic kernels)
    e2e_check = max(float((a.double() - b.double()).abs().max()) for a, b in zip((Yp, Xap, dyp, gtp), ref_out))
    e2e_val = job_rate(samples_per_step * args.steps, e2e_ms, world)
    e2e_serial_val = job_rate(samples_per_step * args.steps, e2e_serial_ms, world)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant operator call: device time of each call alone (own graph)
    steps_img = interp_steps_per_image(w)
    op_names = ["forward_K8", "adjoint_K8", "jac", "jacT"]
    calls = [lambda: ct.ct_forward(op.h, theta, None, X, Y, K),
             lambda: ct.ct_adjoint(op.h, theta, None, Ys, Xa, K),
             lambda: ct.ct_jac(op.h, theta, None, X[0], dth, None, dy),
             lambda: ct.ct_jacT(op.h, theta, None, X[0], Y[0], gt, None)]
    mean_ms = np.array(graph_op_timing(op, calls, 200, flush))
    # the projection kernel alone, with its inputs as warm as in the step: the
    # call followed by a rerun of its kernel (ct_forward_repeat /
    # ct_adjoint_repeat), minus the call alone
    def call_and_repeat(call, repeat):
        def f():
            call()
            repeat()
        return f
    twice = graph_op_timing(op, [call_and_repeat(calls[0], lambda: ct.ct_forward_repeat(op.h, Y, K)),
                                 call_and_repeat(calls[1], lambda: ct.ct_adjoint_repeat(op.h, Xa, K))], 200, flush)
    kernel_ms = {"forward_K8": twice[0] - float(mean_ms[0]), "adjoint_K8": twice[1] - float(mean_ms[1])}
    dom_name = max(kernel_ms, key=kernel_ms.get)
    gather_bytes = 8.0 * K * steps_img       # two FP32 pixels (or bins) per interpolation step
    achieved = gather_bytes / (kernel_ms[dom_name] * 1e-3) / 1e9
    shape = tuple(tuning[i] for i in ((0, 1, 2, 7) if dom_name == "forward_K8" else (3, 4, 9)))
    traffic = PROFILED_DRAM_BYTES.get((dom_name, shape))
    # Gather roofline: the same algorithmic bytes against the measured read
    # bandwidth of the level that serves the gathers (ncu: the L1-gather
    # forward misses L1 and hits L2; the staged kernels read shared memory,
    # and the L1-gather transpose mostly hits L1, which shares its data path).
    l2_gbs, smem_gbs = ct.ct_measure_peaks()
    gather = {}
    for name, staged in (("forward_K8", tuning[7] > 0), ("adjoint_K8", tuning[9] > 0)):
        level = "smem" if staged else ("L2" if name == "forward_K8" else "L1")
        pk = l2_gbs if level == "L2" else smem_gbs
        ach = gather_bytes / (kernel_ms[name] * 1e-3) / 1e9
        gather[name] = {"level": level, "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk}
    sm_mhz = SM_MAX_MHZ_NOMINAL
    peak = NUM_SMS * LSU_BYTES_PER_CLK_SM * sm_mhz * 1e6 / 1e9
    peaks, src = measured_peaks()
    solver = None
    frames = None
    fan = None
    streaming = None
    dynamic = None
    varpro = None
    if not args.no_solver and world == 1:
        solver = solver_comparison(w, dev, args.solver_iters)
        # the same solve with the VarPro parameter update (Alg. "UPDATE-PARAM-VarPro")
        varpro = solver_comparison(w, dev, args.solver_iters, varpro=1)
        varpro["note"] = ("NL-RMM-GKS with the VarPro Gauss-Newton update on the compressed basis; compare "
                          "ms_per_outer_iter, final_rre and rel_angle_err with 'solver' (per-view AltMin update)")
        frames = batched_frames(dev, min(args.steps, 200), flush)
        fan = fan_beam_step(dev, min(args.steps, 200), flush)
        streaming = streaming_c5(dev, args.stream_passes) if args.stream_passes > 0 else None
        wd = synth.make_workload("C4")
        dynamic = solver_comparison(wd, dev, wd.outer_iters, temporal=1)
        dynamic["workload"] = (f"C4: {wd.F} frames of {wd.N}x{wd.N} (phantom translating 1 px per frame), {wd.V} "
                               f"golden-angle views ({min(wd.views_per_frame)}-{max(wd.views_per_frame)} per "
                               f"frame), {wd.B} bins; ANISO-TV")
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": "GSamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": graph_ms, "higher_is_better": True,
        "eager": {"value": value_eager, "ms_per_step": total_ms / args.steps,
                  "note": "the same step as individual launches (per-op times below)"},
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "C2: 256x256 random-ellipse phantom, 180 views (1 deg angle errors), 363 bins; "
                               "step = H on 8 images + H^T on 8 sinograms + J dtheta + J^T r",
                   "krylov_block": K, "samples_per_step": samples_per_step,
                   "l2": "flushed between timed steps (512 MB write, outside the events)",
                   "launch": "step captured once in a CUDA graph and replayed (value); eager launches under 'eager'",
                   "parallelism": f"replicas x{world}"},
        "per_op_ms": dict(zip(op_names, [float(x) for x in mean_ms])),
        "per_op_ms_note": "device time of each call (all its kernels) replayed alone from a CUDA graph, L2 flushed",
        "per_op_ms_eager": dict(zip(op_names, [float(x) for x in per_op.mean(axis=0)])),
        "kernel_ms": kernel_ms,
        "kernel_ms_note": "projection kernel alone: graph of the call followed by ct_forward_repeat / "
                          "ct_adjoint_repeat minus the graph of the call, L2 flushed before each replay",
        "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch (ncu DRAM read+write)",
                     "launch_ms": kernel_ms[dom_name],
                     "basis": f"8 B of gathered FP32 operands per interpolation step x {K} x {steps_img} steps per "
                              f"launch; peak = {NUM_SMS} SMs x {LSU_BYTES_PER_CLK_SM} B/clk L1 data path x "
                              f"{sm_mhz:.0f} MHz",
                     "hbm_peak_gbs": peaks.get("hbm_gbs"), "peak_source": "derived (unit counts x nominal max clock)"},
        "gather_roofline": gather,
        "gather_roofline_note": "algorithmic gather bytes per launch / kernel time against the read bandwidth of the "
                                "level serving the gathers, measured on this GPU by ct_measure_peaks "
                                f"(L2 {l2_gbs:.0f} GB/s, shared memory {smem_gbs:.0f} GB/s)",
        "cpu_baseline": cpu,
        "solver": solver,
        "batched_frames": frames,
        "fan_beam": fan,
        "streaming": streaming,
        "dynamic_solver": dynamic,
        "varpro_solver": varpro,
        "e2e": {"value": e2e_val, "unit": "GSamples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps, "serial_value": e2e_serial_val,
                "max_abs_diff_vs_serial": e2e_check,
                "note": "C ABI calls on host data: every step uploads its inputs from pinned memory and downloads "
                        "all its results, inside the timed region; uploads and downloads run on two copy streams "
                        "overlapping the neighbouring steps' kernels (two device slots); serial_value: the same "
                        "with copies and calls on one stream"},
        "gpu_launches": launches_per_step(tuning) * args.steps,
        "gpu_launches_note": f"{launches_per_step(tuning)} kernels per step in the replayed graph",
        "tuning": dict(zip(ct.TUNING_FIELDS, tuning)),
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
