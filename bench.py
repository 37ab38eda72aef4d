"""Benchmark of the angle-dependent CT operator path on GB300.

One step = one pass of the whole operator path over one batch of the
256 x 256 / 180-view / 363-bin workload (random-ellipse phantom, 1-degree
angle errors):
    Y  = H(theta) X      for a Krylov block of K = 8 images
    X' = H(theta)^T Y'   for a block of K = 8 sinograms
    dy = J_theta dtheta  for one image
    g  = J_theta^T r     for one image and one residual
The metric is sinogram samples produced or consumed per second (GSamples/s),
counted as V*B*(K + K + 1 + 1) per step.  The same step is also measured on
the 512^2 / 360-view workload with detector offsets, on one 120-view chunk of
the 2048^2 / 1440-view workload and in FP64; the batched Jacobian products
(K = 8 images per call) and the NL-RMM-GKS solves (plain FP64 form, packaged
FP64 form, packaged FP32 form) are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank runs its own
replica of the workload (the operators shard by views without any exchange;
this build runs replicas only) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "A/Aᵀ/Jθ GSamples/s + NL-RMM-GKS iter time vs FP64 GPU form at equal error"
WORKLOAD = "C2"
KBLOCK = 8
L2_FLUSH_BYTES = 512 * 1024 * 1024
LSU_BYTES_PER_CLK_SM = 128          # L1/shared data path per SM per clock
NUM_SMS = 152
SM_MAX_MHZ_NOMINAL = 2070.0

# DRAM traffic of the dominant kernels per byte of the layout they read (the
# images' pairs or the interleaved images for the forward, the sinograms' pairs
# for the transpose):
# ncu's dram__bytes_read.sum + dram__bytes_write.sum of one launch (cold
# cache) divided by that launch's pair footprint.  The traffic reported for a
# launch is this ratio times its own footprint (the ray kernels read each pair
# of the layout at least once and L2 holds the rest, whatever the launch
# shape).  Captured with the command in profiles/ncu_operator_kernels_256x180x363.md.
TRAFFIC_PER_FOOTPRINT = {
    "forward": 8.56e6 / (2 * 8 * 256 * 260 * 8),        # k_ray<float, kFwd>: 8.56 MB for 8.52 MB of X and X^T pairs
    "forward_staged": 8.58e6 / (2 * 8 * 256 * 260 * 8),  # k_ray_band
    # k_ray<float, kFwd, ..., interleaved>: 4.30 MB for 4.26 MB of interleaved X and X^T
    "forward_interleaved": 4.30e6 / (2 * 8 * 256 * 260 * 4),
    "adjoint": 3.95e6 / (8 * 180 * 368 * 8),            # k_adjoint: 3.95 MB for 4.24 MB of sinogram pairs
    "adjoint_staged": 4.04e6 / (8 * 180 * 368 * 8),      # k_adj_band
}


def launches_per_step(t):
    """Kernels of one bench step at launch shapes t (the ct_get_tuning values):
    forward and J lay out their images and the transpose its sinograms (1
    each; the same launch brings the view table up to date), J^T reuses the
    layout of the J call and brings the view table up to date (1); the forward
    ray kernel(s) over the 8-image block, the transpose, the JVP, the VJP and
    its per-view reduction; the staged forward with several CTAs per ray adds
    a combining kernel (the staged transpose combines its CTAs per tile inside
    their thread-block cluster)."""
    fkb, fsplit, _, akb, asplit, _, _, fstage, _, astage = t[:10]
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
    return 3 + 1 + fwd + adj + 1 + 1 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of each oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solver", action="store_true", help="skip the NL-RMM-GKS comparisons")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads' operator lines")
    ap.add_argument("--solver-iters", type=int, default=30)
    ap.add_argument("--stream-passes", type=int, default=2,
                    help="passes of the streaming solve on the 2048^2 / 1440-view workload (0: skip)")
    ap.add_argument("--solver-only", action="store_true",
                    help="run only the FP32 NL-RMM-GKS solve of the workload (--solver-iters outer iterations) "
                         "and print its timing: the command the solver's profiles are taken with")
    ap.add_argument("--varpro", action="store_true", help="with --solver-only: the VarPro parameter update")
    ap.add_argument("--plain", action="store_true", help="with --solver-only: the plain (unpackaged) form")
    ap.add_argument("--fp64", action="store_true", help="with --solver-only: FP64 operators")
    ap.add_argument("--solver-workload", default=WORKLOAD, choices=["C1", "C2", "C3", "C4"],
                    help="with --solver-only: the workload (C4: the 16-frame dynamic problem, with ANISO-TV)")
    ap.add_argument("--stream-only", action="store_true",
                    help="run only the streaming solve on the 2048^2 / 1440-view workload (--stream-passes passes) "
                         "and print its timing: the command the streaming profiles are taken with")
    ap.add_argument("--fan-only", action="store_true",
                    help="run only the fan-beam operator step (--steps replays) and print its timing")
    ap.add_argument("--ops-only", default=None, choices=["C2", "C3", "C5chunk", "C2fp64", "jac8"],
                    help="run only one operator line (for profiling)")
    ap.add_argument("--stream-scale", type=float, default=1.0,
                    help="with --stream-only: shrink the streaming workload (image side, bins, views)")
    ap.add_argument("--stream-kmax", type=int, default=None, help="with --stream-only: basis size k_max")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shapes (the 12 ct_set_tuning values, comma separated; 11 = forward on "
                         "the pair images) instead of autotuning")
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


def interp_steps_per_image(w, delta=None):
    """Algorithmic work: number of (ray, sample) pairs with -1 < q < N, summed over
    the views (bin centres moved by the offsets delta, if any).  Along a ray the
    in-row (or in-column) coordinate q is affine in the march index r,
    q = A + r k, so the count per ray is the number of integers r in [0, N-1]
    inside the open interval where -1 < q < N (FP64)."""
    N, B = w.N, w.B
    th = np.asarray(w.theta_true, dtype=np.float64)
    c, s = np.cos(th)[:, None], np.sin(th)[:, None]
    h = 0.5 * (N - 1)
    dl = np.zeros(th.size) if delta is None else np.asarray(delta, dtype=np.float64)
    sb = np.arange(B)[None, :] - 0.5 * (B - 1) + dl[:, None]
    rows = np.abs(c) >= np.abs(s)
    with np.errstate(divide="ignore", invalid="ignore"):
        A = np.where(rows, (sb - h * s) / c + h, h - sb / s - h * c / s)
        k = np.where(rows, s / c, c / s) * np.ones_like(sb)
        lo = np.where(k > 0, (-1.0 - A) / k, (N - A) / k)
        hi = np.where(k > 0, (N - A) / k, (-1.0 - A) / k)
        first = np.maximum(0.0, np.floor(lo) + 1.0)
        last = np.minimum(N - 1.0, np.ceil(hi) - 1.0)
        n = np.where(k == 0, np.where((A > -1.0) & (A < N), N, 0), np.maximum(0.0, last - first + 1.0))
    return int(n.sum())


# ---------------------------------------------------------------------------
# clocks during the timed regions
# ---------------------------------------------------------------------------
_REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}


def _pci_bus_id(index):
    import torch
    p = torch.cuda.get_device_properties(index)
    return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)


class ClockSampler:
    """SM clock, its maximum and the slowdown reasons of this process's GPU,
    polled through NVML every ~1 ms in a thread while a timed region runs (the
    GPU is found by its PCI bus id); nvidia-smi every 50 ms if NVML cannot be
    loaded.  Reading only: nothing here changes a setting."""

    def __init__(self, index):
        self.bus = _pci_bus_id(index)
        self.samples = []
        self.source = None
        self._nvml = None
        self._h = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(self.bus.encode(), ctypes.byref(h)) != 0:
                raise OSError("handle")
            self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self._nvml, self._h = lib, h
            self.source = "nvml"
        except (OSError, AttributeError):
            self.source = "nvidia-smi"

    def _poll(self):
        lib, h = self._nvml, self._h
        cur, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(cur)) == 0 and \
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                r = rs.value if self._reasons(h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(cur.value), float(mx.value), int(r)))
            time.sleep(0.001)

    def start(self):
        self.samples = []
        if self.source == "nvml":
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._poll, daemon=True)
            self._t.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(prefix="clk_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                      "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                      "clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.bus}", f"--query-gpu={fields}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.source == "nvml":
            self._stop.set()
            self._t.join()
            sm = [s[0] for s in self.samples]
            mx = [s[1] for s in self.samples]
            reasons = sorted({n for _, _, r in self.samples for n, bit in _REASON_BITS.items() if r & bit})
        else:
            if getattr(self, "proc", None) is None:
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
                if len(p) < 6:
                    continue
                try:
                    sm.append(float(p[0]))
                    mx.append(float(p[1]))
                except ValueError:
                    continue
                for n, val in zip(names, p[2:6]):
                    if val.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
            reasons = sorted(reasons)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": reasons, "source": self.source}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline legs)
# ---------------------------------------------------------------------------
def _oracle_views_task(args):
    """One process of the all-cores oracle run: H, H^T, J, J^T restricted to a
    subset of the views (the operators are per view; H^T's per-view parts are
    summed by the caller, outside the timing of this process's own work)."""
    N, B, theta, x, y, dth, reps = args
    import oracle
    g = oracle.Geometry(N, B, theta.size)
    for _ in range(reps):
        oracle.forward(g, theta, x)
        oracle.adjoint(g, theta, y)
        oracle.jac(g, theta, x, dth)
        oracle.jacT(g, theta, x, y)
    return reps


def cpu_baseline(w, seconds, cores=1):
    """The FP64 oracle as it stands on the host: passes of H, H^T, J, J^T on one
    image of the workload.  cores > 1: the views split over that many processes
    (spawned, so no CUDA state is inherited), each running the same number of
    passes over its views."""
    import oracle
    g = oracle.Geometry(w.N, w.B, w.V)
    x = w.images.reshape(-1)
    y = oracle.forward(g, w.theta_true, x)
    dth = np.ones(w.V)
    if cores <= 1:
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
                "sample": f"{n} passes of H, H^T, J, J^T on one {w.N}^2 image, {w.V} views (not the 8-image "
                          f"block), FP64, single thread, {dt:.1f} s"}
    import multiprocessing as mp
    t0 = time.perf_counter()
    _oracle_views_task((w.N, w.B, w.theta_true, x, y, dth, 1))
    one = time.perf_counter() - t0
    reps = max(1, int(seconds * cores / max(one, 1e-3)))   # about `seconds` of wall time on `cores` processes
    parts = np.array_split(np.arange(w.V), cores)
    Y = y.reshape(w.V, w.B)
    tasks = [(w.N, w.B, w.theta_true[p], x, Y[p].ravel(), dth[p], reps) for p in parts if p.size]
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        pool.map(_oracle_views_task, [(t[0], t[1], t[2], t[3], t[4], t[5], 1) for t in tasks])  # start-up
        t0 = time.perf_counter()
        pool.map(_oracle_views_task, tasks)
        dt = time.perf_counter() - t0
    return {"value": w.V * w.B * 4 * reps / dt / 1e9, "unit": "GSamples/s", "cores": len(tasks), "kind": "oracle",
            "sample": f"{reps} passes of H, H^T, J, J^T on one {w.N}^2 image, views split over {len(tasks)} "
                      f"processes, FP64, {dt:.1f} s"}


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


# ---------------------------------------------------------------------------
# timing helpers
# ---------------------------------------------------------------------------
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


def capture_step(op, step):
    """`step` (a sequence of C-ABI calls on op's handle) captured once in a CUDA graph."""
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
    return g


def graph_replay_timing(g, steps, flush, clock=None):
    """Mean ms of `steps` replays of graph g (L2 flushed before each replay,
    outside the events), after 3 untimed replays; `clock` samples during them."""
    import torch
    for _ in range(3):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    cur = torch.cuda.current_stream()
    if clock:
        clock.start()
    for a, b in evs:
        flush.zero_()
        a.record(cur)
        g.replay()
        b.record(cur)
    torch.cuda.synchronize()
    clk = clock.stop() if clock else None
    return float(np.mean([a.elapsed_time(b) for a, b in evs])), clk


def graph_step_timing(op, step, steps, flush):
    g = capture_step(op, step)
    ms, _ = graph_replay_timing(g, steps, flush)
    return ms


# ---------------------------------------------------------------------------
# one operator step on a workload, with its kernels alone and their roofline
# ---------------------------------------------------------------------------
class OperatorStep:
    """H on K images, H^T on K sinograms, J dtheta and J^T r on one image, through
    the C ABI, with the inputs resident on the device.  J^T is taken at the
    image of the J call, whose pair layouts it uses again (x = NULL), as a
    Gauss-Newton step does, with r = H's first sinogram.  `step` runs the four
    calls in order on one handle; `step_overlapped` runs them on three handles of
    the same geometry and launch shapes, each on a stream of its own (a handle's
    workspace serves one stream): H on the first, H^T on the second, J and then
    J^T (after H) on the third, so that the shared-memory-bound transpose and the
    latency-bound Jacobian products overlap the L2-bound forward."""

    def __init__(self, w, K, dtype, dev, tuning=None, delta=None, seed=100):
        import torch
        from paper_2605_06336_gb300 import ct
        self.w, self.K, self.dtype, self.ct = w, K, dtype, ct
        N, B, V = w.N, w.B, w.V
        rng = np.random.default_rng(seed)
        self.Xh = np.concatenate([w.images.reshape(1, -1)[:, :N * N],
                                  rng.uniform(size=(K - 1, N * N))]).astype(np.float64)
        self.Ysh = rng.standard_normal((K, V * B))
        self.dth_h = rng.standard_normal(V)
        self.op = ct.CTOperator(N, B, V, max_batch=K, dtype=dtype)
        if tuning:
            self.op.tuning = tuning
        else:
            self.op.autotune()
        self.tuning = self.op.tuning
        self.opT = ct.CTOperator(N, B, V, max_batch=K, dtype=dtype)  # H^T's handle in step_overlapped
        self.opT.tuning = self.tuning
        self.sideT = torch.cuda.Stream(device=dev)
        self.opJ = ct.CTOperator(N, B, V, max_batch=K, dtype=dtype)  # J's and J^T's
        self.opJ.tuning = self.tuning
        self.sideJ = torch.cuda.Stream(device=dev)
        self.theta = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
        self.delta = None if delta is None else torch.tensor(delta, dtype=torch.float64, device=dev)
        self.delta_h = delta
        self.X = torch.tensor(self.Xh, dtype=dtype, device=dev)
        self.Ys = torch.tensor(self.Ysh, dtype=dtype, device=dev)
        self.dth = torch.tensor(self.dth_h, dtype=torch.float64, device=dev)
        self.Y = torch.empty(K, V * B, dtype=dtype, device=dev)
        self.Xa = torch.empty(K, N * N, dtype=dtype, device=dev)
        self.dy = torch.empty(V * B, dtype=dtype, device=dev)
        self.gt = torch.empty(V, dtype=torch.float64, device=dev)
        self.samples_per_step = V * B * (K + K + 1 + 1)

    def calls(self):
        ct, op, K = self.ct, self.op, self.K
        th, dl = self.theta, self.delta
        return [lambda: ct.ct_forward(op.h, th, dl, self.X, self.Y, K),
                lambda: ct.ct_adjoint(op.h, th, dl, self.Ys, self.Xa, K),
                lambda: ct.ct_jac(op.h, th, dl, self.X[0], self.dth, None, self.dy),
                # J^T at the image of the J call: its layouts are used again (x = NULL)
                lambda: ct.ct_jacT(op.h, th, dl, None, self.Y[0], self.gt, None)]

    def step(self, ev=None, stream=None):
        for i, c in enumerate(self.calls()):
            if ev:
                ev[i].record(stream)
            c()
        if ev:
            ev[4].record(stream)

    def step_overlapped(self):
        """The same four calls as three branches forked from and joined back into the
        current stream (of one graph when captured): H on op, H^T on opT, J and J^T on
        opJ, J^T after H (its r is H's first sinogram)."""
        self.overlapped_on(self.theta, self.X, self.Y, self.Ys, self.Xa, self.dth, self.dy, self.gt)

    def overlapped_on(self, th, X, Y, Ys, Xa, dth, dy, gt):
        _, overlapped = four_call_steps(self.op, self.opT, self.sideT, th, X, Y, Ys, Xa, dth, dy, gt, self.K,
                                        dl=self.delta, r=Y[0], opJ=self.opJ, sideJ=self.sideJ, r_from_forward=True)
        overlapped()

    def kernels_alone(self, flush, reps=200):
        """Per-call device time (each call replayed from its own graph) and the
        forward / transpose kernels alone (the call followed by a rerun of its
        projection kernel, minus the call)."""
        ct, op, K = self.ct, self.op, self.K
        calls = self.calls()
        per_call = graph_op_timing(op, calls, reps, flush)

        def both(call, repeat):
            def f():
                call()
                repeat()
            return f
        twice = graph_op_timing(op, [both(calls[0], lambda: ct.ct_forward_repeat(op.h, self.Y, K)),
                                     both(calls[1], lambda: ct.ct_adjoint_repeat(op.h, self.Xa, K))], reps, flush)
        return per_call, {"forward": twice[0] - per_call[0], "adjoint": twice[1] - per_call[1]}

    def roofline(self, kernel_ms, l2_gbs, smem_gbs, steps_img):
        """Roofline of the slower of the forward and transpose kernels: the
        algorithmic gather bytes (8 B = two operands per interpolation step, per
        image) of one launch over its time, against the measured read bandwidth
        of the level that serves its gathers."""
        t = self.tuning
        K, w = self.K, self.w
        esz = 4 if self.dtype.itemsize == 4 else 8
        gather_bytes = 2.0 * esz * K * steps_img
        out = {}
        for name in ("forward", "adjoint"):
            staged = (t[7] > 0) if name == "forward" else (t[9] > 0)
            staged = staged and esz == 4
            # the forward on interleaved images reads one float per pixel and image, not a pair
            inter = name == "forward" and len(t) > 11 and t[11] == 1 and esz == 4
            # the L1-gather forward misses L1 and hits L2; the staged kernels read shared
            # memory; the L1-gather transpose mostly hits L1, which shares shared memory's data path
            level = "smem" if staged else ("l2" if name == "forward" else "l1")
            pk = l2_gbs if level == "l2" else smem_gbs
            ach = gather_bytes / (kernel_ms[name] * 1e-3) / 1e9
            if name == "forward":
                footprint = 2.0 * K * w.F * w.N * (w.N + 4) * (1 if inter else 2) * esz
            else:
                footprint = float(K * w.V * ((w.B + 5) & ~1) * 2 * esz)
            fam = name + ("_staged" if staged else ("_interleaved" if inter else ""))
            ratio = TRAFFIC_PER_FOOTPRINT.get(fam) if esz == 4 else None
            out[name] = {"level": level, "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                         "launch_ms": kernel_ms[name], "gather_bytes": gather_bytes,
                         "traffic": None if ratio is None else ratio * footprint,
                         "traffic_family": fam}
        return out


def operator_line(name, w, K, dtype, dev, steps, flush, peaks, delta=None, tuning=None, clock=None):
    """GSamples/s of the operator step on workload w (graph replay, L2 flushed
    between steps) and the roofline of its slower projection kernel."""
    import torch
    s = OperatorStep(w, K, dtype, dev, tuning=tuning, delta=delta)
    for _ in range(3):
        flush.zero_()
        s.step()
    torch.cuda.synchronize()
    if s.op.status() != s.ct.CT_OK:
        raise RuntimeError(f"{name}: device status not OK")
    g = capture_step(s.op, s.step_overlapped)
    ms, clk = graph_replay_timing(g, steps, flush, clock)
    seq_ms, _ = graph_replay_timing(capture_step(s.op, s.step), steps, flush)
    per_call, kms = s.kernels_alone(flush, reps=min(200, max(steps, 20)))
    steps_img = interp_steps_per_image(w, delta)
    rl = s.roofline(kms, peaks[0], peaks[1], steps_img)
    dom = max(kms, key=kms.get)
    nnz_per_step = 2 * steps_img * (s.K + s.K + 1 + 1)
    out = {"workload": name, "value": s.samples_per_step / (ms * 1e-3) / 1e9, "unit": "GSamples/s",
           "ms_per_step": ms, "gnnz_per_s": nnz_per_step / (ms * 1e-3) / 1e9,
           "sequential": {"value": s.samples_per_step / (seq_ms * 1e-3) / 1e9, "ms_per_step": seq_ms},
           "per_call_ms": dict(zip(["forward", "adjoint", "jac", "jacT"], per_call)), "kernel_ms": kms,
           "roofline": rl[dom] | {"kernel": dom}, "roofline_other": rl["adjoint" if dom == "forward" else "forward"],
           "tuning": dict(zip(s.ct.TUNING_FIELDS, s.tuning)), "interp_steps_per_image": steps_img}
    if clk:
        out["clocks"] = clk
    return out, s


def jacobian_batch_line(w, K, dev, steps, flush, peaks, tuning=None):
    """J and J^T on a block of K images sharing the angles, one batched call each
    (ct_jac_batch, ct_jacT_batch), against K single-image calls; gathers per
    launch 8 B x K x interpolation steps, served from L2 (L1-gather kernels)."""
    import torch
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(8)
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=K, dtype=torch.float32)
    if tuning:
        op.tuning = tuning
    else:
        op.autotune()
    th = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    X = torch.tensor(np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(K - 1, w.N * w.N))]),
                     dtype=torch.float32, device=dev)
    R = torch.tensor(rng.standard_normal((K, w.V * w.B)), dtype=torch.float32, device=dev)
    dth = torch.tensor(rng.standard_normal(w.V), dtype=torch.float64, device=dev)
    dY = torch.empty(K, w.V * w.B, device=dev)
    G = torch.empty(K, w.V, dtype=torch.float64, device=dev)
    g1 = torch.empty(w.V, dtype=torch.float64, device=dev)
    calls = [lambda: ct.ct_jac_batch(op.h, th, None, X, dth, None, dY, K),
             lambda: ct.ct_jacT_batch(op.h, th, None, X, R, G, None, K),
             lambda: [ct.ct_jac(op.h, th, None, X[k], dth, None, dY[k]) for k in range(K)],
             lambda: [ct.ct_jacT(op.h, th, None, X[k], R[k], g1, None) for k in range(K)]]
    ms = graph_op_timing(op, calls, min(200, max(steps, 20)), flush)
    steps_img = interp_steps_per_image(w)
    gather = 8.0 * K * steps_img
    samples = K * w.V * w.B
    out = {"workload": f"{w.name}: J and J^T on {K} images sharing the angles, one call each",
           "jac_batch_ms": ms[0], "jacT_batch_ms": ms[1], "jac_single_x8_ms": ms[2], "jacT_single_x8_ms": ms[3],
           "value": 2 * samples / ((ms[0] + ms[1]) * 1e-3) / 1e9, "unit": "GSamples/s",
           "gather_gbs_jac": gather / (ms[0] * 1e-3) / 1e9, "gather_gbs_jacT": gather / (ms[1] * 1e-3) / 1e9,
           "frac_l2_jac": gather / (ms[0] * 1e-3) / 1e9 / peaks[0],
           "frac_l2_jacT": gather / (ms[1] * 1e-3) / 1e9 / peaks[0],
           "note": "times of the whole call (layout of the K images + ray kernel (+ per-view sums)); frac against "
                   "the measured L2 read bandwidth",
           "tuning": dict(zip(ct.TUNING_FIELDS, op.tuning))}
    op.close()
    return out


def c5_chunk_workload():
    """One 120-view chunk of the 2048^2 / 1440-view workload (the chunk the streaming solve visits first)."""
    from paper_2605_06336_gb300 import synth
    w5 = synth.make_workload("C5")
    ch = np.sort(w5.extra["chunks"][0])
    return types.SimpleNamespace(name="C5 chunk", N=w5.N, B=w5.B, V=len(ch), F=1, views_per_frame=[len(ch)],
                                 theta_true=w5.theta_true[ch], images=w5.images)


# ---------------------------------------------------------------------------
# solver comparisons
# ---------------------------------------------------------------------------
def solver_comparison(w, dev, outer_iters, **extra):
    """NL-RMM-GKS on the workload in three forms, same data, same options
    (`extra`: further solver options, e.g. temporal=1 for ANISO-TV):
      fp64_plain      FP64 operators, no CUDA graphs, one basis column per launch
      fp64_packaged   FP64 operators, batched basis projection, graphs
      fp32_packaged   FP32 operators + FP64 small algebra, batched, graphs
    Speedups: precision (fp64_packaged / fp32_packaged), packaging
    (fp64_plain / fp64_packaged), total (fp64_plain / fp32_packaged)."""
    import torch
    from paper_2605_06336_gb300 import ct
    N, B, V = w.N, w.B, w.V
    u_true = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device=dev)
    th_true = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    op64 = ct.CTOperator(N, B, V, w.views_per_frame, max_batch=8, dtype=torch.float64)
    op64.autotune()
    b_true = op64.forward(u_true, th_true)
    e = torch.tensor(w.noise_dir, dtype=torch.float64, device=dev)
    e *= w.noise_level * b_true.norm() / e.norm()
    b64 = b_true + e
    nn = float(e.norm())
    th0 = torch.tensor(w.theta_nominal, dtype=torch.float64, device=dev)
    op32 = ct.CTOperator(N, B, V, w.views_per_frame, max_batch=8, dtype=torch.float32)
    op32.autotune()
    out = {}
    for name, op, plain in (("fp64_plain", op64, 1), ("fp64_packaged", op64, 0), ("fp32_packaged", op32, 0)):
        dt = op.dtype
        bb = b64.to(dt)
        xt = u_true.to(dt)
        op.solve(bb, th0, x_true=xt, noise_norm=nn, outer_iters=2, stop_on_convergence=0, plain=plain,
                 **extra)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, th, st = op.solve(bb, th0, x_true=xt, noise_norm=nn, outer_iters=outer_iters, stop_on_convergence=0,
                             plain=plain, **extra)
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
    p, a, b_ = out["fp64_plain"], out["fp64_packaged"], out["fp32_packaged"]
    out["equal_error"] = (abs(b_["final_rre"] - p["final_rre"]) <= 1e-3 * p["final_rre"] and
                          b_["rel_angle_err"] <= 1.05 * p["rel_angle_err"])
    out["speedup_total"] = p["total_ms"] / b_["total_ms"]
    out["speedup_precision"] = a["total_ms"] / b_["total_ms"]
    out["speedup_packaging"] = p["total_ms"] / a["total_ms"]
    out["outer_iters"] = outer_iters
    out["initial_max_abs_angle_err_deg"] = float(np.abs(w.theta_nominal - w.theta_true).max()) * 180 / math.pi
    out["options"] = {k: v for k, v in extra.items()}
    if extra.get("temporal"):
        # the same FP32 solve with spatial differences only, for the effect of the temporal coupling
        sp = {k: v for k, v in extra.items() if k != "temporal"}
        _, _, st = op32.solve(b64.float(), th0, x_true=u_true.float(), noise_norm=nn, outer_iters=outer_iters,
                              stop_on_convergence=0, **sp)
        out["fp32_spatial_only_final_rre"] = st["rre"][-1]
    op32.close()
    op64.close()
    return out


def solver_only(w, dev, outer_iters, tuning=None, fp64=False, **extra):
    """One NL-RMM-GKS solve of solver_comparison alone (for profiling): autotune
    (or the given launch shapes), one 2-iteration warm-up solve, then the timed solve."""
    import torch
    from paper_2605_06336_gb300 import ct
    u_true = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device=dev)
    th_true = torch.tensor(w.theta_true, dtype=torch.float64, device=dev)
    op64 = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=8, dtype=torch.float64)
    b_true = op64.forward(u_true, th_true)
    e = torch.tensor(w.noise_dir, dtype=torch.float64, device=dev)
    e *= w.noise_level * b_true.norm() / e.norm()
    dt = torch.float64 if fp64 else torch.float32
    b = (b_true + e).to(dt)
    nn = float(e.norm())
    th0 = torch.tensor(w.theta_nominal, dtype=torch.float64, device=dev)
    op = op64 if fp64 else ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=8, dtype=dt)
    if tuning:
        op.tuning = tuning
    else:
        op.autotune()
    op.solve(b, th0, x_true=u_true.to(dt), noise_norm=nn, outer_iters=2, stop_on_convergence=0, **extra)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, th, st = op.solve(b, th0, x_true=u_true.to(dt), noise_norm=nn, outer_iters=outer_iters,
                         stop_on_convergence=0, **extra)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"ms_per_outer_iter": ms / outer_iters, "enlarge_steps": sum(st["enlarge_steps"]),
            "final_rre": st["rre"][-1], "rel_angle_err": float((th - th_true).norm() / th_true.norm()),
            "outer_iters": outer_iters, "options": extra, "fp64": fp64,
            "tuning": dict(zip(ct.TUNING_FIELDS, op.tuning))}


def streaming_c5(dev, passes, scale=1.0, k_max=None):
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
    k_min = 20
    k_max = k_max or STREAM_KMAX
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
           "tuning": dict(zip(ct.TUNING_FIELDS, tuning)), "note": "data from the FP64 GPU forward"}
    for op in ops:
        op.close()
    return out


STREAM_KMAX = 100  # the memory-bounded basis of the large streaming workload


def four_call_steps(op, opT, side, th, X, Y, Ys, Xa, dth, dy, gt, K, dl=None, r=None, opJ=None, sideJ=None,
                    r_from_forward=False):
    """The step's four calls (H on X, H^T on Ys, J dth and J^T r at X[0]; r defaults
    to Ys[0]) in order on op (sequential), and overlapped: forked from and joined
    back into the current stream (branches of one graph when captured), H^T on
    opT and stream `side`; with opJ, J and J^T on opJ and stream sideJ, a third
    branch, whose J^T waits for the forward when r_from_forward (r is one of the
    forward's sinograms); without it, J and J^T follow H on op."""
    import torch
    from paper_2605_06336_gb300 import ct
    r = Ys[0] if r is None else r

    def sequential():
        ct.ct_forward(op.h, th, dl, X, Y, K)
        ct.ct_adjoint(op.h, th, dl, Ys, Xa, K)
        ct.ct_jac(op.h, th, dl, X[0], dth, None, dy)
        ct.ct_jacT(op.h, th, dl, None, r, gt, None)  # the image of the J call

    def overlapped():
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        branches = [side] + ([sideJ] if opJ else [])
        for b in branches:
            b.wait_event(fork)
        op.set_stream(cur)
        opT.set_stream(side)
        if opJ:
            opJ.set_stream(sideJ)
            with torch.cuda.stream(sideJ):
                ct.ct_jac(opJ.h, th, dl, X[0], dth, None, dy)
        ct.ct_forward(op.h, th, dl, X, Y, K)
        if opJ and r_from_forward:
            done = torch.cuda.Event()
            done.record(cur)
            sideJ.wait_event(done)
        with torch.cuda.stream(side):
            ct.ct_adjoint(opT.h, th, dl, Ys, Xa, K)
        if opJ:
            with torch.cuda.stream(sideJ):
                ct.ct_jacT(opJ.h, th, dl, None, r, gt, None)
        else:
            ct.ct_jac(op.h, th, dl, X[0], dth, None, dy)
            ct.ct_jacT(op.h, th, dl, None, r, gt, None)
        for b in branches:
            join = torch.cuda.Event()
            join.record(b)
            cur.wait_event(join)

    return sequential, overlapped


def overlap_lines(op, seq, ovl, steps, flush, samples):
    """Graph-replayed ms of the overlapped and the sequential step (the same calls,
    the same results: the headline step checks this bit for bit)."""
    ms = graph_step_timing(op, ovl, steps, flush)
    ms_seq = graph_step_timing(op, seq, steps, flush)
    return {"ms_per_step": ms, "value": samples / (ms * 1e-3) / 1e9, "unit": "GSamples/s",
            "sequential": {"ms_per_step": ms_seq, "value": samples / (ms_seq * 1e-3) / 1e9}}


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
    opT = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=K, dtype=torch.float32)
    opT.tuning = tuning
    opJ = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=K, dtype=torch.float32)
    opJ.tuning = tuning
    seq, ovl = four_call_steps(op, opT, torch.cuda.Stream(device=dev), th, X, Y, Ys, Xa, dth, dy, gt, K,
                               opJ=opJ, sideJ=torch.cuda.Stream(device=dev))
    samples = w.V * w.B * (K + K + 1 + 1)
    out = {"workload": f"C4: {w.F} frames of {w.N}x{w.N}, {w.V} views in total "
                       f"({min(w.views_per_frame)}-{max(w.views_per_frame)} per frame), {w.B} bins, Krylov block {K}",
           **overlap_lines(op, seq, ovl, steps, flush, samples),
           "tuning": dict(zip(ct.TUNING_FIELDS, tuning)),
           "launch": "CUDA graph replay, three branches on three handles and streams as in the headline step "
                     "(here J^T's r is an input sinogram, so its branch does not wait for H); the four calls in "
                     "order on one handle under 'sequential'"}
    op.close()
    opT.close()
    opJ.close()
    return out


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
    opT = ct.CTOperator(w.N, w.B, w.V, max_batch=K, dtype=torch.float32, source_distance=D)
    opT.tuning = op.tuning
    opJ = ct.CTOperator(w.N, w.B, w.V, max_batch=K, dtype=torch.float32, source_distance=D)
    opJ.tuning = op.tuning
    seq, ovl = four_call_steps(op, opT, torch.cuda.Stream(device=dev), th, X, Y, Ys, Xa, dth, dy, gt, K,
                               opJ=opJ, sideJ=torch.cuda.Stream(device=dev))
    samples = w.V * w.B * (K + K + 1 + 1)
    out = {"workload": f"fan beam, source at {D:.0f} px: {w.N}x{w.N}, {w.V} views, {w.B} bins, Krylov block {K}",
           **overlap_lines(op, seq, ovl, steps, flush, samples),
           "tuning": dict(zip(ct.TUNING_FIELDS, op.tuning)),
           "launch": "CUDA graph replay, three branches on three handles and streams as in the headline step "
                     "(here J^T's r is an input sinogram, so its branch does not wait for H); the four calls in "
                     "order on one handle under 'sequential'"}
    op.close()
    opT.close()
    opJ.close()
    return out


# ---------------------------------------------------------------------------
# the headline run
# ---------------------------------------------------------------------------
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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tun = [int(x) for x in args.tuning.split(",")] if args.tuning else None

    if args.fan_only:
        print(json.dumps({"fan_beam": fan_beam_step(dev, max(args.steps, 1), flush)}), flush=True)
        return
    if args.stream_only:
        print(json.dumps({"streaming": streaming_c5(dev, max(args.stream_passes, 1), args.stream_scale,
                                                    args.stream_kmax)}), flush=True)
        return
    if args.solver_only:
        ws = synth.make_workload(args.solver_workload)
        extra = {"varpro": int(args.varpro), "plain": int(args.plain)}
        if ws.F > 1:
            extra["temporal"] = 1
            extra["k_max"] = 50
        out = solver_only(ws, dev, args.solver_iters, tun, fp64=args.fp64, **extra)
        print(json.dumps({"solver_only": out}), flush=True)
        return
    l2_gbs, smem_gbs = ct.ct_measure_peaks()
    if args.ops_only:
        w = synth.make_workload(WORKLOAD)
        if args.ops_only == "jac8":
            out = jacobian_batch_line(w, KBLOCK, dev, args.steps, flush, (l2_gbs, smem_gbs), tun)
        else:
            wl = {"C2": w, "C2fp64": w, "C3": synth.make_workload("C3"), "C5chunk": c5_chunk_workload()}[args.ops_only]
            dt = torch.float64 if args.ops_only == "C2fp64" else torch.float32
            dl = getattr(wl, "delta_true", None)
            out, _ = operator_line(args.ops_only, wl, KBLOCK, dt, dev, args.steps, flush, (l2_gbs, smem_gbs),
                                   delta=dl, tuning=tun)
        print(json.dumps({"ops_only": out}), flush=True)
        return

    w = synth.make_workload(WORKLOAD)
    N, B, V, K = w.N, w.B, w.V, KBLOCK
    s = OperatorStep(w, K, torch.float32, dev, tuning=tun, seed=100 + rank)
    op, tuning = s.op, s.tuning
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        s.step()
    torch.cuda.synchronize()
    if op.status() != ct.CT_OK:
        raise RuntimeError("device status not OK after warm-up")

    # ---- eager launches, per-call events
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()              # evict L2 between timed steps (outside the events)
        s.step(evs[k], stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    per_op = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(args.steps)])
    total_ms = max_over_ranks(float(per_op.sum()), world, dev)
    samples_per_step = s.samples_per_step
    value_eager = job_rate(samples_per_step * args.steps, total_ms, world)

    # ---- the headline: the same step replayed from a CUDA graph (what the solver and a serving loop
    # run), H^T and the Jacobian products on handles and streams of their own: parallel branches
    g = capture_step(op, s.step_overlapped)
    clock = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    graph_ms, clocks = graph_replay_timing(g, args.steps, flush, clock)
    if world > 1:
        dist.barrier()
    graph_ms = max_over_ranks(graph_ms, world, dev)
    value = job_rate(samples_per_step, graph_ms, world)
    # the four calls in order on one handle and stream, for comparison
    seq_ms, _ = graph_replay_timing(capture_step(op, s.step), args.steps, flush)
    seq_ms = max_over_ranks(seq_ms, world, dev)
    # the overlapped step computes what the sequential one does, bit for bit
    s.step()
    torch.cuda.synchronize()
    seq_out = [t.clone() for t in (s.Y, s.Xa, s.dy, s.gt)]
    s.step_overlapped()
    torch.cuda.synchronize()
    overlap_same = all(torch.equal(a, b) for a, b in zip(seq_out, (s.Y, s.Xa, s.dy, s.gt)))

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region.
    # Every step uploads its inputs from pinned host memory and downloads all its results.  Serial:
    # the copies and the calls on one stream.  Pipelined (the reported e2e): two device slots for the
    # inputs and outputs; step k+1's upload (one copy stream) and step k-1's download (another) run
    # while step k's kernels run on the handle's stream.
    Xp = torch.tensor(s.Xh, dtype=torch.float32).pin_memory()
    Ysp = torch.tensor(s.Ysh, dtype=torch.float32).pin_memory()
    thp = torch.tensor(w.theta_true, dtype=torch.float64).pin_memory()
    dthp = torch.tensor(s.dth_h, dtype=torch.float64).pin_memory()
    Yp = torch.empty(K, V * B).pin_memory()
    Xap = torch.empty(K, N * N).pin_memory()
    dyp = torch.empty(V * B).pin_memory()
    gtp = torch.empty(V, dtype=torch.float64).pin_memory()
    h2d = Xp.numel() * 4 + Ysp.numel() * 4 + thp.numel() * 8 + dthp.numel() * 8
    d2h = Yp.numel() * 4 + Xap.numel() * 4 + dyp.numel() * 4 + gtp.numel() * 8

    def e2e_step():
        s.theta.copy_(thp, non_blocking=True)
        s.X.copy_(Xp, non_blocking=True)
        s.Ys.copy_(Ysp, non_blocking=True)
        s.dth.copy_(dthp, non_blocking=True)
        s.step()
        Yp.copy_(s.Y, non_blocking=True)
        Xap.copy_(s.Xa, non_blocking=True)
        dyp.copy_(s.dy, non_blocking=True)
        gtp.copy_(s.gt, non_blocking=True)

    slots = [{"theta": torch.empty_like(s.theta), "X": torch.empty_like(s.X), "Ys": torch.empty_like(s.Ys),
              "dth": torch.empty_like(s.dth), "Y": torch.empty_like(s.Y), "Xa": torch.empty_like(s.Xa),
              "dy": torch.empty_like(s.dy), "gt": torch.empty_like(s.gt)} for _ in range(2)]
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]

    def compute_on(sl):
        return lambda: s.overlapped_on(sl["theta"], sl["X"], sl["Y"], sl["Ys"], sl["Xa"], sl["dth"], sl["dy"],
                                       sl["gt"])

    def e2e_pipelined(n, start, graphs=None):
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
            # as in the headline step: three branches, forked and joined; replayed from the
            # slot's graph of those calls, or the calls issued one by one
            if graphs:
                graphs[j].replay()
            else:
                compute_on(sl)()
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
    e2e_eager_ms = timed(lambda e0: e2e_pipelined(args.steps, e0))
    # the pipelined results must be those of the serial form (same inputs, deterministic kernels)
    e2e_check = max(float((a.double() - b.double()).abs().max()) for a, b in zip((Yp, Xap, dyp, gtp), ref_out))
    # the same pipeline with each slot's calls captured once in a graph (as a serving loop would):
    # per step the host issues the copies and one graph launch instead of every call's launches
    slot_graphs = [capture_step(op, compute_on(sl)) for sl in slots]
    w1 = torch.cuda.Event()
    w1.record(stream)
    e2e_pipelined(3, w1, slot_graphs)
    torch.cuda.synchronize()
    for t in (Yp, Xap, dyp, gtp):
        t.zero_()
    e2e_ms = timed(lambda e0: e2e_pipelined(args.steps, e0, slot_graphs))
    e2e_check = max(e2e_check, max(float((a.double() - b.double()).abs().max())
                                   for a, b in zip((Yp, Xap, dyp, gtp), ref_out)))
    e2e_val = job_rate(samples_per_step * args.steps, e2e_ms, world)
    e2e_eager_val = job_rate(samples_per_step * args.steps, e2e_eager_ms, world)
    e2e_serial_val = job_rate(samples_per_step * args.steps, e2e_serial_ms, world)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- the headline's kernels alone and their roofline
    per_call, kernel_ms = s.kernels_alone(flush)
    steps_img = interp_steps_per_image(w)
    rl = s.roofline(kernel_ms, l2_gbs, smem_gbs, steps_img)
    dom = max(kernel_ms, key=kernel_ms.get)
    l1_path = NUM_SMS * LSU_BYTES_PER_CLK_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e9
    peaks, src = measured_peaks()
    d = rl[dom]
    roofline = {"bound": d["level"], "kernel": f"{dom}_K{K}", "achieved": d["achieved"], "peak": d["peak"],
                "unit": "GB/s", "frac": d["frac"], "traffic": d["traffic"],
                "traffic_basis": f"ncu DRAM read + write per byte of the launch's image or sinogram layout "
                                 f"({d['traffic_family']} family) x this launch's layout footprint",
                "launch_ms": d["launch_ms"],
                "basis": f"8 B of gathered FP32 operands per interpolation step x {K} images x {steps_img} steps per "
                         f"launch, over the kernel's CUDA-event time",
                "peak_source": f"measured on this GPU by ct_measure_peaks: {d['level']} read bandwidth "
                               f"(L2 {l2_gbs:.0f} GB/s, shared memory / L1 data path {smem_gbs:.0f} GB/s)",
                "l1_data_path_peak": l1_path, "frac_of_l1_data_path": d["achieved"] / l1_path,
                "l1_data_path_basis": f"{NUM_SMS} SMs x {LSU_BYTES_PER_CLK_SM} B/clk x {SM_MAX_MHZ_NOMINAL:.0f} MHz",
                "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": src,
                "hbm_frac": (d["traffic"] / (d["launch_ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"])
                if d["traffic"] else None}
    other = rl["adjoint" if dom == "forward" else "forward"]
    nnz_per_step = 2 * steps_img * (K + K + 1 + 1)

    extra_lines = {}
    if not args.no_extra and world == 1:
        pk = (l2_gbs, smem_gbs)
        w3 = synth.make_workload("C3")
        extra_lines["C3"], _ = operator_line("C3: 512x512, 360 views with per-view offsets, 725 bins, K = 8", w3,
                                             K, torch.float32, dev, min(args.steps, 200), flush, pk,
                                             delta=w3.delta_true)
        extra_lines["C5_chunk"], _ = operator_line("C5 chunk: 2048x2048, 120 views of the 1440-view grid, 2897 bins, "
                                                   "K = 8", c5_chunk_workload(), K, torch.float32, dev,
                                                   min(args.steps, 50), flush, pk)
        extra_lines["C2_fp64"], _ = operator_line("C2 in FP64 (the precision of the paper's arithmetic)", w, K,
                                                  torch.float64, dev, min(args.steps, 200), flush, pk)
        extra_lines["jacobian_batched"] = jacobian_batch_line(w, K, dev, min(args.steps, 200), flush, pk)

    solver = frames = fan = streaming = dynamic = varpro = None
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
        dynamic = solver_comparison(wd, dev, wd.outer_iters, temporal=1, k_max=50)
        dynamic["workload"] = (f"C4: {wd.F} frames of {wd.N}x{wd.N} (phantom translating 1 px per frame), {wd.V} "
                               f"golden-angle views ({min(wd.views_per_frame)}-{max(wd.views_per_frame)} per "
                               f"frame), {wd.B} bins; ANISO-TV; recycling space capped at 50 vectors (k_max)")
    cpu = cpu_all = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, args.cpu_seconds)
        cpu_all = cpu_baseline(w, args.cpu_seconds, cores=os.cpu_count() or 1)

    line = {
        "metric": METRIC, "value": value, "unit": "GSamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": graph_ms, "higher_is_better": True,
        "eager": {"value": value_eager, "ms_per_step": total_ms / args.steps,
                  "note": "the same step as individual launches (per-op times below)"},
        "sequential": {"value": job_rate(samples_per_step, seq_ms, world), "ms_per_step": seq_ms,
                       "same_results_as_overlapped": overlap_same,
                       "note": "the four calls in order on one handle and stream, graph-replayed"},
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "C2: 256x256 random-ellipse phantom, 180 views (1 deg angle errors), 363 bins; "
                               "step = H on 8 images + H^T on 8 sinograms + J dtheta + J^T r at one image "
                               "(J^T reuses the image layout of the J call)",
                   "krylov_block": K, "samples_per_step": samples_per_step,
                   "l2": "flushed between timed steps (512 MB write, outside the events)",
                   "launch": "step captured once in a CUDA graph and replayed (value): three parallel branches "
                             "on three handles of the same geometry, each on its own stream: H; H^T; J, then J^T "
                             "once H is done (its r is H's first sinogram); the four calls in order on one handle "
                             "under 'sequential'; eager launches under 'eager'",
                   "parallelism": f"replicas x{world}"},
        "gnnz_per_s": nnz_per_step / (graph_ms * 1e-3) / 1e9,
        "gnnz_note": "interpolation nonzeros (two per interpolation step) touched per step over the step time",
        "per_op_ms": dict(zip(["forward_K8", "adjoint_K8", "jac", "jacT"], [float(x) for x in per_call])),
        "per_op_ms_note": "device time of each call (all its kernels) replayed alone from a CUDA graph, L2 flushed",
        "per_op_ms_eager": dict(zip(["forward_K8", "adjoint_K8", "jac", "jacT"],
                                    [float(x) for x in per_op.mean(axis=0)])),
        "kernel_ms": {f"{k}_K{K}": v for k, v in kernel_ms.items()},
        "kernel_ms_note": "projection kernel alone: graph of the call followed by ct_forward_repeat / "
                          "ct_adjoint_repeat minus the graph of the call, L2 flushed before each replay",
        "roofline": roofline,
        "roofline_other_kernel": other,
        "roofline_note": "the 60 % target is judged against the measured read bandwidth of the level that serves "
                         "the kernel's gathers (roofline.peak); the derived L1 data path is given beside it",
        "operators": extra_lines or None,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "solver": solver,
        "batched_frames": frames,
        "fan_beam": fan,
        "streaming": streaming,
        "dynamic_solver": dynamic,
        "varpro_solver": varpro,
        "e2e": {"value": e2e_val, "unit": "GSamples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps, "eager_value": e2e_eager_val,
                "eager_ms_per_step": e2e_eager_ms / args.steps, "serial_value": e2e_serial_val,
                "max_abs_diff_vs_serial": e2e_check,
                "note": "C ABI calls on host data: every step uploads its inputs from pinned memory and downloads "
                        "all its results, inside the timed region; uploads and downloads run on two copy streams "
                        "overlapping the neighbouring steps' kernels (two device slots), and the calls run as "
                        "the headline step's three branches, captured once per slot in a CUDA graph and "
                        "replayed every step; eager_value: the same with the calls issued one by one every "
                        "step; serial_value: copies and the four calls in order on one stream, issued one by "
                        "one"},
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
