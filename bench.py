"""Benchmark of the NUFFT-Jacobian hot path on the radial 320x320, 16-coil workload.

One step = nufft_set_points (bin sort of omega) + nufft_forward (y = E x) +
nufft_vjp_omega_x (grad_omega by the fused interpolation epilogue, grad_x =
E' v by the register-strip spread): every row of the hot path on one batch.
Throughput unit: non-uniform points x channels per second, with channels =
C (1 + D) per step (C coils, the plain image plus D coordinate-weighted
images per coil).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling); rank 0
prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NU-pts*channels/s & % HBM roofline, batched Jacobian vs plain path; p50/p99 ms"
UNIT = "NU-pts*channels/s"
WORKLOAD = ("radial320: 320x320 complex64 image, 16 Gaussian-bump coil maps, 80 golden-angle spokes x 640 "
            "readout = 51200 points, Kaiser-Bessel J=6, sigma=2 (640x640 grid); step = set_points + forward "
            "+ vjp(grad_omega, grad_x)")
FALLBACK_HBM = 6800.0
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="radial320", choices=["radial320", "cgsense3d", "batched", "serving"],
                    help="radial320: the hot-path step (default); cgsense3d: gradient of an unrolled "
                         "CG-SENSE loss on the 3-D radial workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="radial320: skip the batched, cgsense3d and cuFFT records added to the line")
    ap.add_argument("--sigma", type=float, default=2.0, help="grid oversampling (radial320 workload)")
    ap.add_argument("--J", type=int, default=6, help="interpolation width (radial320 workload)")
    ap.add_argument("--spread", default="auto", choices=["auto", "strips", "tiles", "general"],
                    help="radial320: adjoint spread kernel (auto: the library's choice, register strips in 2-D)")
    ap.add_argument("--serve-problems", type=int, default=64,
                    help="serving: distinct problems (trajectory + maps) the requests draw from")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serving: offered requests per second")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="serving: length of the arrival process")
    ap.add_argument("--serve-fuse", type=int, default=8,
                    help="serving: most same-problem reconstructions fused into one job (1: no fusion)")
    ap.add_argument("--small3d", action="store_true",
                    help="cgsense3d: the same problem at half the side (64x64x48, 250,000 points), for profiling")
    ap.add_argument("--no-graph", action="store_true",
                    help="radial320: time the eager per-call step only (default: replay the step from a CUDA graph)")
    return ap.parse_args()


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the slowest rank sets the job time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


# ------------------------------------------------------------------ workload
def make_inputs():
    from paper_2111_02912_gb300.workloads import workload
    w = workload("radial320")
    C, M = w["C"], w["omega"].shape[1]
    g = np.random.default_rng(2111_02912 + 101)
    v = ((g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))) / math.sqrt(2)).astype(np.complex64)
    w["v"] = v
    return w


def touched_cells(omega, K, J, chunk=65536):
    """Grid cells inside some sample's J-tap window (algorithmic grid footprint U), marked in a
    boolean grid a chunk of samples at a time."""
    D, M = omega.shape
    hit = np.zeros(int(np.prod(K)), dtype=bool)
    for m0 in range(0, M, chunk):
        om = omega[:, m0:m0 + chunk]
        lin = np.zeros((om.shape[1], 1), dtype=np.int64)
        for d in range(D):
            t = om[d].astype(np.float64) * K[d] / (2 * np.pi)
            start = np.floor(t - J / 2.0).astype(np.int64) + 1
            k = np.mod(start[:, None] + np.arange(J)[None, :], K[d])
            lin = (lin[:, :, None] * K[d] + k[:, None, :]).reshape(om.shape[1], -1)
        hit[lin.ravel()] = True
    return int(hit.sum())


# Nominal L1 data return of one SM per cycle (32 lanes x 4 bytes) and the SM count: the 3-D gathers
# read J^D taps x ch channels per point through L1, far more than they move from HBM.
L1_BYTES_PER_CYCLE_SM = 128
SM_COUNT = 152


def gather3d_roofline(prof, omega, K, C, J, sm_mhz):
    """HBM and L1 figures of the 3-D forward and VJP gathers from the library's per-kernel events:
    HBM algorithmic bytes U ch 8 + M D 4 + M C 8 (+ M D 4 for grad_omega), L1 tap bytes M J^D ch 8
    against SM_COUNT x L1_BYTES_PER_CYCLE_SM x the median SM clock."""
    D, M = omega.shape
    U = touched_cells(omega, K, J)
    hbm, hbm_src = peaks()
    l1_peak = SM_COUNT * L1_BYTES_PER_CYCLE_SM * sm_mhz * 1e6 / 1e9
    out = {"U_cells": U, "l1_peak_gbs": round(l1_peak, 1),
           "l1_peak_source": "derived: %d SMs x %d B/cycle x %.0f MHz (median SM clock of the run)" %
                             (SM_COUNT, L1_BYTES_PER_CYCLE_SM, sm_mhz),
           "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    for kind, ch, extra in (("gather_fwd", C, 0), ("gather_vjp", C * D, M * D * 4)):
        if kind not in prof or prof[kind][0] == 0:
            continue
        launches, ms = prof[kind]
        sec = ms / 1e3 / launches
        b_hbm = U * ch * 8 + M * D * 4 + M * C * 8 + extra
        b_l1 = M * J ** D * ch * 8
        out[kind] = {"launches": launches, "us_per_launch": round(sec * 1e6, 1),
                     "hbm_bytes_per_launch": b_hbm, "hbm_gbs": round(b_hbm / sec / 1e9, 1),
                     "hbm_frac": round(b_hbm / sec / 1e9 / hbm, 4),
                     "l1_tap_bytes_per_launch": b_l1, "l1_gbs": round(b_l1 / sec / 1e9, 1),
                     "l1_frac": round(b_l1 / sec / 1e9 / l1_peak, 4)}
    return out


def algorithmic_bytes(w, info):
    """Bytes each kernel kind must move per launch (inputs read once, outputs written once)."""
    N = [info.n[d] for d in range(2)]
    K = [info.k[d] for d in range(2)]
    C, M, D = w["C"], w["omega"].shape[1], 2
    U = touched_cells(w["omega"], K, info.J)
    c8 = 8
    Nimg, Kt = N[0] * N[1], K[0] * K[1]
    fwd_first = lambda ch: Nimg * c8 + C * Nimg * c8 + N[0] * K[1] * ch * c8
    fwd_mid = lambda ch: N[0] * K[1] * ch * c8 + Kt * ch * c8
    return {
        # forward (ch = C) and VJP (ch = C D) launches of the same kinds, averaged per launch
        "fft_fwd_first": (fwd_first(C) + fwd_first(C * D)) / 2,
        "fft_fwd_mid": (fwd_mid(C) + fwd_mid(C * D)) / 2,
        "gather_fwd": U * C * c8 + M * D * 4 + M * C * c8,
        "gather_vjp": U * C * D * c8 + M * D * 4 + M * C * c8 + M * D * 4,
        "spread": M * C * c8 + M * D * 4 + U * C * c8,
        "zero": Kt * C * c8,
        "fft_inv_mid": Kt * C * c8 + N[0] * K[1] * C * c8,
        "fft_inv_last": N[0] * K[1] * C * c8 + C * Nimg * c8 + Nimg * c8,
        "bin_count": M * D * 4 + M * 8, "bin_scatter": M * D * 4 + M * 8 + M * 32,
    }, U


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # samples go to a private temporary file (NUFFT_BENCH_CLOCKS names a file to keep them in)
        self.path = os.environ.get("NUFFT_BENCH_CLOCKS") or os.path.join(
            tempfile.gettempdir(), "nufft_bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_2111_02912_gb300 import Plan, nufft_launch_count
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    # the oracle's worker processes (spawn) start first and warm up while the GPU work runs
    pool = OraclePool(16) if rank == 0 and not args.no_cpu_baseline else None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_inputs()
    C, M, D = w["C"], w["omega"].shape[1], 2
    units = M * C * (1 + D)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    om, X, S, V = t(w["omega"]), t(w["x"]), t(w["smaps"]), t(w["v"])
    plan = Plan(w["shape"], om, max_coils=C, J=args.J, sigma=args.sigma, spread=args.spread)
    y = torch.empty((C, M), dtype=torch.complex64, device=dev)
    go = torch.empty((D, M), dtype=torch.float32, device=dev)
    gx = torch.empty(tuple(w["shape"]), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.set_points(om)
        plan.forward(X, S, out=y)
        return plan.vjp_omega_x(X, V, S, out=(go, gx))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()

    # The whole step (sort, forward, VJP: the same kernels, inputs read at replay) captured once in a
    # CUDA graph and replayed each step, as a static-shape training loop would; the eager per-call
    # step is timed as well.
    graph, graph_launches = None, 0
    if not args.no_graph:
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        c0 = nufft_launch_count()
        with torch.cuda.graph(graph):
            step()
        graph_launches = nufft_launch_count() - c0
        torch.cuda.synchronize()
        for _ in range(max(3, args.warmup)):
            graph.replay()

    def timed_region(profile, use_graph=False):
        plan.profile_enable(profile)
        if profile:
            plan.profile_read()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        n0 = nufft_launch_count()
        for a, b in evs:
            flush.fill_(1.0)                 # evict L2 between steps (outside the events)
            a.record(stream)
            if use_graph:
                graph.replay()
            else:
                step()
            b.record(stream)
        barrier()
        n1 = nufft_launch_count() + (graph_launches * len(evs) if use_graph else 0)
        ms = [a.elapsed_time(b) for a, b in evs]
        prof = plan.profile_read() if profile else None
        plan.profile_enable(False)
        return ms, n1 - n0, prof

    # both ways of running the step, back to back: replayed from the graph and issued call by call;
    # the line reports the faster one (the same on every rank: the comparison is over the max)
    with ClockSampler(local) as clk:
        ms_graph, launches_graph, _ = timed_region(False, use_graph=True) if graph is not None else (None, 0, None)
        ms_eager, launches_eager, _ = timed_region(False)
    clocks = clk.summary()
    graph_ms = max_over_ranks(float(sum(ms_graph)), dev) if graph is not None else None
    eager_ms = max_over_ranks(float(sum(ms_eager)), dev)
    if graph is not None and graph_ms < eager_ms:
        ms, launches, total_ms, step_mode = ms_graph, launches_graph, graph_ms, "CUDA graph of the whole step, captured once"
    else:
        ms, launches, total_ms, step_mode = ms_eager, launches_eager, eager_ms, "eager per-call (public API calls)"
    value = ws * units * args.steps / (total_ms / 1e3)

    # kernel roofline: the same timed region with per-kernel events on the launching stream
    ms_p, _, prof = timed_region(True)
    info = plan.info()
    algo, U = algorithmic_bytes(w, info)
    hbm, hbm_src = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, kms) = dom
    per_launch_ms = kms / nl
    achieved = algo.get(name, 0.0) / (per_launch_ms / 1e3) / 1e9
    roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)"
            if hbm_src == "measured" else "fallback",
            "traffic": traffic_for(name) if args.spread == "auto" else None, "algorithmic_bytes_per_launch": int(algo.get(name, 0)),
            "launch_ms": round(per_launch_ms, 5), "share_of_step": round(kms / sum(v[1] for v in prof.values()), 3),
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4), "gbs": round(algo[k] * v[0] / (v[1] / 1e3) / 1e9, 1)
                            if k in algo else None} for k, v in prof.items()},
            "profiled_ms_per_step": round(float(np.mean(ms_p)), 5), "U_cells": U}

    # end to end through the public API from pinned host memory
    hx = torch.from_numpy(w["x"]).pin_memory()
    hs = torch.from_numpy(w["smaps"]).pin_memory()
    hom = torch.from_numpy(w["omega"]).pin_memory()
    hv = torch.from_numpy(w["v"]).pin_memory()
    hy = torch.empty((C, M), dtype=torch.complex64).pin_memory()
    hgo = torch.empty((D, M), dtype=torch.float32).pin_memory()
    hgx = torch.empty(w["shape"], dtype=torch.complex64).pin_memory()
    h2d = sum(a.numel() * a.element_size() for a in (hx, hs, hom, hv))
    d2h = sum(a.numel() * a.element_size() for a in (hy, hgo, hgx))

    # Copies run on a second stream and each input is waited for just before its first use:
    # omega first, sorted on a third stream (nufft_sort_points) while x and the maps are still
    # being copied; then the forward; v (VJP) arrives during the forward; y goes back to the host
    # while the VJP runs.  The step's events bracket all three streams.
    copy_stream = torch.cuda.Stream()
    sort_stream = torch.cuda.Stream()
    ev_om, ev_xs, ev_v, ev_y, ev_done, ev_sorted = (torch.cuda.Event() for _ in range(6))

    def e2e_step():
        copy_stream.wait_stream(stream)          # the previous step no longer reads the buffers
        sort_stream.wait_stream(stream)          # ... nor the plan's sorted points
        with torch.cuda.stream(copy_stream):
            om.copy_(hom, non_blocking=True)
            ev_om.record(copy_stream)
            X.copy_(hx, non_blocking=True)
            S.copy_(hs, non_blocking=True)
            ev_xs.record(copy_stream)
            V.copy_(hv, non_blocking=True)
            ev_v.record(copy_stream)
        with torch.cuda.stream(sort_stream):
            sort_stream.wait_event(ev_om)
            plan.set_points(om)
            plan.sort_points()
            ev_sorted.record(sort_stream)
        stream.wait_event(ev_xs)
        stream.wait_event(ev_sorted)
        plan.forward(X, S, out=y)
        ev_y.record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_y)
            hy.copy_(y, non_blocking=True)
            ev_done.record(copy_stream)
        stream.wait_event(ev_v)
        go_, gx_ = plan.vjp_omega_x(X, V, S, out=(go, gx))
        hgo.copy_(go_, non_blocking=True)
        hgx.copy_(gx_, non_blocking=True)
        stream.wait_event(ev_done)

    for _ in range(3):
        e2e_step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for a, b in evs:
        flush.fill_(1.0)
        a.record(stream)
        e2e_step()
        b.record(stream)
    barrier()
    e2e_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), dev)
    e2e = {"value": ws * units * args.steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
           "path": "public API calls (eager), copies from pinned host memory on a second stream overlapped "
                   "with the compute that does not need them; omega sorted (nufft_sort_points) on a third "
                   "stream while x and the maps are copied"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "accuracy": {"sigma": args.sigma, "J": args.J}, "spread": args.spread,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 complex)",
            "data": "synthetic (seeded; shapes of the paper's 2-D multicoil radial case)",
            "config": {"workload": WORKLOAD, "points": M, "coils": C, "channels_per_step": C * (1 + D),
                       "units_per_step": units, "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "step_replay": step_mode,
                       "step_modes": "graph replay and eager calls timed back to back, the faster reported",
                       "graph_ms_per_step": graph_ms / args.steps if graph is not None else None,
                       "eager_ms_per_step": eager_ms / args.steps},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    if pool is not None:
        line["cpu_baseline"] = cpu_baseline(pool, w)
        pool.close()
    if not args.no_extras:
        # the metric's other forms, measured in the same run: the batched path against the plain path,
        # the 3-D CG-SENSE gradient step, and cuFFT beside the library's FFT passes
        line["cufft_compare"] = cufft_compare(info, C)
        line["cufft_compare"]["library_fft_us"] = {k: round(1e3 * v[1] / v[0], 2)
                                                   for k, v in prof.items() if k.startswith("fft_")}
        line["batched"], _ = batched_record(20, 3)
        line["cgsense3d"], _ = cgsense_record(3, 2)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic_radial320.txt")
    if not os.path.exists(path):
        return None
    src = source_hash()
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and f[0] == kernel and f[2] == src:
            return int(float(f[1]))
    return None


def source_hash():
    """Hash of every kernel source: a committed traffic figure applies only to the sources it was taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_02912_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h", ".inc")):
            h.update(name.encode())
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ oracle
def oracle_step(w, coils):
    """The oracle's FP64 same-kernel NUFFT on the same step, restricted to the coils `coils` (a slice)."""
    from oracle import jacobian as jb
    from oracle.nufft import KBNufft
    S = w["smaps"][coils]
    v = w["v"][coils]
    op = KBNufft(w["shape"], w["omega"])           # plan = window geometry (set_points)
    jb.sense_forward(op, w["x"], S)
    jb.vjp_omega_x(op, w["x"], v, S)


_POOL_W = None


def _pool_init():
    """Worker set-up: one host thread per worker (the pool supplies the parallelism) and the
    workload regenerated from its seeds (nothing large crosses the process boundary)."""
    global _POOL_W
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    _POOL_W = make_inputs()


def _pool_step(bounds):
    oracle_step(_POOL_W, slice(*bounds))
    return bounds


class OraclePool:
    """The oracle step with its coils split over worker processes (started with spawn, before or
    apart from any GPU work), one per host core the process may use."""

    def __init__(self, coils):
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        self.workers = max(1, min(self.cores, coils))
        self.chunks = [(c, c + 1) for c in range(coils)]
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_pool_init)
        self.pool.map(_pool_step, self.chunks[: self.workers])   # warm the workers (imports, workload)

    def step(self):
        t0 = time.perf_counter()
        self.pool.map(_pool_step, self.chunks, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(pool, w, reps=3):
    M, D, C = w["omega"].shape[1], 2, w["C"]
    t = float(np.median([pool.step() for _ in range(reps)]))
    return {"value": M * C * (1 + D) / t, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "ms_per_step": 1e3 * t,
            "sample": "the whole radial320 step (all 16 coils, all 51200 points), median of %d; the oracle as it "
                      "stands, one coil per task on %d worker processes (one host thread each) over the %d cores "
                      "this process may use" % (reps, pool.workers, pool.cores)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = make_inputs()
    M, D, C = w["omega"].shape[1], 2, w["C"]
    pool = OraclePool(C)
    for _ in range(args.warmup):
        pool.step()
    times = [pool.step() for _ in range(args.steps)]
    pool.close()
    total = float(sum(times))
    units = M * C * (1 + D)
    value = units * args.steps / total
    sample = ("each step: the whole radial320 step (all 16 coils, all 51200 points), one coil per task on %d worker "
              "processes over %d host cores" % (pool.workers, pool.cores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ cuFFT, for comparison only
def cufft_compare(info, C, steps=20):
    """torch.fft (cuFFT) on the same oversampled grids, timed beside the library's own FFT passes.

    The library's forward FFT is two line passes over the [K0][K1][ch] grid (channels innermost), the
    first fed straight from the image (scaling, maps and zero padding fused, the zero rows never
    transformed).  cuFFT is timed on the already padded grid in the same layout (fft over dims 0 and 1
    of [K0][K1][ch]) and in its preferred layout ([ch][K0][K1]); neither includes the scaling, the
    maps or the padding."""
    import torch
    K0, K1 = info.k[0], info.k[1]
    out = {"note": "comparison only; the product path never calls cuFFT", "grid": [K0, K1]}
    for ch in (C, 2 * C):
        res = {}
        for name, shape, dims in (("same_layout", (K0, K1, ch), (0, 1)), ("batched_layout", (ch, K0, K1), (1, 2))):
            x = torch.randn(shape, dtype=torch.complex64, device="cuda")
            for _ in range(3):
                torch.fft.fftn(x, dim=dims)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in evs:
                a.record()
                torch.fft.fftn(x, dim=dims)
                b.record()
            torch.cuda.synchronize()
            ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
            nbytes = 2 * K0 * K1 * ch * 8 * 2   # two passes, read + write of the full grid
            res[name] = {"us": round(1e3 * ms, 2), "gbs_two_pass": round(nbytes / (ms / 1e3) / 1e9, 1)}
            del x
        out["channels_%d" % ch] = res
    return out


# ------------------------------------------------------------------ 3-D unrolled CG-SENSE
CG_ITERS = 10


def cgsense_units(M, C, D, K):
    """NU-point x channel passes of one loss-gradient step (forward + backward with recomputation).

    forward: E'y, then K Gram products (K forward, K adjoint); backward: per iteration a
    recomputed Gram product, E x and E g, E'E g, and two omega-VJP interpolations of D
    channels; plus the omega-VJP of E'y.  Forward / adjoint passes carry C channels."""
    return M * C * ((4 * K) + (3 * K + 1)) + M * C * D * (2 * K + 1)


def cgsense_record(steps, warmup, name="radial3d"):
    """The 3-D CG-SENSE loss-gradient step: (JSON fields, value, ms per step, clocks)."""
    import torch

    from paper_2111_02912_gb300 import nufft_launch_count
    from paper_2111_02912_gb300.autograd import NufftOperator, cg_sense_unrolled, nufft
    from paper_2111_02912_gb300.workloads import workload
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workload(name)
    C, M, D = w["C"], w["omega"].shape[1], 3
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    om = t(w["omega"]).requires_grad_(True)
    x_true = t(w["x"])
    op = NufftOperator(w["shape"], om, smaps=t(w["smaps"]))
    with torch.no_grad():
        y = nufft(x_true, om.detach(), op)
    lam = 1e-3 * float(M)
    stream = torch.cuda.current_stream()

    def step():
        om.grad = None
        xk = cg_sense_unrolled(y, om, op, lam, CG_ITERS, recompute=True)
        loss = torch.sum(torch.abs(xk - x_true) ** 2)
        loss.backward()
        return loss

    for _ in range(max(1, warmup)):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    n0 = nufft_launch_count()
    torch.cuda.reset_peak_memory_stats()
    with ClockSampler(dev.index or 0) as clk:
        for a, b in evs:
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
    n1 = nufft_launch_count()
    ms = [a.elapsed_time(b) for a, b in evs]
    # one more step, untimed, with the library's per-kernel events: where the 3-D step spends its time
    op.plan.profile_enable(True)
    op.plan.profile_read()
    step()
    torch.cuda.synchronize()
    prof = op.plan.profile_read()
    op.plan.profile_enable(False)
    units = cgsense_units(M, C, D, CG_ITERS)
    clocks = clk.summary()
    shape, spokes, reads = w["shape"], w["omega"].shape[1] // (250 if name == "radial3d" else 125), \
        250 if name == "radial3d" else 125
    rec = {"workload": "cgsense3d: %dx%dx%d image, %d coils, %d points (%d 3-D radial spokes x %d, "
                       "random-walk perturbed); loss = ||x_K - x||^2, x_K = %d unrolled CG-SENSE iterations on "
                       "(E'E + lam I) x = E'y, lam = 1e-3 M; backward with per-iteration recomputation; gradient "
                       "w.r.t. omega (D = 3)" % (shape[0], shape[1], shape[2], C, M, spokes, reads, CG_ITERS),
           "value": units / (float(np.mean(ms)) / 1e3), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
           "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)), "steps": steps,
           "units_per_step": units, "peak_device_bytes": int(torch.cuda.max_memory_allocated()),
           "plan_workspace_bytes": int(op.plan.info().workspace_bytes), "gpu_launches": n1 - n0,
           "l2": "inputs larger than L2",
           "kernels_one_step": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()}}
    rec["gather_roofline"] = gather3d_roofline(prof, w["omega"], [2 * n for n in shape], C, 6,
                                               clocks["sm_mhz"] if clocks else 2070.0)
    return rec, clocks


def run_cgsense3d(args):
    ws, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    rec, clocks = cgsense_record(args.steps, max(3, args.warmup), "radial3d_small" if args.small3d else "radial3d")
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_step"], "p50_ms": rec["p50_ms"],
            "p99_ms": rec["p99_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 (fp32 complex)",
            "data": "synthetic (seeded 3-D radial with random walk, ellipsoid phantom, Gaussian-bump maps)",
            "config": {k: rec[k] for k in ("workload", "units_per_step", "l2", "peak_device_bytes",
                                           "plan_workspace_bytes", "kernels_one_step", "gather_roofline")},
            "gpu_launches": rec["gpu_launches"], "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------------------ batched uneven problems
def config_picks(configs):
    """How many problems the autotuner gave each configuration (a configuration: a tuple of fields)."""
    picks = {}
    for cfg in configs:
        k = ",".join(str(f) for f in cfg) if cfg else "default"
        picks[k] = picks.get(k, 0) + 1
    return picks


def batched_record(steps, warmup):
    """64 uneven problems: the captured-graph batch against the plain per-call path."""
    import torch

    from paper_2111_02912_gb300 import nufft_launch_count
    from paper_2111_02912_gb300.batch import BatchedJacobian
    from paper_2111_02912_gb300.workloads import batched_problems
    probs = batched_problems(64)
    bj = BatchedJacobian(probs, device="cuda", streams=4, autotune=True)
    units = bj.units()
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(max(1, warmup)):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        n0 = nufft_launch_count()
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], nufft_launch_count() - n0

    ms_plain, launches_plain = timed(bj.run_plain)
    bj.capture()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms_graph, _ = timed(bj.replay)
    picks = config_picks(it.config for it in bj.items)
    rec = {"workload": "batched: 64 independent 2-D problems, side uniform over {64,...,384}, M uniform 4000-200000 "
                       "random-angle radial points (spokes of 2N), coils uniform 1-32; per problem set_points + "
                       "forward + vjp(grad_omega, grad_x); autotuned configuration; one CUDA graph over 4 streams",
           "value": units * steps / (sum(ms_graph) / 1e3), "unit": UNIT, "ms_per_step": sum(ms_graph) / steps,
           "p50_ms": float(np.percentile(ms_graph, 50)), "p99_ms": float(np.percentile(ms_graph, 99)),
           "plain_value": units * steps / (sum(ms_plain) / 1e3), "plain_ms_per_step": sum(ms_plain) / steps,
           "plain_p50_ms": float(np.percentile(ms_plain, 50)), "plain_p99_ms": float(np.percentile(ms_plain, 99)),
           "speedup_vs_plain": sum(ms_plain) / sum(ms_graph), "steps": steps, "units_per_step": units,
           "points": sum(it.M for it in bj.items), "configs_picked": picks,
           "config_candidates": "(spread kernel, bin shape, hits per strip part, forward gather lanes)",
           "gpu_launches_plain": launches_plain,
           "l2": "inputs larger than L2"}
    return rec, clk.summary()


def run_batched(args):
    ws, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    rec, clocks = batched_record(args.steps, max(3, args.warmup))
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_step"], "p50_ms": rec["p50_ms"],
            "p99_ms": rec["p99_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 (fp32 complex)", "data": "synthetic (seeded uneven radial problems)",
            "config": {k: v for k, v in rec.items() if k not in ("value", "unit", "ms_per_step", "p50_ms", "p99_ms")},
            "gpu_launches": rec["gpu_launches_plain"], "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------------------ serving
def run_serving(args):
    import torch

    from paper_2111_02912_gb300.serve import Request, Server, latency_summary
    from paper_2111_02912_gb300.workloads import batched_problems
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    probs = batched_problems(args.serve_problems)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pool = [dict(shape=p["shape"], om=t(p["omega"]), S=t(p["smaps"]), x=t(p["x"]), y=t(p["v"]), C=p["C"],
                 M=p["omega"].shape[1]) for p in probs]
    rate, seconds = args.serve_rate, args.serve_seconds
    g = np.random.default_rng(2111_02912 + 5)
    n_req = int(rate * seconds)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n_req))
    picks = g.integers(0, len(pool), n_req)
    kinds = np.where(g.random(n_req) < 0.5, "recon", "traj_grad")

    def make(i, j, kind):
        q = pool[j]
        return Request(i, kind, q["shape"], q["om"], q["S"], x=q["x"], y=q["y"], lam=1e-3, iters=15)

    srv = Server(budget_bytes=120 << 30, slots=8, device=dev, fuse=args.serve_fuse)
    for j in range(len(pool)):                  # warm-up: resident plans for every problem class
        srv.submit(make(-1, j, "recon"))
    srv.drain()
    if args.serve_fuse > 1:
        for j in range(len(pool)):              # and for fused jobs (one plan serves every job size)
            srv.submit(make(-1, j, "recon"))
            srv.submit(make(-1, j, "recon"))
        srv.drain()
    srv.done.clear()

    def units(r, q):
        D = 2
        return q["M"] * q["C"] * (31 if r.kind == "recon" else 1 + D)

    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        k = 0
        while k < n_req or srv.pending or srv.running:
            now = time.perf_counter() - t0
            while k < n_req and arrivals[k] <= now:
                srv.submit(make(k, picks[k], kinds[k]), now=t0 + arrivals[k])
                k += 1
            srv.poll()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    done = srv.done
    tot_units = sum(units(r, pool[picks[r.rid]]) for r in done)
    lat = latency_summary(done)
    line = {"metric": METRIC, "value": tot_units / wall, "unit": UNIT, "n_gpus": ws, "steps": len(done),
            "warmup": len(pool), "ms_per_step": 1e3 * wall / len(done), "p50_ms": lat["p50_ms"],
            "p99_ms": lat["p99_ms"], "latency_phases": {k: lat[k] for k in (
                "wait_p50_ms", "wait_p99_ms", "exec_p50_ms", "exec_p99_ms", "fused_requests", "mean_job_size")},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 (fp32 complex)", "data": "synthetic (seeded uneven radial problems, Poisson arrivals)",
            "config": {"workload": "serving: Poisson arrivals at %.0f req/s for %.1f s; each request picks one of "
                                   "%d uneven 2-D problems (sides 64-384, M 4k-200k, coils 1-32) and is a CG-SENSE "
                                   "reconstruction (15 iterations of E'E + 1e-3 I) or a trajectory gradient of "
                                   "||E x - y||^2 (50/50); 8 slots (streams), 120 GiB admission budget, resident "
                                   "plans, same-problem reconstructions fused up to %d per job"
                                   % (rate, seconds, len(pool), args.serve_fuse),
                       "requests": len(done), "requests_per_s": len(done) / wall, "wall_s": wall,
                       "latency_mean_ms": lat["mean_ms"], "l2": "inputs larger than L2"},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.workload == "serving" and a.impl != "reference":
        run_serving(a)
        sys.exit(0)
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "cgsense3d":
        run_cgsense3d(a)
    elif a.workload == "batched":
        run_batched(a)
    else:
        run_ours(a)
