"""Many independent problems of uneven shape: autotuned plans, one CUDA graph per batch.

Each problem (image size, trajectory, coil count) gets its own plan.  One
"Jacobian step" per problem is nufft_set_points + nufft_forward + nufft_vjp_omega_x
(y, grad_omega, grad_x), the hot path of the 2-D radial case.  Two ways to run
a batch:

* plain: the problems' calls one after another on the current stream;
* graph: every problem's calls recorded once into a CUDA graph, the problems
  dealt round-robin to several streams so that independent problems overlap;
  a step is then one graph launch.

The autotuner times one step per candidate configuration on the device and keeps
the fastest, cached per (shape, coils, log2 M) class.  A configuration is the
adjoint spread kernel (register strips or shared-memory tiles), the bin shape of
the sort (the locality of the gathers' tap reads, and the tile of the tile spread),
for the strips the hits one warp adds before a unit is split into parts (the
work per warp), and the forward gather's lanes (coil pairs or quads).
"""
import math

import torch

from .plan import Plan

# (spread kernel, bin shape, strip part, forward gather lanes); the tile kernel ignores the strip part
CONFIG_CANDIDATES_2D = (
    ("strips", (16, 16), 64, "auto"), ("strips", (16, 16), 32, "auto"), ("strips", (16, 16), 128, "auto"),
    ("strips", (32, 32), 64, "auto"), ("tiles", (16, 16), 0, "auto"), ("tiles", (16, 32), 0, "auto"),
    ("strips", (16, 16), 64, "pairs"), ("strips", (16, 16), 64, "quads"),
)
BIN_CANDIDATES_2D = tuple(sorted({c[1] for c in CONFIG_CANDIDATES_2D}))


def plan_for(item, config):
    spread, bins, part, gather = config
    return Plan(item.shape, item.om, max_coils=item.C, bin_size=bins, spread=spread, strip_part=part, gather=gather)


class Autotuner:
    def __init__(self, candidates=CONFIG_CANDIDATES_2D, reps=3):
        self.candidates = tuple(candidates)
        self.reps = reps
        self.cache = {}
        self.timings = {}

    @staticmethod
    def key(shape, C, M):
        return (tuple(shape), 1 << max(0, int(C) - 1).bit_length(), int(math.log2(max(M, 1))))

    def choose(self, item):
        k = self.key(item.shape, item.C, item.M)
        if k in self.cache:
            return self.cache[k]
        best, best_ms, times = None, float("inf"), {}
        for cfg in self.candidates:
            if any(bd > n * 2 for bd, n in zip(cfg[1], item.shape)):
                continue
            try:
                plan = plan_for(item, cfg)
            except RuntimeError:   # the kernel does not apply to this problem (NUFFT_ERR_UNSUPPORTED)
                continue
            run = lambda: _step(plan, item)
            run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(self.reps):
                run()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / self.reps
            times[cfg] = ms
            if ms < best_ms:
                best, best_ms = cfg, ms
            del plan
        self.cache[k] = best
        self.timings[k] = times
        return best


class _Item:
    def __init__(self, p, device):
        t = lambda a: torch.from_numpy(a).to(device)
        self.shape = tuple(p["shape"])
        self.C = int(p["C"])
        self.om, self.x, self.v = t(p["omega"]), t(p["x"]), t(p["v"])
        self.S = t(p["smaps"]) if p.get("smaps") is not None else None
        self.M = int(self.om.shape[1])
        self.y = torch.empty((self.C, self.M), dtype=torch.complex64, device=device)
        self.go = torch.empty((len(self.shape), self.M), dtype=torch.float32, device=device)
        self.gx = torch.empty(self.shape if self.S is not None else (self.C,) + self.shape,
                              dtype=torch.complex64, device=device)
        self.plan = None
        self.config = None


def _step(plan, it):
    plan.set_points(it.om)
    plan.forward(it.x, it.S, out=it.y)
    plan.vjp_omega_x(it.x, it.v, it.S, out=(it.go, it.gx))


class BatchedJacobian:
    """A batch of independent problems; see the module docstring."""

    def __init__(self, problems, device="cuda", streams=4, autotune=True, tuner=None):
        self.device = torch.device(device)
        self.items = [_Item(p, self.device) for p in problems]
        self.tuner = tuner if tuner is not None else (Autotuner() if autotune else None)
        for it in self.items:
            it.config = self.tuner.choose(it) if self.tuner is not None else None
            it.plan = plan_for(it, it.config) if it.config is not None else Plan(it.shape, it.om, max_coils=it.C)
        self.nstreams = max(1, int(streams))
        self.graph = None

    def units(self):
        """NU-points x channels of one batch step: M C (1 + D) per problem."""
        return sum(it.M * it.C * (1 + len(it.shape)) for it in self.items)

    def run_plain(self):
        for it in self.items:
            _step(it.plan, it)

    def capture(self):
        streams = [torch.cuda.Stream(device=self.device) for _ in range(self.nstreams)]
        main = torch.cuda.current_stream(self.device)
        # warm-up on the side streams (first launches set kernel attributes outside the capture)
        for i, it in enumerate(self.items):
            s = streams[i % self.nstreams]
            s.wait_stream(main)
            with torch.cuda.stream(s):
                _step(it.plan, it)
        for s in streams:
            main.wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cap = torch.cuda.current_stream(self.device)
            for s in streams:
                s.wait_stream(cap)
            for i, it in enumerate(self.items):
                with torch.cuda.stream(streams[i % self.nstreams]):
                    _step(it.plan, it)
            for s in streams:
                cap.wait_stream(s)
        self.graph = g
        self._streams = streams
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def outputs(self):
        return [(it.y, it.go, it.gx) for it in self.items]
