"""Continuous-batching server for NUFFT reconstruction and trajectory-gradient requests.

Request kinds (2-D, SENSE model E = (I kron A) S, Sec. II-B, II-G):

* ``recon``: CG-SENSE, ``iters`` CG iterations on (E'E + lam I) x = E'y; returns x.
* ``traj_grad``: the gradient w.r.t. omega of L = ||E(omega) x - y||^2, i.e.
  v = 2 (E x - y) and grad_omega = Re{conj(v) (-i) E(x . r^[d])} (Eq. (e,jac,Ax,v)).

Scheduling: requests wait in FIFO order and are admitted as soon as an
execution slot (a CUDA stream) is free and their device memory fits the budget
(plan workspace from nufft_workspace_bytes plus the request's tensors and CG
temporaries).  Plans stay resident, pooled by (shape, channels, point capacity),
and are reused by later requests (nufft_set_points re-sorts their bins).  An
admitted job enqueues all its GPU work on its slot's stream without
synchronising the host (the CG scalars stay on the device), so requests that
arrive while others run overlap on the GPU.

Fusion: reconstruction requests on the same problem (the same trajectory and
maps, lam and iteration count) that are pending together are admitted as one
job of up to ``fuse`` right-hand sides: one batched CG whose NUFFT calls carry
all their coil images as channels of one plan (the kernels' per-point weights
and sorted bins are then shared by the whole batch), with the CG scalars kept
per request.

Completion is detected by polling a CUDA event; latency is arrival to
completion on the host clock, split into the wait before admission and the
execution after it.
"""
import collections
import time

import numpy as np
import torch

from . import _abi
from .autograd import cg_solve
from .plan import Plan


class Request:
    __slots__ = ("rid", "kind", "shape", "omega", "x", "smaps", "y", "lam", "iters", "arrival", "admitted_at",
                 "done_at", "result", "bytes", "plan", "event", "slot", "batch")

    def __init__(self, rid, kind, shape, omega, smaps, x=None, y=None, lam=1e-3, iters=15):
        self.rid, self.kind, self.shape = rid, kind, tuple(shape)
        self.omega, self.smaps, self.x, self.y = omega, smaps, x, y
        self.lam, self.iters = float(lam), int(iters)
        self.arrival = self.admitted_at = self.done_at = None
        self.result = self.plan = self.event = self.slot = None
        self.bytes = 0
        self.batch = 1   # requests in its job


class Server:
    def __init__(self, budget_bytes=120 << 30, slots=8, device="cuda", fuse=8):
        self.device = torch.device(device)
        self.fuse = max(1, int(fuse))
        self.budget = int(budget_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.pending = collections.deque()
        self.running = []
        self.done = []
        self.pool = collections.defaultdict(list)   # key -> idle plans
        self.plan_bytes = {}                        # id(plan) -> workspace bytes
        self.in_use = 0                             # bytes of admitted requests and idle plans
        self._next = 0

    # ---------------------------------------------------------------- API
    def submit(self, req, now=None):
        req.arrival = time.perf_counter() if now is None else now
        self.pending.append(req)

    def poll(self):
        """Admit what fits, retire what finished; returns the number of finished requests."""
        self._retire()
        self._admit()
        return len(self.done)

    def drain(self):
        while self.pending or self.running:
            self.poll()
        return self.done

    # ---------------------------------------------------------------- internals
    def _fuse_limit(self, req):
        """Most right-hand sides of one fused job: fuse, and no more coil images than one call takes."""
        return max(1, min(self.fuse, _abi.NUFFT_MAX_COILS // int(req.smaps.shape[0])))

    def _channels(self, req, batch):
        """Channel capacity of the plan a job runs on: its coils, or for a fused job coils x the fuse
        limit (one resident plan then serves fused jobs of every size)."""
        C = int(req.smaps.shape[0])
        return C if batch == 1 else C * self._fuse_limit(req)

    def _key(self, req, batch=1):
        M = int(req.omega.shape[1])
        return (req.shape, self._channels(req, batch), 1 << max(0, M - 1).bit_length())

    @staticmethod
    def _same_problem(a, b):
        return (a.kind == b.kind == "recon" and a.shape == b.shape and a.omega is b.omega and a.smaps is b.smaps
                and a.lam == b.lam and a.iters == b.iters)

    def _estimate(self, req, need_plan, batch=1):
        """Device bytes of a job: its plan (if a new one is needed) and its tensors.  A reconstruction
        keeps y, b = E'y and the CG vectors x, r, p, F p plus one forward output per right-hand side (a
        fused one also the coil images S x and E'E p of every right-hand side); a trajectory gradient
        keeps y, E x, v and grad_omega."""
        C, M, N = int(req.smaps.shape[0]), int(req.omega.shape[1]), int(np.prod(req.shape))
        D = len(req.shape)
        if req.kind == "recon":
            tensors = 8 * batch * (2 * C * M + 6 * N + (2 * C * N if batch > 1 else 0))
        else:
            tensors = 8 * (3 * C * M + N) + 4 * D * M
        if not need_plan:
            return tensors
        o = _abi.nufft_default_opts(len(req.shape), req.shape)
        o.max_coils = self._channels(req, batch)
        return tensors + _abi.nufft_workspace_bytes(o, self._key(req)[2])

    def _admit(self):
        while self.pending and self.free_slots:
            req = self.pending[0]
            # requests on the same problem waiting behind it join its job (FIFO order kept)
            group = [req]
            limit = self._fuse_limit(req) if req.kind == "recon" else 1
            if limit > 1:
                for other in list(self.pending)[1:]:
                    if len(group) == limit:
                        break
                    if self._same_problem(req, other):
                        group.append(other)
            batch = len(group)
            key = self._key(req, batch)
            idle = self.pool.get(key)
            need_plan = not idle
            est = self._estimate(req, need_plan, batch)
            if need_plan and self.in_use + est > self.budget:
                self._evict(est)
            if self.in_use + est > self.budget and self.running:
                return                                  # wait for memory (FIFO: no overtaking)
            for r in group:
                self.pending.remove(r)
            slot = self.free_slots.pop()
            now = time.perf_counter()
            with torch.cuda.stream(self.streams[slot]):
                if need_plan:
                    plan = Plan(req.shape, req.omega, max_coils=self._channels(req, batch))
                    self.plan_bytes[id(plan)] = est - self._estimate(req, False, batch)
                else:
                    plan = idle.pop()
                job_bytes = self._estimate(req, False, batch)
                self.in_use += job_bytes + (self.plan_bytes[id(plan)] if need_plan else 0)
                for r in group:
                    r.plan, r.slot, r.bytes, r.batch, r.admitted_at = plan, slot, 0, batch, now
                req.bytes = job_bytes
                if batch == 1:
                    self._launch(req)
                else:
                    self._launch_fused(group)
            self.running.append(group)

    def _evict(self, need):
        for key in list(self.pool):
            while self.pool[key] and self.in_use + need > self.budget:
                plan = self.pool[key].pop()
                self.in_use -= self.plan_bytes.pop(id(plan), 0)
                del plan

    def _launch(self, req):
        plan = req.plan
        plan.set_points(req.omega)
        S = req.smaps
        if req.kind == "recon":
            b = plan.adjoint(req.y, S)
            F = lambda v: plan.adjoint(plan.forward(v, S), S) + req.lam * v
            req.result = cg_solve(F, b, req.iters)
        else:   # traj_grad: L = ||E x - y||^2, v = 2 (E x - y)
            v = 2.0 * (plan.forward(req.x, S) - req.y)
            go, _ = plan.vjp_omega_x(req.x, v, S, need_omega=True, need_x=False)
            req.result = go
        req.event = torch.cuda.Event()
        req.event.record(self.streams[req.slot])

    def _launch_fused(self, group):
        """One CG for B right-hand sides on one problem: E and E' act on all B x C coil images at once
        (maps applied around the channel-batched calls), every scalar per request."""
        req0 = group[0]
        plan, S = req0.plan, req0.smaps
        B, C = len(group), int(S.shape[0])
        plan.set_points(req0.omega)
        conjS = S.conj()

        def E(X):    # [B][N...] -> [B C][M]
            return plan.forward((S.unsqueeze(0) * X.unsqueeze(1)).reshape((B * C,) + req0.shape))

        def Eh(Y):   # [B C][M] -> [B][N...]
            coil = plan.adjoint(Y).reshape((B, C) + req0.shape)
            return (conjS.unsqueeze(0) * coil).sum(dim=1)

        dims = tuple(range(1, 1 + len(req0.shape)))
        vdot = lambda a, b: (a.conj() * b).sum(dim=dims).real.reshape((B,) + (1,) * len(dims))
        Y = torch.cat([r.y for r in group], dim=0)
        bvec = Eh(Y)
        x = torch.zeros_like(bvec)
        r = bvec.clone()
        p = r.clone()
        rr = vdot(r, r)
        for _ in range(req0.iters):
            Fp = Eh(E(p)) + req0.lam * p
            alpha = rr / vdot(p, Fp)
            x = x + alpha * p
            r = r - alpha * Fp
            rr_new = vdot(r, r)
            p = r + (rr_new / rr) * p
            rr = rr_new
        ev = torch.cuda.Event()
        ev.record(self.streams[req0.slot])
        for b, rq in enumerate(group):
            rq.result = x[b]
            rq.event = ev

    def _retire(self):
        still = []
        for group in self.running:
            req = group[0]
            if req.event.query():
                now = time.perf_counter()
                self.free_slots.append(req.slot)
                self.in_use -= req.bytes
                self.pool[self._key(req, len(group))].append(req.plan)
                for r in group:
                    r.done_at = now
                    r.plan = None
                    self.done.append(r)
            else:
                still.append(group)
        self.running = still


def latency_summary(done):
    """Arrival-to-completion latency, and its two phases: the wait before admission and the execution
    after it (a request in a fused job shares its job's execution)."""
    lat = np.array([(r.done_at - r.arrival) * 1e3 for r in done])
    wait = np.array([(r.admitted_at - r.arrival) * 1e3 for r in done])
    run = lat - wait
    batch = np.array([r.batch for r in done])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "n": int(lat.size),
            "wait_p50_ms": float(np.percentile(wait, 50)), "wait_p99_ms": float(np.percentile(wait, 99)),
            "exec_p50_ms": float(np.percentile(run, 50)), "exec_p99_ms": float(np.percentile(run, 99)),
            "fused_requests": int((batch > 1).sum()), "mean_job_size": float(batch.mean())}
