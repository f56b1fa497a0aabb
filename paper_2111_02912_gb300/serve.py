"""Continuous-batching server for NUFFT reconstruction and trajectory-gradient requests.

Request kinds (2-D, SENSE model E = (I kron A) S, Sec. II-B, II-G):

* ``recon``: CG-SENSE, ``iters`` CG iterations on (E'E + lam I) x = E'y; returns x.
* ``traj_grad``: the gradient w.r.t. omega of L = ||E(omega) x - y||^2, i.e.
  v = 2 (E x - y) and grad_omega = Re{conj(v) (-i) E(x . r^[d])} (Eq. (e,jac,Ax,v)).

Scheduling: requests wait in FIFO order and are admitted as soon as an
execution slot (a CUDA stream) is free and their device memory fits the budget
(plan workspace from nufft_workspace_bytes plus the request's tensors).  Plans
stay resident, pooled by (shape, coils, point capacity), and are reused by
later requests (nufft_set_points re-sorts their bins).  An admitted request
enqueues all its GPU work on its slot's stream without synchronising the host
(the CG scalars stay on the device), so requests that arrive while others run
overlap on the GPU.  Completion is detected by polling a CUDA event; latency is
arrival to completion on the host clock.
"""
import collections
import time

import numpy as np
import torch

from . import _abi
from .autograd import cg_solve
from .plan import Plan


class Request:
    __slots__ = ("rid", "kind", "shape", "omega", "x", "smaps", "y", "lam", "iters", "arrival", "done_at",
                 "result", "bytes", "plan", "event", "slot")

    def __init__(self, rid, kind, shape, omega, smaps, x=None, y=None, lam=1e-3, iters=15):
        self.rid, self.kind, self.shape = rid, kind, tuple(shape)
        self.omega, self.smaps, self.x, self.y = omega, smaps, x, y
        self.lam, self.iters = float(lam), int(iters)
        self.arrival = self.done_at = None
        self.result = self.plan = self.event = self.slot = None
        self.bytes = 0


class Server:
    def __init__(self, budget_bytes=120 << 30, slots=8, device="cuda"):
        self.device = torch.device(device)
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
    @staticmethod
    def _key(req):
        M = int(req.omega.shape[1])
        C = int(req.smaps.shape[0])
        return (req.shape, C, 1 << max(0, M - 1).bit_length())

    def _estimate(self, req, need_plan):
        C, M, N = int(req.smaps.shape[0]), int(req.omega.shape[1]), int(np.prod(req.shape))
        tensors = 8 * (C * M * 3 + N * 8)             # y / residual / forward output, CG vectors
        if not need_plan:
            return tensors
        o = _abi.nufft_default_opts(len(req.shape), req.shape)
        o.max_coils = C
        return tensors + _abi.nufft_workspace_bytes(o, self._key(req)[2])

    def _admit(self):
        while self.pending and self.free_slots:
            req = self.pending[0]
            key = self._key(req)
            idle = self.pool.get(key)
            need_plan = not idle
            est = self._estimate(req, need_plan)
            if need_plan and self.in_use + est > self.budget:
                self._evict(est)
            if self.in_use + est > self.budget and self.running:
                return                                  # wait for memory (FIFO: no overtaking)
            self.pending.popleft()
            slot = self.free_slots.pop()
            with torch.cuda.stream(self.streams[slot]):
                if need_plan:
                    plan = Plan(req.shape, req.omega, max_coils=int(req.smaps.shape[0]))
                    self.plan_bytes[id(plan)] = est - self._estimate(req, False)
                else:
                    plan = idle.pop()
                req.plan, req.slot, req.bytes = plan, slot, self._estimate(req, False)
                self.in_use += req.bytes + (self.plan_bytes[id(plan)] if need_plan else 0)
                self._launch(req)
            self.running.append(req)

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

    def _retire(self):
        still = []
        for req in self.running:
            if req.event.query():
                req.done_at = time.perf_counter()
                self.free_slots.append(req.slot)
                self.in_use -= req.bytes
                self.pool[self._key(req)].append(req.plan)
                req.plan = None
                self.done.append(req)
            else:
                still.append(req)
        self.running = still


def latency_summary(done):
    lat = np.array([(r.done_at - r.arrival) * 1e3 for r in done])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "n": int(lat.size)}
