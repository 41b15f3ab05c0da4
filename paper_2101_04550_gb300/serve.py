"""Serving loop: continuous batching of independent lattice Boltzmann solves.

Requests (a grid, its stretch, temperature, viscosity, advection velocity,
storage mode and number of steps) arrive over time.  The server keeps the
populations of admitted requests resident on the GPU, admits waiting
requests whenever the HBM budget and the slot limit allow, and advances all
resident solves together in chunks of steps with the batched step of the
library, one batch for every group of requests that share lattice, storage
mode and kernel form: D3Q27 grids the single pass takes (x a multiple of 32
nodes, y of 16) run in it, one launch per step of the flattened single-pass
kernel over every such request of the group (or per-request graphs, if the
library's autotuner finds them faster for the group's size); the others run
in the two-pass form, one CUDA graph of two launches per step for the whole
group.  Requests that arrive while others run join at the next
chunk boundary; finished ones are read out and freed.  The "plain" mode
serves the same trace one request at a time in arrival order, in the same
kernel forms, with per-step launches and no graphs.

Every computation runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import elbm, inputs

Q_BYTES = {elbm.F32: 4, elbm.F32_SHIFT: 4, elbm.F16_SHIFT: 2, elbm.BF16_SHIFT: 2}
BATCH_MAX = 40  # members of one batch at most


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the trace
    n: tuple                       # (nx, ny, nz)
    stretch: tuple                 # (lam_x, lam_y, lam_z)
    T: float
    nu: float
    advection: tuple               # uniform velocity added to the initial field
    storage: int
    steps: int
    kind: str                      # "shear" or "taylor_green"
    seed: int
    lattice: int = elbm.D3Q27

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def single_pass_fits(self) -> bool:
        """Whether the single-pass form takes this grid (D3Q27, x a multiple
        of 32 nodes, y of 16, 16-byte aligned rows)."""
        nx, ny, _ = self.n
        return (self.lattice == elbm.D3Q27 and nx % 32 == 0 and ny % 16 == 0
                and (nx * Q_BYTES[self.storage]) % 16 == 0)

    def device_bytes(self, single_pass: bool = False) -> int:
        """Populations (with tail padding; two arrays in the single-pass form)
        and the anomaly field."""
        arrays = 2 if single_pass else 1
        return arrays * (self.lattice * self.cells * Q_BYTES[self.storage] + 16) + 3 * self.cells * 4


def make_trace(n_requests=200, rate=20.0, seed=0, steps=2000, sizes=(32, 48, 64, 96, 128)):
    """Seeded Poisson trace: sizes uniform in sizes^3 and 64x32x64 with stretch
    (1, 2, 1); T uniform in [1/3, 0.6]; advection speed uniform in [0, 0.3]
    along a random direction; nu chosen so that omega is uniform in
    [1.6, 1.95]; storage FP32 or FP16 (shifted) with equal odds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    shapes = [((s, s, s), (1.0, 1.0, 1.0)) for s in sizes] + [((64, 32, 64), (1.0, 2.0, 1.0))]
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n, lam = shapes[rng.integers(len(shapes))]
        T = rng.uniform(1.0 / 3.0, 0.6)
        omega = rng.uniform(1.6, 1.95)
        nu = (1.0 / omega - 0.5) * T
        speed = rng.uniform(0.0, 0.3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        storage = elbm.F32_SHIFT if rng.random() < 0.5 else elbm.F16_SHIFT
        kind = "shear" if rng.random() < 0.5 else "taylor_green"
        out.append(Request(rid, t, n, lam, float(T), float(nu), tuple(float(v) for v in speed * d),
                           storage, steps, kind, int(rng.integers(1 << 30))))
    return out


def initial_field(req: Request):
    """Initial rho, u of a request (shear wave along a seeded lattice direction,
    or a Taylor-Green vortex), plus its uniform advection."""
    rng = np.random.Generator(np.random.PCG64(req.seed))
    if req.kind == "shear":
        kd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)][rng.integers(6)]
        k = np.array(kd, float)
        s_dir = np.cross(k, rng.standard_normal(3))
        rho, u, _, _ = inputs.shear_wave(req.n, req.stretch, kd, tuple(s_dir), 1e-2, 0.0)
    else:
        rho, u = inputs.taylor_green_3d(req.n, req.stretch, U=0.02)
    for a in range(3):
        u[a] += req.advection[a]
    return rho, u


@dataclasses.dataclass
class _Slot:
    """A resident request: its solver, the steps it still has to run, when it
    was admitted, and whether its solver is currently a member of its batch."""
    req: Request
    solver: object
    left: int
    t_admit: float
    form: int = 1
    in_batch: bool = False

    @property
    def key(self):
        return (self.req.lattice, self.req.storage, self.form)


class Server:
    """Continuous-batching server over one GPU stream.

    hbm_budget        bytes of populations + anomaly fields that may be resident
    chunk_steps       steps between admission points
    max_active        resident requests at most
    policy            "fifo": admit in arrival order and advance every resident
                      request each chunk; "srpt": admit the smallest waiting
                      request that fits, and each chunk advance the resident
                      requests with the least remaining work (cells x steps
                      left) until step_floor_nodes nodes are in the batch, so
                      that small solves are not held back by large ones while
                      the GPU stays full
    step_floor_nodes  nodes per batched step below which "srpt" adds more requests
    kernels           "auto": the single-pass form for the grids it takes, the
                      two-pass form for the rest; "two-pass": the two-pass form
                      for every request
    sp_config         configuration of the single-pass batches (None: the
                      library's autotuner; 0..11 the flattened launch, 12
                      per-member graphs -- see elbm_batch_set_config)
    clock             callable giving seconds (wall clock by default)
    """

    def __init__(self, hbm_budget=8 << 30, chunk_steps=100, max_active=64, clock=time.perf_counter,
                 stream=None, sleep=time.sleep, policy="fifo", step_floor_nodes=8 << 20, kernels="auto",
                 sp_config=None):
        if policy not in ("fifo", "srpt"):
            raise ValueError("policy must be 'fifo' or 'srpt'")
        if kernels not in ("auto", "two-pass"):
            raise ValueError("kernels must be 'auto' or 'two-pass'")
        self.kernels = kernels
        self.sp_config = sp_config
        self.hbm_budget = int(hbm_budget)
        self.chunk_steps = int(chunk_steps)
        self.max_active = int(max_active)
        self.policy = policy
        self.step_floor_nodes = int(step_floor_nodes)
        self.clock = clock
        self.sleep = sleep
        self.stream = stream
        self.results = {}
        self.failed = {}

    def form(self, req):
        """Kernel form of a request: 3 (single pass) or 1 (two-pass)."""
        return 3 if self.kernels == "auto" and req.single_pass_fits else 1

    def device_bytes(self, req):
        return req.device_bytes(single_pass=self.form(req) == 3)

    def _start(self, req):
        s = elbm.Solver(req.lattice, req.n, stretch=req.stretch, T=req.T, nu=req.nu, storage=req.storage,
                        stream=self.stream, kernel=self.form(req),
                        u_ref=req.advection if req.storage != elbm.F32 else None)
        rho, u = initial_field(req)
        s.init(rho, u)
        return s

    def _finish(self, req, solver, t_start, t_admit):
        _, u = solver.moments(dtype=np.float32)
        t_done = self.clock() - t_start
        solver.close()
        self.results[req.rid] = {"u": u, "arrival": req.arrival, "admitted": t_admit, "done": t_done,
                                 "latency": t_done - req.arrival, "cells": req.cells, "steps": req.steps}

    def _next_waiting(self, queue, used, kinds, n_active):
        """Index in the queue of the request to admit next, or None."""
        if n_active >= self.max_active:
            return None
        order = range(len(queue))
        if self.policy == "srpt":
            order = sorted(order, key=lambda i: (queue[i].cells * queue[i].steps, queue[i].arrival))
        for i in order:
            req = queue[i]
            fits = (used + self.device_bytes(req) <= self.hbm_budget
                    and kinds[(req.lattice, req.storage, self.form(req))] < BATCH_MAX)
            if fits:
                return i
            if self.policy == "fifo":
                return None  # strict arrival order
        return None

    def _stepping(self, active):
        """The resident requests to advance in this chunk."""
        if self.policy == "fifo":
            return list(active)
        chosen, nodes = [], 0
        for a in sorted(active, key=lambda a: (a.req.cells * a.left, a.req.arrival)):
            chosen.append(a)
            nodes += a.req.cells
            if nodes >= self.step_floor_nodes:
                break
        return chosen

    def run(self, trace, mode="batched"):
        """Serve a trace; returns the summary (latencies, makespan, throughput)."""
        self.results = {}
        self.failed = {}
        trace = sorted(trace, key=lambda r: r.arrival)
        t0 = self.clock()
        if mode == "plain":
            for req in trace:
                now = self.clock() - t0
                if now < req.arrival:
                    self.sleep(req.arrival - now)
                t_admit = self.clock() - t0
                s = self._start(req)
                s.step(req.steps)
                self._finish(req, s, t0, t_admit)
            return self.summary(trace)

        pending = collections.deque(trace)
        queue = []
        active = []           # _Slot of every resident request
        used = 0
        batches = {}          # (lattice, storage, form) -> Batch of the stepping members of that kind
        while pending or queue or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            kinds = collections.Counter(a.key for a in active)
            while queue:
                i = self._next_waiting(queue, used, kinds, len(active))
                if i is None:
                    break
                req = queue[i]
                try:
                    solver = self._start(req)
                except elbm.ElbmError as err:
                    if err.code != -3 or not active:  # out of memory with nothing to wait for: give up on it
                        queue.pop(i)
                        self.failed[req.rid] = str(err)
                    break  # out of memory while others run: retry once some finish
                queue.pop(i)
                used += self.device_bytes(req)
                slot = _Slot(req, solver, req.steps, self.clock() - t0, self.form(req))
                kinds[slot.key] += 1
                active.append(slot)
            if not active:
                if queue and all(used + self.device_bytes(r) > self.hbm_budget for r in queue):
                    req = min(queue, key=lambda r: r.arrival)  # larger than the whole budget
                    queue.remove(req)
                    self.failed[req.rid] = f"needs {self.device_bytes(req)} bytes, budget {self.hbm_budget}"
                    continue
                if pending and not queue:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            stepping = self._stepping(active)
            chosen = set(id(a) for a in stepping)
            # batch membership follows the stepping set
            for a in active:
                if a.in_batch and id(a) not in chosen:
                    batches[a.key].remove(a.solver)
                    a.in_batch = False
            for key in [k for k, b in batches.items() if len(b) == 0]:
                batches.pop(key).close()
            for a in stepping:
                if not a.in_batch:
                    if a.key not in batches:
                        batches[a.key] = elbm.Batch([a.solver])
                        if a.form == 3 and self.sp_config is not None:
                            batches[a.key].set_config(self.sp_config)
                    else:
                        batches[a.key].add(a.solver)
                    a.in_batch = True
            chunk = min(self.chunk_steps, min(a.left for a in stepping))
            for b in batches.values():
                b.step(chunk)
            still = []
            for a in active:
                if id(a) in chosen:
                    a.left -= chunk
                if a.left == 0:
                    batches[a.key].remove(a.solver)
                    a.in_batch = False
                    self._finish(a.req, a.solver, t0, a.t_admit)
                    used -= self.device_bytes(a.req)
                else:
                    still.append(a)
            active = still
            for key in [k for k, b in batches.items() if len(b) == 0]:
                batches.pop(key).close()
        for b in batches.values():
            b.close()
        return self.summary(trace)

    def summary(self, trace):
        served = [r for r in trace if r.rid in self.results]
        lat = np.array([self.results[r.rid]["latency"] for r in served]) if served else np.array([np.nan])
        first = min(r.arrival for r in trace)
        makespan = max(self.results[r.rid]["done"] for r in served) - first if served else float("nan")
        work = sum(r.cells * r.steps for r in served)
        span = max(r.arrival for r in trace) - first
        offered = sum(r.cells * r.steps for r in trace) / span / 1e6 if span > 0 else float("nan")
        return {"requests": len(trace), "served": len(served), "failed": len(self.failed),
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "makespan_s": float(makespan), "aggregate_MLUPS": work / makespan / 1e6,
                "offered_MLUPS": offered, "node_updates": int(work)}
