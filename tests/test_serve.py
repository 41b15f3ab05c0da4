"""Host-side logic of the serving loop, with fake solvers (no GPU): trace
generation, HBM-budget admission, continuous batching (requests join while
others are mid-flight), and an allocation failure injected on the host."""
import dataclasses

import numpy as np
import pytest

from paper_2101_04550_gb300 import elbm, serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class World:
    """Fake device: solvers count steps; one step of one node costs 1 ns."""

    def __init__(self, clock, fail_rids=()):
        self.clock = clock
        self.fail_rids = set(fail_rids)
        self.live = {}
        self.peak_bytes = 0
        self.batch_log = []
        self.batch_kernels = []
        self.kernels = {}

    def solver_cls(self, server):
        world = self

        class FakeSolver:
            def __init__(self, lattice, n, stretch, T, nu, storage, stream=None, kernel=0, u_ref=None):
                req = server._current
                if req.rid in world.fail_rids:
                    raise elbm.ElbmError(-3, "injected out of memory")
                self.req, self.steps_done, self.N, self.kernel = req, 0, n[0] * n[1] * n[2], kernel
                world.kernels[req.rid] = kernel
                world.live[id(self)] = server.device_bytes(req)
                world.peak_bytes = max(world.peak_bytes, sum(world.live.values()))

            def init(self, rho, u):
                self.u0 = u

            def step(self, k):
                self.steps_done += k
                world.clock.t += k * self.N * 1e-9

            def moments(self, dtype=np.float64):
                return None, np.full(3, float(self.steps_done))

            def close(self):
                world.live.pop(id(self), None)

        return FakeSolver

    def batch_cls(self):
        world = self

        class FakeBatch:
            def __init__(self, solvers):
                self.solvers = list(solvers)

            def add(self, s):
                self.solvers.append(s)

            def remove(self, s):
                self.solvers.remove(s)

            def __len__(self):
                return len(self.solvers)

            def step(self, k):
                world.batch_log.append(tuple(s.req.rid for s in self.solvers))
                world.batch_kernels.append(set(s.kernel for s in self.solvers))
                for s in self.solvers:
                    s.steps_done += k
                world.clock.t += k * sum(s.N for s in self.solvers) * 1e-9 / 4  # batching fills the GPU

            def close(self):
                pass

        return FakeBatch


def serve_fake(monkeypatch, trace, budget, fail_rids=(), mode="batched", chunk=50, policy="fifo", floor=4 << 20,
               kernels="auto"):
    clock = FakeClock()
    server = serve.Server(hbm_budget=budget, chunk_steps=chunk, clock=clock, sleep=clock.sleep, policy=policy,
                          step_floor_nodes=floor, kernels=kernels)
    world = World(clock, fail_rids)
    orig_start = server._start

    def start(req):
        server._current = req
        return orig_start(req)

    monkeypatch.setattr(serve.elbm, "Solver", world.solver_cls(server))
    monkeypatch.setattr(serve.elbm, "Batch", world.batch_cls())
    monkeypatch.setattr(serve, "initial_field", lambda req: (None, None))
    server._start = start
    return server, server.run(trace, mode=mode), world


def test_trace_is_seeded_and_in_range():
    a = serve.make_trace(50, seed=3)
    b = serve.make_trace(50, seed=3)
    assert [(r.n, r.T, r.storage) for r in a] == [(r.n, r.T, r.storage) for r in b]
    for r in a:
        assert 1 / 3 <= r.T <= 0.6 and np.linalg.norm(r.advection) <= 0.3 + 1e-12
        omega = 1.0 / (r.nu / r.T + 0.5)
        assert 1.6 - 1e-9 <= omega <= 1.95 + 1e-9
        assert r.n in [(s, s, s) for s in (32, 48, 64, 96, 128)] + [(64, 32, 64)]
    gaps = np.diff([0.0] + [r.arrival for r in serve.make_trace(2000, rate=20.0, seed=1)])
    assert abs(gaps.mean() - 1 / 20) < 0.005


def test_budget_bounds_resident_bytes_and_everything_completes(monkeypatch):
    trace = serve.make_trace(30, seed=5, steps=200)
    budget = 3 * max(r.device_bytes() for r in trace)
    server, summary, world = serve_fake(monkeypatch, trace, budget)
    assert summary["served"] == 30 and summary["failed"] == 0
    assert world.peak_bytes <= budget
    for r in trace:
        assert server.results[r.rid]["u"][0] == 200  # every request ran exactly its steps


def test_requests_join_while_others_run(monkeypatch):
    trace = serve.make_trace(12, seed=2, steps=400, rate=200.0)
    server, summary, world = serve_fake(monkeypatch, trace, budget=1 << 40, chunk=50)
    # some batch contains a request admitted after another member had already started
    admitted = {rid: server.results[rid]["admitted"] for rid in server.results}
    assert any(len(set(admitted[r] for r in ids)) > 1 for ids in world.batch_log)
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0


def test_injected_allocation_failure_is_reported_and_others_finish(monkeypatch):
    trace = serve.make_trace(10, seed=4, steps=100)
    server, summary, world = serve_fake(monkeypatch, trace, budget=1 << 40, fail_rids={3})
    assert 3 in server.failed and summary["served"] == 9


def test_plain_mode_serves_in_order(monkeypatch):
    trace = serve.make_trace(8, seed=6, steps=100)
    server, summary, world = serve_fake(monkeypatch, trace, budget=1 << 40, mode="plain")
    done = [server.results[r.rid]["done"] for r in trace]
    assert done == sorted(done) and summary["served"] == 8


@pytest.mark.parametrize("policy", ["fifo", "srpt"])
def test_every_policy_runs_every_request_exactly(monkeypatch, policy):
    trace = serve.make_trace(40, seed=8, steps=300, rate=100.0)
    budget = 6 * max(r.device_bytes() for r in trace)
    server, summary, world = serve_fake(monkeypatch, trace, budget, policy=policy, floor=1 << 20)
    assert summary["served"] == 40 and world.peak_bytes <= budget
    for r in trace:
        assert server.results[r.rid]["u"][0] == 300


def test_srpt_lets_small_requests_pass_a_large_one(monkeypatch):
    """A 128^3 request arrives first, then ten 32^3 ones: with "srpt" most small
    ones finish before it (the large one fills in whenever the small ones fall
    short of the node floor), and the median latency drops below "fifo"'s."""
    base = serve.make_trace(11, seed=9, steps=400, rate=1000.0)
    big = dataclasses.replace(base[0], n=(128, 128, 128), arrival=0.0, rid=0)
    small = [dataclasses.replace(r, n=(32, 32, 32), arrival=1e-3 * (k + 1), rid=k + 1) for k, r in enumerate(base[1:])]
    trace = [big] + small
    floor = 3 * 32 ** 3
    server, summary, world = serve_fake(monkeypatch, trace, budget=1 << 40, policy="srpt", floor=floor)
    done = {rid: server.results[rid]["done"] for rid in server.results}
    assert sum(done[k] < done[0] for k in range(1, 11)) >= 8
    cells = {r.rid: r.cells for r in trace}
    for ids in world.batch_log:
        stepped = sum(cells[i] for i in ids)
        # the floor is met, or everything resident is being stepped
        assert stepped >= floor or len(ids) == len(set(ids))
    fifo_server, fifo_summary, _ = serve_fake(monkeypatch, trace, budget=1 << 40, policy="fifo")
    assert summary["p50_latency_s"] < fifo_summary["p50_latency_s"]


def test_single_pass_fit_and_bytes():
    """The single-pass form takes D3Q27 grids with x a multiple of 32 nodes and
    y of 16, and holds two population arrays."""
    base = serve.make_trace(1, seed=0)[0]
    fits = {n: dataclasses.replace(base, n=n).single_pass_fits
            for n in [(32, 32, 32), (48, 48, 48), (64, 32, 64), (96, 96, 96), (128, 128, 128), (64, 40, 64)]}
    assert fits == {(32, 32, 32): True, (48, 48, 48): False, (64, 32, 64): True, (96, 96, 96): True,
                    (128, 128, 128): True, (64, 40, 64): False}
    r = dataclasses.replace(base, n=(64, 64, 64), storage=elbm.F16_SHIFT)
    pop = 27 * 64 ** 3 * 2 + 16
    assert r.device_bytes() == pop + 3 * 64 ** 3 * 4
    assert r.device_bytes(single_pass=True) == 2 * pop + 3 * 64 ** 3 * 4


@pytest.mark.parametrize("policy", ["fifo", "srpt"])
def test_kernel_forms_per_grid_and_batches_never_mix_them(monkeypatch, policy):
    """"auto" runs the grids the single pass takes in it (kernel 3) and the rest
    in the two-pass form (kernel 1), in separate batches; "two-pass" runs every
    request in the two-pass form; plain mode chooses as "auto" does."""
    trace = serve.make_trace(40, seed=11, steps=200, rate=200.0)
    server, summary, world = serve_fake(monkeypatch, trace, budget=1 << 40, policy=policy, floor=1 << 20)
    assert summary["served"] == 40
    assert all(world.kernels[r.rid] == (3 if r.single_pass_fits else 1) for r in trace)
    assert {1, 3} <= set(world.kernels.values())
    assert world.batch_kernels and all(len(k) == 1 for k in world.batch_kernels)
    _, summary2, world2 = serve_fake(monkeypatch, trace, budget=1 << 40, policy=policy, kernels="two-pass")
    assert summary2["served"] == 40 and set(world2.kernels.values()) == {1}
    _, _, world3 = serve_fake(monkeypatch, trace[:6], budget=1 << 40, mode="plain")
    assert all(world3.kernels[r.rid] == (3 if r.single_pass_fits else 1) for r in trace[:6])


def test_unknown_kernel_choice_is_rejected():
    with pytest.raises(ValueError):
        serve.Server(kernels="single")
