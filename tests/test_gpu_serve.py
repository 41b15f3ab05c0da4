"""Served mix on the GPU: every request's result is the same alone (plain
mode) and in the continuously batched mix, bit for bit, and matches the FP64
oracle within the stated tolerances (FP32 1e-5, FP16 2e-3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_04550_gb300 import elbm, serve

pytestmark = pytest.mark.gpu


def small_trace():
    trace = serve.make_trace(10, rate=500.0, seed=11, steps=60, sizes=(16, 24, 32))
    for r in trace:
        if r.n == (64, 32, 64):
            r.n = (24, 12, 24)
    return trace


@pytest.mark.parametrize("policy", ["fifo", "srpt"])
def test_mix_equals_alone_and_oracle(policy):
    """With either policy (the "srpt" one changes the batch membership from
    chunk to chunk) every request ends bit-identical to its solo run."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    trace = small_trace()
    stream = torch.cuda.current_stream()
    mixed = serve.Server(hbm_budget=3 * max(r.device_bytes() for r in trace), chunk_steps=20, stream=stream,
                         policy=policy, step_floor_nodes=2 * 24 ** 3)
    s_mix = mixed.run(trace, mode="batched")
    alone = serve.Server(stream=stream)
    s_alone = alone.run(trace, mode="plain")
    assert s_mix["served"] == s_alone["served"] == len(trace)
    for r in trace:
        assert np.array_equal(mixed.results[r.rid]["u"], alone.results[r.rid]["u"]), r.rid
    for r in trace[:3]:
        o = oracle.Oracle(3, r.n, lam=r.stretch, T=r.T, nu=r.nu)
        rho, u = serve.initial_field(r)
        o.init(rho, u)
        o.step(r.steps)
        uo = o.macros()[1]
        err = np.abs(mixed.results[r.rid]["u"] - uo).max() / np.abs(uo).max()
        assert err <= (1e-5 if r.storage == elbm.F32_SHIFT else 2e-3), (r.rid, r.storage, err)
