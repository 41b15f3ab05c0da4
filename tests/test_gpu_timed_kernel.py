"""The kernel the benchmark times -- the TMEM single pass (k_single_pass_tmem)
-- against the FP64 oracle over 1000 steps, and the automatic choice of the
kernel form (ELBM_OPT_KERNEL = 0).

Tolerances are the path's: relative L-infinity on the velocity,
max|u_gpu - u_oracle| / max|u_oracle|, <= 1e-5 for FP32 storage and <= 2e-3
for FP16 shifted storage after 1000 steps.  The same norm is also taken on the
perturbation u - u_mean (u_mean the oracle's mean velocity), so that the
uniform advection cannot hide an error; the rounding error of the step is set
by |u|, not by the perturbation (about a tenth of |u| here), so that check
allows 20 times the tolerance.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu

TOL = {elbm.F32: 1e-5, elbm.F32_SHIFT: 1e-5, elbm.F16_SHIFT: 2e-3}
STEPS = 1000


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()


# 2 x 2 tiles of 32 x 16 columns and one 32-plane segment; lam_z = 2; a wave
# along (1, 1, 1) periods with the advection along its wave vector, so the
# central-difference correction (Eq. Paastar1) is active along every axis
PERIODIC = dict(n=(64, 32, 32), lam=(1.0, 1.0, 2.0), T=1.0 / 3.0, nu=0.02)
# channel lattice of Sec. III.E on one tile column pair: walls in y, force in x
CHANNEL = dict(n=(32, 32, 16), lam=(2.0, 1.0, 2.0), T=0.55, nu=0.02, g=(2e-5, 0.0, 0.0))


def periodic_field():
    c = PERIODIC
    rho, u, _, _ = inputs.shear_wave(c["n"], c["lam"], (1, 1, 1), (-1, 0, 1), 1e-2, 0.1)
    return rho, u


def channel_field():
    c = CHANNEL
    return inputs.channel(c["n"], c["lam"], u_center=0.05, perturbation=0.05, seed=7)


@functools.lru_cache(maxsize=None)
def oracle_result(case):
    """Oracle velocity after STEPS steps (computed once per case)."""
    if case == "periodic":
        c = PERIODIC
        rho, u = periodic_field()
        o = oracle.Oracle(3, c["n"], lam=c["lam"], T=c["T"], nu=c["nu"])
    else:
        c = CHANNEL
        rho, u = channel_field()
        o = oracle.Oracle(3, c["n"], lam=c["lam"], T=c["T"], nu=c["nu"], walls_y=True, g=c["g"])
    o.init(rho, u)
    o.step(STEPS)
    return o.macros()[1]


def check(ug, uo, storage):
    err = rel_linf(ug, uo)
    mean = uo.reshape(3, -1).mean(axis=1).reshape(3, 1, 1, 1)
    err_pert = rel_linf(ug - mean, uo - mean)
    assert err <= TOL[storage], err
    assert err_pert <= 20 * TOL[storage], err_pert
    return err, err_pert


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_tmem_single_pass_1000_steps_periodic(storage):
    """Rotated advected shear wave (Sec. III.A) on a stretched periodic
    64 x 32 x 32 grid, 1000 steps of the TMEM single pass against the oracle."""
    c = PERIODIC
    rho, u = periodic_field()
    with elbm.Solver(elbm.D3Q27, c["n"], stretch=c["lam"], T=c["T"], nu=c["nu"], storage=storage, kernel=3,
                     u_ref="mean" if storage == elbm.F16_SHIFT else None) as s:
        assert s.kernel_form == (3, 1)
        s.init(rho, u)
        # launches of 1, 7, 100 and 892 steps: both array orders between launches
        for k in (1, 7, 100, STEPS - 108):
            s.step(k)
        _, ug = s.moments()
    check(ug, oracle_result("periodic"), storage)


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_fused_in_place_1000_steps_periodic(storage):
    """The fused in-place form (one array, AA pattern, one cooperative launch
    per step) on the same wave over 1000 steps against the oracle, launched in
    pieces of odd and even length (both AA parities between launches)."""
    c = PERIODIC
    rho, u = periodic_field()
    with elbm.Solver(elbm.D3Q27, c["n"], stretch=c["lam"], T=c["T"], nu=c["nu"], storage=storage, kernel=4,
                     u_ref="mean" if storage == elbm.F16_SHIFT else None) as s:
        assert s.kernel_form == (4, 0)
        s.init(rho, u)
        for k in (1, 7, 100, STEPS - 108):
            s.step(k)
        _, ug = s.moments()
    check(ug, oracle_result("periodic"), storage)


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_tmem_single_pass_1000_steps_walls_and_force(storage):
    """Channel lattice lam = (2, 1, 2), T = 0.55, half-way bounce-back walls in
    y and a body force along x (Sec. III.E), 1000 steps of the TMEM single pass
    (its walls-and-force instantiation) against the oracle."""
    c = CHANNEL
    rho, u = channel_field()
    with elbm.Solver(elbm.D3Q27, c["n"], stretch=c["lam"], T=c["T"], nu=c["nu"], storage=storage, kernel=3,
                     walls_y=True, force=c["g"],
                     u_ref=(0.0333, 0.0, 0.0) if storage == elbm.F16_SHIFT else None) as s:
        assert s.kernel_form == (3, 1)
        s.init(rho, u)
        s.step(STEPS)
        _, ug = s.moments()
    check(ug, oracle_result("channel"), storage)


@pytest.mark.parametrize("lattice,n,opts,want", [
    (elbm.D3Q27, (64, 32, 32), {}, (3, 1)),                       # TMEM geometry: single pass
    (elbm.D3Q27, (64, 32, 32), {"walls_y": True, "force": (1e-6, 0, 0)}, (3, 1)),
    (elbm.D3Q27, (64, 32, 32), {"equilibrium": 2}, (1, 0)),       # second order: two-pass only
    (elbm.D3Q27, (48, 48, 48), {}, (1, 0)),                       # x not a multiple of 32
    (elbm.D3Q27, (32, 8, 16), {}, (1, 0)),                        # y not a multiple of 16
    (elbm.D2Q9, (64, 64), {}, (3, 4)),                             # D2Q9: the row-march single pass
    (elbm.D2Q9, (33, 5), {}, (3, 4)),
    (elbm.D2Q9, (64, 64), {"walls_y": True}, (1, 0)),             # walls: two-pass (no D2Q9 single pass)
    (elbm.D2Q9, (64, 64), {"equilibrium": 2}, (1, 0)),
    (elbm.D3Q27, (32, 8, 16), {"kernel": 3}, (3, 2)),             # requested: 32 x 8 TMA tiles
    (elbm.D3Q27, (37, 20, 23), {"kernel": 3}, (3, 3)),            # requested: cp.async-staged
    (elbm.D3Q27, (37, 20, 23), {"kernel": 3, "walls_y": True}, (1, 0)),
    (elbm.D3Q27, (64, 32, 32), {"kernel": 2}, (2, 0)),
    (elbm.D3Q27, (48, 40, 36), {"kernel": 4}, (4, 0)),            # fused in place, ragged tiles
    (elbm.D3Q27, (64, 32, 32), {"kernel": 4, "walls_y": True}, (1, 0)),
    (elbm.D3Q27, (64, 32, 32), {"kernel": 4, "equilibrium": 2}, (1, 0)),
    (elbm.D2Q9, (64, 64), {"kernel": 4}, (1, 0)),
])
def test_automatic_kernel_form(lattice, n, opts, want):
    """ELBM_OPT_KERNEL = 0 (the default) takes the TMEM single pass where its
    geometry holds and the two-pass form elsewhere (the fused in-place form
    only when asked for); the form reported is the one the step runs."""
    with elbm.Solver(lattice, n, T=1 / 3, nu=0.02, storage=elbm.F32_SHIFT, **opts) as s:
        assert s.kernel_form == want


def test_automatic_form_memory_and_bits():
    """The automatic form holds the second array on a TMEM grid, releases it
    when an in-place form is requested, and gives the bits of the explicit
    single pass and of the two-pass form."""
    n = (64, 32, 32)
    rho, u = inputs.isotropic_turbulence(n, seed=9, k0=3.0, u_rms=0.05)
    pops = []
    for kernel in (0, 3, 1):
        with elbm.Solver(elbm.D3Q27, n, T=0.4, nu=0.02, storage=elbm.F32_SHIFT, kernel=kernel) as s:
            one = 27 * s.N * 4 + 16
            arrays = 1 if kernel == 1 else 2
            assert s.device_bytes == arrays * one + 3 * s.N * 4
            s.init(rho, u)
            for k in (1, 2, 4):
                s.step(k)
            pops.append(s.get_populations())
            if kernel == 0:
                s.set_option(elbm.OPT_KERNEL, 1)
                assert s.kernel_form == (1, 0)
                assert s.device_bytes == one + 3 * s.N * 4
                s.step(3)
                s.set_option(elbm.OPT_KERNEL, 0)
                assert s.kernel_form == (3, 1)
                s.step(3)
                s.sync()
    assert np.array_equal(pops[0], pops[1])
    assert np.array_equal(pops[0], pops[2])
