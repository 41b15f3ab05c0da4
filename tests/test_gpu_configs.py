"""The benchmark configurations as GPU parity cases, at their full sizes where
the oracle can follow a few steps, and the shear-wave viscosity measurement
on the GPU (Sec. III.A).

Tolerances as everywhere: relative L-infinity on u of 1e-5 (FP32 storage) and
2e-3 (FP16 shifted storage)."""
import numpy as np
import pytest
import torch

import oracle
from flowdiag import decay_rate, mode_amplitude
from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu

TOL = {elbm.F32: 1e-5, elbm.F32_SHIFT: 1e-5, elbm.F16_SHIFT: 2e-3}


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()


def gpu_nu(n, lam, k_dir, s_dir, U, T, nu, steps=1000, every=50, t_min=100):
    """Viscosity from the decay of the shear mode's Fourier amplitude, both
    measured on the GPU (FP64 mode projection, elbm_mode_sums), fitted on the
    host (reading c8: least squares on ln A after step t_min)."""
    D = len(n)
    rho, u, k, s = inputs.shear_wave(n, lam, k_dir, s_dir, 1e-3, U)
    ts, A = [], []
    with elbm.Solver(elbm.D2Q9 if D == 2 else elbm.D3Q27, n, stretch=lam, T=T, nu=nu,
                     storage=elbm.F32_SHIFT) as s_:
        s_.init(rho, u)
        for t in range(0, steps + 1, every):
            if t:
                s_.step(every)
            ts.append(t)
            A.append(s_.mode_amplitude(k, s))
    return decay_rate(ts, A, t_min) / (k @ k)


@pytest.mark.parametrize("lattice,n,lam,kd,sd", [(elbm.D2Q9, (64, 128), (2.0, 1.0), (1, 1), (-1, 1)),
                                                  (elbm.D3Q27, (32, 16, 24), (1.0, 1.5, 2.0), (1, 0, 1), (-1, 0, 1))])
def test_mode_projection_on_gpu_matches_numpy(lattice, n, lam, kd, sd):
    """elbm_mode_sums (FP64 on the GPU) against the numpy projection of the
    velocity read back from the GPU, on a stretched lattice."""
    rho, u, k, s = inputs.shear_wave(n, lam, kd, sd, 1e-2, 0.1)
    with elbm.Solver(lattice, n, stretch=lam, T=0.4, nu=0.02, storage=elbm.F32_SHIFT) as sv:
        sv.init(rho, u)
        sv.step(37)
        got = sv.mode_amplitude(k, s)
        _, ug = sv.moments()
    want = mode_amplitude(ug.astype(np.float64), k, s, lam)
    assert abs(got - want) <= 1e-9 * want + 1e-15


def test_shear_wave_viscosity_on_gpu():
    """D2Q9 64 x 64, T = 1/3, u_x = 0.1, u_y = 1e-3 sin(2 pi x / 64), nu = 0.01,
    1000 steps: the decay gives nu = (1/omega - 1/2) T (Eq. nu) within 1 %."""
    nu = 0.01
    got = gpu_nu((64, 64), (1.0, 1.0), (1, 0), (0, 1), 0.1, 1 / 3, nu)
    assert abs(got - nu) / nu < 1e-2


def oracle_nu(n, lam, k_dir, s_dir, U, T, nu, steps=1000, every=50, t_min=100):
    rho, u, k, s = inputs.shear_wave(n, lam, k_dir, s_dir, 1e-3, U)
    o = oracle.Oracle(len(n), n, lam=tuple(lam) + (1.0,) * (3 - len(lam)), T=T, nu=nu)
    o.init(rho, u)
    ts, A = [], []
    for t in range(0, steps + 1, every):
        if t:
            o.step(every)
        ts.append(t)
        A.append(mode_amplitude(o.macros()[1], k, s, lam))
    return decay_rate(ts, A, t_min) / (k @ k)


@pytest.mark.parametrize("T", [1 / 3, 0.5])
def test_viscosity_independent_of_advection_on_gpu(T):
    """Galilean invariance (Figs. 1-3): a rotated wave on a lam_x = 2 lattice
    decays at the same rate for U = 0, 0.1 and 0.2 (spread below 1 % of nu),
    and the GPU's fitted viscosity matches the oracle's within 1e-3."""
    nu, n, lam = 0.01, (64, 128), (2.0, 1.0)
    vals = [gpu_nu(n, lam, (1, 1), (-1, 1), U, T, nu) for U in (0.0, 0.1, 0.2)]
    assert (max(vals) - min(vals)) / nu < 1e-2, vals
    ref = oracle_nu(n, lam, (1, 1), (-1, 1), 0.2, T, nu)
    assert abs(vals[2] - ref) / ref < 1e-3, (vals[2], ref)


@pytest.mark.parametrize("n,lam", [((1024, 1024), (1.0, 1.0)), ((1024, 512), (1.0, 2.0))])
@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT])
@pytest.mark.parametrize("kernel", [0, 1])
def test_double_shear_layer_full_size(n, lam, storage, kernel):
    """D2Q9 double shear layer at full size, cubic and stretched (dy/dx = 2),
    T = 0.5, U = 0.2, Re = 3e4 (nu = U L / Re, L = 1024), 21 steps (both
    parities), every node against the oracle; the automatic form (the row-march
    single pass the benchmark times) and the two-pass form."""
    U, Re, T, steps = 0.2, 3e4, 0.5, 21
    nu = U * 1024 / Re
    rho, u = inputs.double_shear_layer(n, U=U)
    with elbm.Solver(elbm.D2Q9, n, stretch=lam, T=T, nu=nu, storage=storage, kernel=kernel) as s:
        assert s.kernel_form == ((3, 4) if kernel == 0 else (1, 0))
        s.init(rho, u)
        s.step(steps)
        _, ug = s.moments()
    o = oracle.Oracle(2, n, lam=lam + (1.0,), T=T, nu=nu)
    o.init(rho, u)
    o.step(steps)
    _, uo = o.macros()
    assert rel_linf(ug, uo) <= TOL[storage]


def test_channel_full_size_two_steps():
    """D3Q27 turbulent channel at full size: 512 x 128 x 256, lam = (2, 1, 2),
    walls in y, Re_tau = 180 (H = 64 nodes, u_tau = 0.1/(ln(180)/0.41 + 5.5),
    nu = u_tau H / 180, g = u_tau^2 / H), T = 0.55, laminar profile with a 5 %
    perturbation, FP32; every node against the oracle after two steps."""
    n, lam, T = (512, 128, 256), (2.0, 1.0, 2.0), 0.55
    u_tau = 0.1 / (np.log(180.0) / 0.41 + 5.5)
    nu, g = u_tau * 64 / 180.0, u_tau ** 2 / 64
    rho, u = inputs.channel(n, lam, u_center=0.1, perturbation=0.05, seed=0)
    o = oracle.Oracle(3, n, lam=lam, T=T, nu=nu, walls_y=True, g=(g, 0.0, 0.0))
    o.init(rho, u)
    o.step(2)
    _, uo = o.macros()
    for kernel in (1, 3):  # two-pass and the TMEM single pass (bench.py times the latter)
        with elbm.Solver(elbm.D3Q27, n, stretch=lam, T=T, nu=nu, storage=elbm.F32, walls_y=True,
                         force=(g, 0.0, 0.0), kernel=kernel) as s:
            s.init(rho, u)
            s.step(2)
            _, ug = s.moments()
        assert rel_linf(ug, uo) <= 1e-5, kernel


@pytest.mark.parametrize("storage", [elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_turbulence_at_T_half_single_pass(storage):
    """The turbulence configuration at T = 0.5 in the single-pass form (the
    benchmark's), on a 64 x 32 x 32 box, 150 steps."""
    n = (64, 32, 32)
    rho, u = inputs.isotropic_turbulence(n, seed=3, k0=4.0, u_rms=0.08)
    with elbm.Solver(elbm.D3Q27, n, T=0.5, nu=0.0233, storage=storage, kernel=3) as s:
        s.init(rho, u)
        s.step(150)
        _, ug = s.moments()
    o = oracle.Oracle(3, n, T=0.5, nu=0.0233)
    o.init(rho, u)
    o.step(150)
    _, uo = o.macros()
    assert rel_linf(ug, uo) <= TOL[storage]
