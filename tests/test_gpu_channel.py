"""GPU parity of the wall-bounded and forced step (the channel setup of
Sec. III.E: half-way bounce-back walls in y, the anomaly's ghost rule next to
a wall, exact-difference body force) against the FP64 oracle.

Same tolerances as the periodic parity tests: relative L-infinity on u of
1e-5 for FP32 storage and 2e-3 for FP16 shifted storage."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu

TOL = {elbm.F32: 1e-5, elbm.F32_SHIFT: 1e-5, elbm.F16_SHIFT: 2e-3, elbm.BF16_SHIFT: 2e-2}


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()


def run_pair(lattice, n, lam, T, nu, rho, u, steps, storage=elbm.F32_SHIFT, walls=True, force=(0, 0, 0),
             equilibrium=0, kernel=1, u_ref=None):
    D = 2 if lattice == elbm.D2Q9 else 3
    lam3 = tuple(lam) + (1.0,) * (3 - len(lam))
    with elbm.Solver(lattice, n, stretch=lam, T=T, nu=nu, storage=storage, kernel=kernel,
                     equilibrium=equilibrium, walls_y=walls, force=force[:D], u_ref=u_ref) as s:
        s.init(rho, u)
        s.step(steps)
        s.sync()
        rg, ug = s.moments()
    mode = {0: oracle.EXTENDED, 1: oracle.PRODUCT, 2: oracle.SECOND_ORDER}[equilibrium]
    o = oracle.Oracle(D, n, lam=lam3, T=T, nu=nu, mode=mode, walls_y=walls, g=tuple(force) + (0.0,) * (3 - len(force)))
    o.init(rho, u)
    o.step(steps)
    ro, uo = o.macros()
    return (rg, ug), (ro, uo)


CHANNEL_N, CHANNEL_LAM, CHANNEL_T = (24, 16, 20), (2.0, 1.0, 2.0), 0.55


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
@pytest.mark.parametrize("steps", [200, 201])
def test_d3q27_channel_walls_and_force(storage, steps):
    """Channel lattice lam = (2, 1, 2), T = 0.55, laminar profile plus a 5 %
    seeded perturbation, walls in y and a body force along x; an odd step
    count ends on the other streaming parity."""
    rho, u = inputs.channel(CHANNEL_N, CHANNEL_LAM, u_center=0.05, perturbation=0.05, seed=0)
    (rg, ug), (ro, uo) = run_pair(elbm.D3Q27, CHANNEL_N, CHANNEL_LAM, CHANNEL_T, 0.02, rho, u, steps, storage,
                                  force=(2e-5, 0.0, 0.0),
                                  u_ref=(0.0333, 0.0, 0.0) if storage == elbm.F16_SHIFT else None)
    assert rel_linf(ug, uo) <= TOL[storage]
    # the wall-normal and spanwise components alone (their size, ~3e-4 here, is
    # near the rounding floor of unshifted FP32 populations, so shifted only)
    if storage != elbm.F32:
        assert rel_linf(ug[1:], uo[1:]) <= 20 * TOL[storage]
    assert np.abs(rg - ro).max() <= 10 * TOL[storage]


@pytest.mark.parametrize("lam", [(1.0, 1.0), (2.0, 1.0), (1.0, 1.5)])
def test_d2q9_poiseuille_start_up(lam):
    """Start-up of channel flow from rest under a constant force, both walls
    in play and every node's velocity changing each step."""
    n = (4, 32)
    rho, u = inputs.uniform(n, (0.0, 0.0))
    (_, ug), (_, uo) = run_pair(elbm.D2Q9, n, lam, 0.5 if lam != (1.0, 1.0) else 1 / 3, 0.1, rho, u, 3001,
                                force=(1e-5, 0.0))
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("equilibrium", [0, 1, 2])
def test_d2q9_walls_without_force(equilibrium):
    """Walls alone with each equilibrium: a random flow decaying between the
    walls (the ghost rule acts through u_y at the wall-adjacent nodes)."""
    n, lam = (24, 20), (2.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(5))
    rho = 1.0 + 0.01 * rng.standard_normal((n[1], n[0]))
    u = 0.05 * rng.standard_normal((2, n[1], n[0]))
    (_, ug), (_, uo) = run_pair(elbm.D2Q9, n, lam, 0.55, 0.05, rho, u, 301, equilibrium=equilibrium)
    assert rel_linf(ug, uo) <= 1e-5


def test_d3q27_force_without_walls():
    """Body force on a periodic grid with a turbulent field, force along a
    diagonal."""
    n, lam = (16, 12, 20), (1.0, 1.5, 2.0)
    rho, u = inputs.isotropic_turbulence(n, k0=2, u_rms=0.05, seed=2)
    (_, ug), (_, uo) = run_pair(elbm.D3Q27, n, lam, 0.5, 0.03, rho, u, 150, walls=False,
                                force=(1e-4, -2e-4, 5e-5))
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT])
def test_uniform_flow_accelerates_by_g_per_step(storage):
    """Closed form: under the exact-difference force a uniform flow stays
    uniform and its reported velocity after n steps is u0 + (n + 1/2) g."""
    n, lam = (8, 6, 10), (1.5, 1.0, 2.0)
    g = np.array([1e-4, -2e-4, 3e-4])
    u0 = np.array([0.05, -0.02, 0.03])
    rho, u = inputs.uniform(n, tuple(u0))
    with elbm.Solver(elbm.D3Q27, n, stretch=lam, T=0.5, nu=0.05, storage=storage, force=tuple(g)) as s:
        s.init(rho, u)
        s.step(100)
        s.sync()
        _, ug = s.moments()
    want = u0 + 100.5 * g
    for a in range(3):
        assert np.abs(ug[a] - want[a]).max() <= 1e-5 * np.abs(want).max()


def test_wall_gradient_reduction():
    """elbm_reduce with walls: the wall-normal gradient of u_x summed over
    both walls, and y-differences with the no-slip ghost, against numpy on
    the moments read back from the GPU."""
    n, lam = (16, 12, 10), (2.0, 1.0, 2.0)
    rho, u = inputs.channel(n, lam, u_center=0.05, perturbation=0.05, seed=4)
    with elbm.Solver(elbm.D3Q27, n, stretch=lam, T=0.55, nu=0.02, storage=elbm.F32_SHIFT, walls_y=True,
                     force=(1e-5, 0, 0)) as s:
        s.init(rho, u)
        s.step(37)
        red = s.reduce()
        _, ug = s.moments()
    uu = ug.astype(np.float64)
    ux = uu[0]  # (nz, ny, nx)
    grad = (9 * ux[:, 0, :] - ux[:, 1, :]) / (3 * lam[1]) + (9 * ux[:, -1, :] - ux[:, -2, :]) / (3 * lam[1])
    assert np.isclose(red["wall_dudn"], grad.sum(), rtol=1e-5)
    # vorticity with the ghost rule in y
    pad = np.concatenate([-uu[:, :, :1], uu, -uu[:, :, -1:]], axis=2)
    dy = lambda f: (pad[f][:, 2:, :] - pad[f][:, :-2, :]) / (2 * lam[1])
    dx = lambda f: (np.roll(uu[f], -1, 2) - np.roll(uu[f], 1, 2)) / (2 * lam[0])
    dz = lambda f: (np.roll(uu[f], -1, 0) - np.roll(uu[f], 1, 0)) / (2 * lam[2])
    curl2 = (dy(2) - dz(1)) ** 2 + (dz(0) - dx(2)) ** 2 + (dx(1) - dy(0)) ** 2
    assert np.isclose(red["curl2"], curl2.sum(), rtol=1e-5)
    # without walls the entry is zero
    with elbm.Solver(elbm.D3Q27, n, stretch=lam, T=0.55, nu=0.02, storage=elbm.F32_SHIFT) as s:
        s.init(rho, u)
        assert s.reduce()["wall_dudn"] == 0.0


def test_requested_kernel_forms_fall_back_bitwise():
    """On a grid the TMEM single pass does not take (nx = 24), walls and force
    run in the two-pass form whatever form is requested; bit-identical."""
    rho, u = inputs.channel(CHANNEL_N, CHANNEL_LAM, u_center=0.05, perturbation=0.05, seed=1)
    out = []
    for kernel in (1, 2, 3):
        with elbm.Solver(elbm.D3Q27, CHANNEL_N, stretch=CHANNEL_LAM, T=CHANNEL_T, nu=0.02, storage=elbm.F32_SHIFT,
                         kernel=kernel, walls_y=True, force=(1e-5, 0, 0)) as s:
            s.init(rho, u)
            s.step(11)
            out.append(s.get_populations())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_batch_rejects_walls_and_force():
    n = (16, 16, 16)
    rho, u = inputs.uniform(n, (0.0, 0.0, 0.0))
    a = elbm.Solver(elbm.D3Q27, n, T=0.4, nu=0.02, storage=elbm.F32_SHIFT)
    b = elbm.Solver(elbm.D3Q27, n, T=0.4, nu=0.02, storage=elbm.F32_SHIFT, walls_y=True)
    c = elbm.Solver(elbm.D3Q27, n, T=0.4, nu=0.02, storage=elbm.F32_SHIFT, force=(1e-5, 0, 0))
    for s in (a, b, c):
        s.init(rho, u)
    for bad in (b, c):
        with pytest.raises(elbm.ElbmError):
            elbm.Batch([a, bad])
    for s in (a, b, c):
        s.close()


TMEM_N = (64, 32, 20)


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
@pytest.mark.parametrize("steps", [1, 2, 7])
@pytest.mark.parametrize("force", [(2e-5, 0, 0), (2e-5, -1e-5, 3e-5)])
def test_single_pass_walls_and_force_bitwise(storage, steps, force):
    """The TMEM single pass with walls and body force (nx a multiple of 32,
    ny of 16) against the two-pass form: bit-identical populations, rest
    storage baseline, both parities; a force along x alone (the lighter force
    increment of the single pass) and along all three axes."""
    rho, u = inputs.channel(TMEM_N, CHANNEL_LAM, u_center=0.05, perturbation=0.05, seed=3)
    out = []
    for kernel in (1, 3):
        with elbm.Solver(elbm.D3Q27, TMEM_N, stretch=CHANNEL_LAM, T=CHANNEL_T, nu=0.02, storage=storage,
                         kernel=kernel, walls_y=True, force=force) as s:
            s.init(rho, u)
            s.step(steps)
            out.append(s.get_populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("storage,u_ref", [(elbm.F32_SHIFT, None), (elbm.F16_SHIFT, (0.0333, 0.0, 0.0))])
def test_single_pass_channel_against_oracle(storage, u_ref):
    """The TMEM single pass with walls and force against the oracle after 201
    steps; with FP16 storage at a moving baseline (bounced populations are
    rebased when they are written, where the two-pass form rebases them when
    read, so the two forms differ by FP16 rounding there)."""
    rho, u = inputs.channel(TMEM_N, CHANNEL_LAM, u_center=0.05, perturbation=0.05, seed=0)
    (_, ug), (_, uo) = run_pair(elbm.D3Q27, TMEM_N, CHANNEL_LAM, CHANNEL_T, 0.02, rho, u, 201, storage,
                                force=(2e-5, 0.0, 0.0), kernel=3, u_ref=u_ref)
    assert rel_linf(ug, uo) <= TOL[storage]
