"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (stated for the path): relative L-infinity on the velocity,
max|u_gpu - u_oracle| / max|u_oracle|, <= 1e-5 for FP32 storage and <= 2e-3
for FP16 shifted storage after up to 1000 steps.  BF16 shifted storage keeps
8 mantissa bits and is held to a looser 2e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu

TOL = {elbm.F32: 1e-5, elbm.F32_SHIFT: 1e-5, elbm.F16_SHIFT: 2e-3, elbm.BF16_SHIFT: 2e-2}


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def run_gpu(lattice, n, lam, T, nu, rho, u, steps, storage=elbm.F32, kernel=1, equilibrium=0,
            chunked=None, u_ref=None):
    with elbm.Solver(lattice, n, stretch=lam, T=T, nu=nu, storage=storage, kernel=kernel,
                     equilibrium=equilibrium, u_ref=u_ref) as s:
        s.init(rho, u)
        if chunked:
            for k in chunked:
                s.step(k)
        else:
            s.step(steps)
        s.sync()
        return s.moments()


def run_oracle(D, n, lam, T, nu, rho, u, steps, mode=oracle.EXTENDED):
    o = oracle.Oracle(D, n, lam=tuple(lam) + (1.0,) * (3 - len(lam)), T=T, nu=nu, mode=mode)
    o.init(rho, u)
    o.step(steps)
    return o.macros()


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()


# ------------------------------------------------------------ D2Q9 cases
@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT])
@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_d2q9_shear_wave_64_1000_steps(storage, kernel):
    """D2Q9 advected shear wave, 64x64 periodic, T = 1/3, u_x = 0.1,
    u_y = 1e-3 sin(2 pi x / 64), nu = 0.01, 1000 steps."""
    n = (64, 64)
    rho, u, _, _ = inputs.shear_wave(n, (1.0, 1.0), (1, 0), (0, 1), 1e-3, 0.1)
    _, ug = run_gpu(elbm.D2Q9, n, (1.0, 1.0), 1 / 3, 0.01, rho, u, 1000, storage, kernel)
    _, uo = run_oracle(2, n, (1.0, 1.0), 1 / 3, 0.01, rho, u, 1000)
    assert rel_linf(ug, uo) <= TOL[storage]
    # the perturbation alone (uniform advection cannot hide an error)
    assert rel_linf(ug[1], uo[1]) <= 20 * TOL[storage]


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("T", [1 / 3, 0.5])
def test_d2q9_rotated_stretched_correction_active(kernel, T):
    """Rotated wave on a lam_x = 2 lattice: the central-difference correction
    is large here (Fig. 3)."""
    n, lam = (32, 64), (2.0, 1.0)
    rho, u, _, _ = inputs.shear_wave(n, lam, (1, 1), (-1, 1), 1e-3, 0.1)
    _, ug = run_gpu(elbm.D2Q9, n, lam, T, 0.01, rho, u, 1000, elbm.F32_SHIFT, kernel)
    _, uo = run_oracle(2, n, lam, T, 0.01, rho, u, 1000)
    assert rel_linf(ug, uo) <= 1e-5


def test_d2q9_double_shear_layer_128():
    """Double shear layer (Sec. III.C) at 128x64, lam_y = 2, T = 0.5, 300 steps."""
    n, lam = (128, 64), (1.0, 2.0)
    rho, u = inputs.double_shear_layer(n, U=0.1)
    _, ug = run_gpu(elbm.D2Q9, n, lam, 0.5, 0.002, rho, u, 300, elbm.F32_SHIFT, 2)
    _, uo = run_oracle(2, n, lam, 0.5, 0.002, rho, u, 300)
    assert rel_linf(ug, uo) <= 1e-5


def test_d2q9_product_form_mode():
    """Correction switched off: the product-form equilibrium of Eq. 27eq."""
    n, lam = (32, 64), (2.0, 1.0)
    rho, u, _, _ = inputs.shear_wave(n, lam, (1, 1), (-1, 1), 1e-3, 0.1)
    _, ug = run_gpu(elbm.D2Q9, n, lam, 1 / 3, 0.01, rho, u, 500, elbm.F32_SHIFT, 1, equilibrium=1)
    _, uo = run_oracle(2, n, lam, 1 / 3, 0.01, rho, u, 500, mode=oracle.PRODUCT)
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("lattice,n,lam", [(elbm.D2Q9, (64, 64), (1.0, 1.0)),
                                           (elbm.D3Q27, (24, 16, 20), (1.0, 1.5, 2.0))])
def test_second_order_equilibrium_mode(lattice, n, lam):
    """The conventional second-order equilibrium (Sec. III preamble) against
    the oracle's, on an advected rotated wave."""
    D = 2 if lattice == elbm.D2Q9 else 3
    kd, sd = ((1, 1), (-1, 1)) if D == 2 else ((1, 0, 1), (-1, 0, 1))
    rho, u, _, _ = inputs.shear_wave(n, lam, kd, sd, 1e-2, 0.1)
    _, ug = run_gpu(lattice, n, lam, 0.4, 0.02, rho, u, 300, elbm.F32_SHIFT, 1, equilibrium=2)
    _, uo = run_oracle(D, n, lam, 0.4, 0.02, rho, u, 300, mode=oracle.SECOND_ORDER)
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("kernel", [1, 3])
@pytest.mark.parametrize("storage", [elbm.F16_SHIFT, elbm.BF16_SHIFT])
def test_d2q9_half_storage_advected(storage, kernel):
    """Half-precision storage of an advected rotated wave (U = 0.1, amplitude
    1e-2), with the storage baseline at the field's mean velocity."""
    n = (64, 64)
    rho, u, _, _ = inputs.shear_wave(n, (1.0, 1.0), (1, 1), (-1, 1), 1e-2, 0.1)
    _, ug = run_gpu(elbm.D2Q9, n, (1.0, 1.0), 1 / 3, 0.01, rho, u, 1000, storage, kernel, u_ref="mean")
    _, uo = run_oracle(2, n, (1.0, 1.0), 1 / 3, 0.01, rho, u, 1000)
    assert rel_linf(ug, uo) <= TOL[storage]


def test_baseline_velocity_mean_is_detected_and_harmless_in_fp32():
    n = (64, 64)
    rho, u, _, _ = inputs.shear_wave(n, (1.0, 1.0), (1, 1), (-1, 1), 1e-2, 0.1)
    with elbm.Solver(elbm.D2Q9, n, T=1 / 3, nu=0.01, storage=elbm.F32_SHIFT, u_ref="mean") as s:
        s.init(rho, u)
        np.testing.assert_allclose(s.u_ref, [0.1 / np.sqrt(2)] * 2, rtol=1e-6)
        s.step(1000)
        _, ug = s.moments()
    _, uo = run_oracle(2, n, (1.0, 1.0), 1 / 3, 0.01, rho, u, 1000)
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("storage", [elbm.F16_SHIFT, elbm.BF16_SHIFT])
def test_d3q27_half_storage_turbulence(storage):
    """Zero-mean turbulence (rest baseline, f_i - w_i rho0): 48^3, u_rms = 0.08, 200 steps."""
    n = (48, 48, 48)
    rho, u = inputs.isotropic_turbulence(n, seed=6, k0=4.0, u_rms=0.08)
    _, ug = run_gpu(elbm.D3Q27, n, (1.0, 1.0, 1.0), 0.5, 0.02, rho, u, 200, storage, 2)
    _, uo = run_oracle(3, n, (1.0, 1.0, 1.0), 0.5, 0.02, rho, u, 200)
    assert rel_linf(ug, uo) <= TOL[storage]


# ----------------------------------------------------------- D3Q27 cases
@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
def test_d3q27_turbulence_ragged_stretched(kernel):
    """Seeded solenoidal field on a ragged 37x20x23 grid, lam = (1, 1.5, 2), T = 0.5."""
    n, lam = (37, 20, 23), (1.0, 1.5, 2.0)
    rho, u = inputs.isotropic_turbulence(n, seed=1, k0=3.0, u_rms=0.05)
    _, ug = run_gpu(elbm.D3Q27, n, lam, 0.5, 0.02, rho, u, 200, elbm.F32_SHIFT, kernel)
    _, uo = run_oracle(3, n, lam, 0.5, 0.02, rho, u, 200)
    assert rel_linf(ug, uo) <= 1e-5


@pytest.mark.parametrize("storage", [elbm.F32, elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_d3q27_shear_wave_1000_steps(storage):
    n, lam = (32, 8, 16), (1.0, 1.0, 2.0)
    rho, u, _, _ = inputs.shear_wave(n, lam, (1, 0, 1), (-1, 0, 1), 1e-2, 0.1)
    _, ug = run_gpu(elbm.D3Q27, n, lam, 1 / 3, 0.02, rho, u, 1000, storage, 2)
    _, uo = run_oracle(3, n, lam, 1 / 3, 0.02, rho, u, 1000)
    assert rel_linf(ug, uo) <= TOL[storage]


def test_d3q27_minimum_grid():
    """Smallest grid the central difference allows: 3x3x3."""
    n = (3, 3, 3)
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.01 * rng.standard_normal((3, 3, 3))
    u = 0.03 * rng.standard_normal((3, 3, 3, 3))
    _, ug = run_gpu(elbm.D3Q27, n, (1.0, 1.0, 1.0), 1 / 3, 0.05, rho, u, 50, elbm.F32_SHIFT, 1)
    _, uo = run_oracle(3, n, (1.0, 1.0, 1.0), 1 / 3, 0.05, rho, u, 50)
    assert rel_linf(ug, uo) <= 1e-5


# ---------------------------------------------------- kernels and state
@pytest.mark.parametrize("lattice,n", [(elbm.D3Q27, (64, 64, 48)), (elbm.D3Q27, (40, 24, 3)),
                                       (elbm.D3Q27, (5, 3, 70)), (elbm.D3Q27, (70, 20, 33)),
                                       (elbm.D3Q27, (64, 8, 3)), (elbm.D3Q27, (32, 16, 35)),
                                       (elbm.D2Q9, (300, 700)), (elbm.D2Q9, (33, 5))])
@pytest.mark.parametrize("storage", [elbm.F32, elbm.F16_SHIFT, elbm.F32_SHIFT, elbm.BF16_SHIFT])
@pytest.mark.parametrize("lam,T", [((1.0, 2.0, 1.0), 0.5), ((1.5, 1.0, 2.0), 0.45)])
def test_kernel_forms_agree_bitwise(lattice, n, storage, lam, T):
    """The two-pass, graph-pipelined, single-pass and (D3Q27) fused in-place
    forms evaluate the same per-node arithmetic, so the states agree bit for
    bit, across launches of several steps and both streaming parities.  A
    spacing of 1.5 (no power of two) and T = 0.45 leave no product of the
    lattice constants exact, so a rounding step taken in another order shows."""
    D = 2 if lattice == elbm.D2Q9 else 3
    if D == 3:
        rho, u = inputs.isotropic_turbulence(n, seed=2, k0=3.0, u_rms=0.05)
    else:
        rho, u = inputs.double_shear_layer(n, U=0.1)
    lam = lam[:D]
    outs = []
    for kernel in ((1, 2, 3, 4) if D == 3 else (1, 2, 3)):
        with elbm.Solver(lattice, n, stretch=lam, T=T, nu=0.01, storage=storage, kernel=kernel) as s:
            s.init(rho, u)
            for k in (1, 2, 4):
                s.step(k)
            outs.append(s.get_populations())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("lattice,n", [(elbm.D2Q9, (20, 12)), (elbm.D3Q27, (9, 7, 5))])
def test_populations_one_and_two_steps(lattice, n):
    """Populations after init (Eq. 27eq), one (even parity) and two (odd
    parity) steps against the oracle's, element by element."""
    D = 2 if lattice == elbm.D2Q9 else 3
    rng = np.random.default_rng(11)
    shape = tuple(n[::-1])
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((D,) + shape)
    lam = (1.5, 1.0, 2.0)[:D]
    o = oracle.Oracle(D, n, lam=tuple(lam) + (1.0,) * (3 - D), T=0.4, nu=0.03)
    o.init(rho, u)
    with elbm.Solver(lattice, n, stretch=lam, T=0.4, nu=0.03, storage=elbm.F32_SHIFT) as s:
        s.init(rho, u)
        for steps in (0, 1, 1):
            if steps:
                s.step(1)
                o.step(1)
            fg = s.get_populations().reshape(o.f.shape)
            assert np.abs(fg - o.f).max() <= 2e-7


def test_set_get_populations_roundtrip():
    n = (10, 9, 8)
    rng = np.random.default_rng(4)
    f = 0.03 + 0.01 * rng.random((27,) + tuple(n[::-1]))
    with elbm.Solver(elbm.D3Q27, n, T=1 / 3, nu=0.02, storage=elbm.F32) as s:
        s.set_populations(f)
        np.testing.assert_allclose(s.get_populations(), f, rtol=1e-7, atol=0)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_page_locked_host_fields_match_device_fields(dt):
    """elbm_init and elbm_moments with page-locked host buffers (read and
    written in place by the kernels), pageable host buffers (staged through
    device memory) and device buffers: the same populations and moments, bit
    for bit."""
    n = (40, 24, 18)
    rho, u = inputs.isotropic_turbulence(n, seed=6, k0=3.0, u_rms=0.05)
    rho_t, u_t = torch.as_tensor(rho, dtype=dt).contiguous(), torch.as_tensor(u, dtype=dt).contiguous()
    sources = {"device": (rho_t.cuda(), u_t.cuda()), "pinned": (rho_t.pin_memory(), u_t.pin_memory()),
               "pageable": (rho_t.numpy(), u_t.numpy())}
    f, mom = {}, {}
    for name, (r, v) in sources.items():
        with elbm.Solver(elbm.D3Q27, n, stretch=(1.0, 1.5, 1.0), T=0.4, nu=0.02, storage=elbm.F32_SHIFT) as s:
            s.init(r, v)
            s.step(3)
            f[name] = s.get_populations()
            if name == "device":
                ro, uo = torch.empty(r.shape, dtype=dt, device="cuda"), torch.empty(v.shape, dtype=dt, device="cuda")
            elif name == "pinned":
                ro, uo = torch.empty(r.shape, dtype=dt).pin_memory(), torch.empty(v.shape, dtype=dt).pin_memory()
            else:
                ro, uo = np.empty(r.shape, dtype=r.dtype), np.empty(v.shape, dtype=v.dtype)
            s.moments(ro, uo)
            mom[name] = [np.asarray(x.cpu()) if isinstance(x, torch.Tensor) else x for x in (ro, uo)]
    for name in ("pinned", "pageable"):
        assert np.array_equal(f[name], f["device"]), name
        for a, b in zip(mom[name], mom["device"]):
            assert np.array_equal(a, b), name


def test_reductions_fp64():
    """elbm_reduce against numpy on the moments read back from the GPU."""
    n, lam = (24, 20, 16), (1.0, 1.0, 2.0)
    rho, u = inputs.isotropic_turbulence(n, seed=3, k0=3.0, u_rms=0.05)
    with elbm.Solver(elbm.D3Q27, n, stretch=lam, T=0.5, nu=0.02, storage=elbm.F32_SHIFT) as s:
        s.init(rho, u)
        s.step(10)
        r, uu = s.moments(dtype=np.float32)
        red = s.reduce()
        f = s.get_populations()
    r = r.astype(np.float64)
    uu = uu.astype(np.float64)
    assert np.isclose(red["mass"], r.sum(), rtol=1e-9)
    assert np.isclose(red["rho_u2"], (r * (uu ** 2).sum(0)).sum(), rtol=1e-6)
    assert np.isclose(red["u2"], (uu ** 2).sum(), rtol=1e-6)
    dx = lambda a, ax, h: (np.roll(a, -1, ax) - np.roll(a, 1, ax)) / (2 * h)
    # axes of the (z, y, x) arrays: x -> 2, y -> 1, z -> 0
    wx = dx(uu[2], 1, lam[1]) - dx(uu[1], 0, lam[2])
    wy = dx(uu[0], 0, lam[2]) - dx(uu[2], 2, lam[0])
    wz = dx(uu[1], 2, lam[0]) - dx(uu[0], 1, lam[1])
    assert np.isclose(red["curl2"], (wx ** 2 + wy ** 2 + wz ** 2).sum(), rtol=1e-5)
    assert np.isclose(red["dxux2"], (dx(uu[0], 2, lam[0]) ** 2).sum(), rtol=1e-5)
    assert np.isclose(red["fmin"], f.min(), rtol=1e-6)
    assert red["nonfinite"] == 0
    assert np.isclose(red["umax"], np.sqrt((uu ** 2).sum(0)).max(), rtol=1e-6)


def test_mass_momentum_conserved_on_gpu():
    n = (32, 32, 32)
    rho, u = inputs.isotropic_turbulence(n, seed=4, k0=4.0, u_rms=0.08)
    with elbm.Solver(elbm.D3Q27, n, T=0.5, nu=0.02, storage=elbm.F32_SHIFT, kernel=2) as s:
        s.init(rho, u)
        r0 = s.reduce()
        s.step(500)
        r1 = s.reduce()
    assert abs(r1["mass"] - r0["mass"]) / r0["mass"] < 1e-6
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(r1[k] - r0[k]) / r0["mass"] < 1e-7


def test_full_size_benchmark_workload_two_steps():
    """The benchmark workload at full size (D3Q27 256^3 turbulence, T = 1/3,
    nu = 0.0233, FP32-shift storage), in the launch configurations bench.py
    times, against the oracle on every node after two steps (both parities);
    FP16 storage and the single-pass form on the same field."""
    n = (256, 256, 256)
    rho, u = inputs.isotropic_turbulence(n, seed=0, k0=4.0, u_rms=0.08)
    _, uo = run_oracle(3, n, (1.0, 1.0, 1.0), 1 / 3, 0.0233, rho, u, 2)
    for storage, kernel, tol in ((elbm.F32_SHIFT, 1, 1e-5), (elbm.F32_SHIFT, 3, 1e-5), (elbm.F16_SHIFT, 1, 2e-3)):
        _, ug = run_gpu(elbm.D3Q27, n, (1.0, 1.0, 1.0), 1 / 3, 0.0233, rho, u, 2, storage, kernel)
        assert rel_linf(ug, uo) <= tol, (storage, kernel)
