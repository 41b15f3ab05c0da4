"""Pins of the FP64 oracle's whole step against what the paper and the
mathematics fix: conservation (Eqs. density, momentum), fixed points, the
dormant correction of the axis-aligned shear wave (Sec. III.A), the viscosity
law of Eq. nu measured from shear-wave decay (Sec. III.A, Figs. 1-3),
Taylor-Green decay and forced channel flow."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2101_04550_gb300 import inputs
from flowdiag import decay_rate, mode_amplitude

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "shear_wave_setups.json")


def measure_nu(D, n, lam, k_dir, s_dir, U, T, nu, mode=oracle.EXTENDED, steps=1000, every=50,
               t_min=100):
    rho, u, k, s = inputs.shear_wave(n, lam[:D], k_dir, s_dir, 1e-3, U)
    o = oracle.Oracle(D, n, lam=tuple(lam) + (1.0,) * (3 - len(lam)), T=T, nu=nu, mode=mode)
    o.init(rho, u)
    ts, A = [], []
    for t in range(0, steps + 1, every):
        if t:
            o.step(every)
        ts.append(t)
        A.append(mode_amplitude(o.macros()[1], k, s, lam))
    return decay_rate(ts, A, t_min) / (k @ k)


def test_uniform_flow_is_a_fixed_point():
    """A uniform state has no gradients: the correction vanishes and f^eq is steady."""
    n = (6, 5, 4)
    rho, u = inputs.uniform(n, (0.1, -0.05, 0.2), rho0=1.02)
    o = oracle.Oracle(3, n, lam=(1.0, 1.5, 2.0), T=0.5, nu=0.02)
    o.init(rho, u)
    f0 = o.f.copy()
    o.step(20)
    np.testing.assert_allclose(o.f, f0, rtol=1e-13, atol=0)


@pytest.mark.parametrize("D,n,lam", [(2, (24, 20), (1.0, 2.0, 1.0)), (3, (10, 8, 12), (2.0, 1.0, 1.5))])
def test_mass_and_momentum_conserved(D, n, lam):
    """Eqs. density, momentum: the extended equilibrium conserves rho and rho u
    per cell, and streaming permutes populations, so a periodic run keeps the
    totals to round-off."""
    rng = np.random.default_rng(7)
    shape = tuple(n[::-1])
    rho = 1.0 + 0.02 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((D,) + shape)
    o = oracle.Oracle(D, n, lam=lam, T=0.45 if D == 3 else 0.4, nu=0.05)
    o.init(rho, u)
    r0, u0 = o.macros()
    m0, j0 = r0.sum(), (r0 * u0).reshape(D, -1).sum(1)
    o.step(100)
    r1, u1 = o.macros()
    assert abs(r1.sum() - m0) / m0 < 1e-13
    j1 = (r1 * u1).reshape(D, -1).sum(1)
    np.testing.assert_allclose(j1, j0, rtol=0, atol=1e-12 * m0)


def test_axis_aligned_correction_dormant():
    """Sec. III.A: for the axis-aligned shear wave both derivatives of the
    anomaly vanish, so extended and product-form equilibria give the same run."""
    g = json.load(open(GOLDEN))["axis_aligned"]
    n = (16, 64)
    rho, u, _, _ = inputs.shear_wave(n, (1.0, 1.0), (0, 1), (1, 0), g["a0"], 0.1, rho0=g["rho0"])
    outs = []
    for mode in (oracle.EXTENDED, oracle.PRODUCT):
        o = oracle.Oracle(2, n, T=1 / 3, nu=0.01, mode=mode)
        o.init(rho, u)
        o.step(200)
        outs.append(o.macros()[1])
    assert np.abs(outs[0] - outs[1]).max() <= 1e-15


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["viscosity_law"]["cases"])
def test_viscosity_axis_aligned(case):
    """Eq. nu through the decay of the axis-aligned wave at Ma = 0.1/sqrt(T)*sqrt(T)
    (advection 0.1 along the wave vector), T = 1/3 and 1/2 (Fig. 2)."""
    got = measure_nu(2, (64, 64), (1.0, 1.0), (1, 0), (0, 1), 0.1, case["T"], case["nu"])
    assert abs(got / case["nu"] - 1) < 0.005


@pytest.mark.parametrize("U", [0.0, 0.1, 0.2])
def test_viscosity_rotated_galilean_invariant(U):
    """Fig. 3: the pi/4-rotated wave recovers the imposed viscosity at every
    advection velocity with the extended equilibrium."""
    got = measure_nu(2, (64, 64), (1.0, 1.0), (1, 1), (-1, 1), U, 1 / 3, 0.01)
    assert abs(got / 0.01 - 1) < 0.003


def test_viscosity_rotated_product_form_drifts_with_velocity():
    """Fig. 3: without the correction the rotated wave's viscosity falls with
    the advection velocity."""
    nu0 = measure_nu(2, (64, 64), (1.0, 1.0), (1, 1), (-1, 1), 0.0, 1 / 3, 0.01, mode=oracle.PRODUCT)
    nu2 = measure_nu(2, (64, 64), (1.0, 1.0), (1, 1), (-1, 1), 0.2, 1 / 3, 0.01, mode=oracle.PRODUCT)
    assert nu2 / nu0 < 0.95


def test_viscosity_stretched_second_order_convergent():
    """Fig. 3 with lam_x = 2: the product form shows a large hyper-viscosity,
    the extended equilibrium recovers nu with an error that falls 4x per
    doubling of resolution (second-order central difference)."""
    e1 = measure_nu(2, (32, 64), (2.0, 1.0), (1, 1), (-1, 1), 0.1, 1 / 3, 0.01) / 0.01 - 1
    e2 = measure_nu(2, (64, 128), (2.0, 1.0), (1, 1), (-1, 1), 0.1, 1 / 3, 0.01) / 0.01 - 1
    assert abs(e2) < 0.01
    assert 3.0 < e1 / e2 < 5.0
    bad = measure_nu(2, (32, 64), (2.0, 1.0), (1, 1), (-1, 1), 0.1, 1 / 3, 0.01, mode=oracle.PRODUCT)
    assert bad / 0.01 > 2.0


def test_second_order_equilibrium_loses_galilean_invariance():
    """Fig. 1: the conventional second-order equilibrium's viscosity drops with
    the advection Mach number even for the axis-aligned wave."""
    a = measure_nu(2, (64, 64), (1.0, 1.0), (1, 0), (0, 1), 0.0, 1 / 3, 0.01, mode=oracle.SECOND_ORDER)
    b = measure_nu(2, (64, 64), (1.0, 1.0), (1, 0), (0, 1), 0.2, 1 / 3, 0.01, mode=oracle.SECOND_ORDER)
    assert abs(a / 0.01 - 1) < 0.005
    assert b / a < 0.95


def test_viscosity_3d_rotated_stretched():
    """D3Q27 with lam_z = 2 and the wave rotated in the x-z plane, T = 1/2: the
    extended equilibrium converges to nu at second order; the product form
    keeps a large error."""
    args = ((1.0, 1.0, 2.0), (1, 0, 1), (-1, 0, 1), 0.1, 0.5, 0.02)
    kw = dict(steps=400, every=40, t_min=80)
    e1 = measure_nu(3, (32, 4, 16), *args, **kw) / 0.02 - 1
    e2 = measure_nu(3, (64, 4, 32), *args, **kw) / 0.02 - 1
    assert abs(e2) < 0.015
    assert 3.0 < e1 / e2 < 5.0
    bad = measure_nu(3, (32, 4, 16), *args, mode=oracle.PRODUCT, **kw)
    assert bad / 0.02 > 1.3


def test_taylor_green_decay():
    """2-D Taylor-Green vortex: kinetic energy decays as exp(-2 nu (kx^2+ky^2) t)."""
    n = (64, 64)
    nu = 0.02
    rho, u, (kx, ky) = inputs.taylor_green_2d(n, U=0.01)
    o = oracle.Oracle(2, n, T=1 / 3, nu=nu)
    o.init(rho, u)
    ts, KE = [], []
    for t in range(0, 1001, 50):
        if t:
            o.step(50)
        ts.append(t)
        KE.append(0.5 * (o.macros()[1] ** 2).sum(0).mean())
    rate = decay_rate(ts, KE, 200)
    assert abs(rate / (2 * nu * (kx ** 2 + ky ** 2)) - 1) < 0.001


def test_axis_permutation_symmetry():
    """The product form treats the axes alike: swapping x and y (stretch and
    field) gives the transposed result."""
    rng = np.random.default_rng(3)
    n = (12, 10)
    rho = 1.0 + 0.01 * rng.standard_normal((10, 12))
    u = 0.05 * rng.standard_normal((2, 10, 12))
    a = oracle.Oracle(2, n, lam=(1.0, 1.6, 1.0), T=0.5, nu=0.03)
    a.init(rho, u)
    a.step(30)
    b = oracle.Oracle(2, (10, 12), lam=(1.6, 1.0, 1.0), T=0.5, nu=0.03)
    b.init(rho.T.copy(), np.stack([u[1].T, u[0].T]))
    b.step(30)
    ra, ua = a.macros()
    rb, ub = b.macros()
    np.testing.assert_allclose(rb, ra.T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ub[0], ua[1].T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ub[1], ua[0].T, rtol=0, atol=1e-14)


def test_forced_channel_poiseuille():
    """Walls and body force (readings of the channel setup, Sec. III.E): a
    constant force g between half-way bounce-back walls settles to the
    parabola u = g y (H - y) / (2 nu), H = ny."""
    ny, nu, g = 32, 0.1, 1e-6
    o = oracle.Oracle(2, (4, ny), T=1 / 3, nu=nu, walls_y=True, g=(g, 0.0, 0.0))
    rho, u = inputs.uniform((4, ny), (0.0, 0.0))
    o.init(rho, u)
    o.step(20000)
    prof = o.macros()[1][0, :, 0]
    y = np.arange(ny) + 0.5
    exact = g / (2 * nu) * y * (ny - y)
    assert np.abs(prof - exact).max() / exact.max() < 2e-3
