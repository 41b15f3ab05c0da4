"""Pins of the oracle's wall and body-force options (the channel setup of
Sec. III.E), each against something other than the oracle itself: closed
forms of a uniformly accelerated flow, exact conservation, the exact
difference quotient of fields that are odd about the walls, mirror symmetry
and the steady Poiseuille parabola with its second-order convergence."""
import numpy as np
import pytest

import oracle
from paper_2101_04550_gb300 import inputs


def test_force_accelerates_uniform_flow_exactly():
    """Exact-difference forcing on a uniform flow: f = f^eq(rho, u) relaxes to
    itself (the anomaly is uniform, its difference vanishes) and gains
    f^eq(rho, u + g) - f^eq(rho, u), so after n steps f = f^eq(rho, u0 + n g)
    (Eq. 27eq) and the reported half-step velocity is u0 + (n + 1/2) g."""
    lam, T = (1.5, 1.0, 2.0), 0.5
    n, steps = (4, 3, 5), 7
    u0 = np.array([0.05, -0.02, 0.03])
    g = np.array([1e-3, -2e-3, 3e-3])
    o = oracle.Oracle(3, n, lam=lam, T=T, nu=0.05, g=tuple(g))
    rho, u = inputs.uniform(n, tuple(u0), rho0=1.1)
    o.init(rho, u)
    o.step(steps)
    want = oracle.equilibrium(3, 1.1, u0 + steps * g, T, lam)
    np.testing.assert_allclose(o.f, np.repeat(want[:, None], o.N, axis=1), rtol=0, atol=1e-14)
    r, uu = o.macros()
    np.testing.assert_allclose(r, 1.1, rtol=0, atol=1e-13)
    for a in range(3):
        np.testing.assert_allclose(uu[a], u0[a] + (steps + 0.5) * g[a], rtol=0, atol=1e-14)


@pytest.mark.parametrize("D,n,lam", [(2, (12, 10), (2.0, 1.0)), (3, (6, 5, 7), (1.0, 1.5, 2.0))])
def test_force_adds_momentum_rho_g_per_step(D, n, lam):
    """On a periodic grid the only momentum source is the force: the total
    momentum grows by sum(rho) g every step, while mass stays fixed."""
    g = (2e-4, -1e-4, 3e-4)[:D]
    shape = n[::-1]
    rng = np.random.Generator(np.random.PCG64(1))
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((D,) + shape)
    o = oracle.Oracle(D, n, lam=tuple(lam) + (1.0,) * (3 - len(lam)), T=0.5, nu=0.05,
                      g=tuple(g) + (0.0,) * (3 - D))
    o.init(rho, u)
    c = oracle.velocities(D)
    lam3 = np.array(tuple(lam) + (1.0,) * (3 - len(lam)))

    def totals():
        mass = o.f.sum()
        mom = np.array([(lam3[a] * c[:, a][:, None] * o.f).sum() for a in range(D)])
        return mass, mom

    m0, p0 = totals()
    for _ in range(5):
        o.step(1)
        m1, p1 = totals()
        assert abs(m1 - m0) <= 1e-13 * m0
        np.testing.assert_allclose(p1 - p0, m0 * np.array(g), rtol=1e-9, atol=1e-15)
        m0, p0 = m1, p1


def test_central_difference_ghost_is_exact_for_fields_odd_about_the_walls():
    """The anomaly Q~_yyy is odd in u_y, which vanishes on the walls, so its
    ghost value beyond a wall is the negated first value.  On
    q = sin(m pi y / H) (y = (j + 1/2) lam_y, odd about both walls) the
    difference with that ghost is cos(k y) sin(k lam)/lam exactly at every
    node, the wall-adjacent ones included; a periodic wrap is not."""
    for lam_y, ny, m in [(1.0, 16, 1), (1.5, 12, 3), (0.8, 20, 2)]:
        o = oracle.Oracle(2, (3, ny), lam=(1.0, lam_y, 1.0), T=0.3, nu=0.1, walls_y=True)
        H = ny * lam_y
        y = (np.arange(ny) + 0.5) * lam_y
        k = m * np.pi / H
        q = np.tile(np.sin(k * y)[:, None], (1, 3))
        d = o.central_difference(q, 1)
        want = np.cos(k * y) * np.sin(k * lam_y) / lam_y
        np.testing.assert_allclose(d, np.tile(want[:, None], (1, 3)), rtol=0, atol=1e-14)
        if m % 2 == 1:  # (for even m the periodic wrap happens to agree with the ghost)
            periodic = oracle.Oracle(2, (3, ny), lam=(1.0, lam_y, 1.0), T=0.3, nu=0.1)
            dp = periodic.central_difference(q, 1)
            assert np.abs(dp[0] - want[0]).max() > 1e-2 * np.abs(want).max()
        # along x the walls change nothing
        assert np.abs(o.central_difference(q, 0)).max() == 0.0


@pytest.mark.parametrize("D,n,lam,T", [(2, (10, 12), (2.0, 1.0), 0.55), (3, (6, 8, 5), (2.0, 1.0, 2.0), 0.55)])
def test_walls_conserve_mass(D, n, lam, T):
    """Half-way bounce-back returns every population that reaches a wall, so
    the total mass of a walled grid stays fixed (Eq. density summed)."""
    shape = n[::-1]
    rng = np.random.Generator(np.random.PCG64(7))
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((D,) + shape)
    o = oracle.Oracle(D, n, lam=tuple(lam) + (1.0,) * (3 - len(lam)), T=T, nu=0.02, walls_y=True,
                      g=(1e-4, 0.0, 0.0))
    o.init(rho, u)
    m0 = o.f.sum()
    o.step(60)
    assert abs(o.f.sum() - m0) <= 1e-13 * m0


def test_walls_mirror_symmetry():
    """Reflecting the initial field about the channel's mid-plane (y -> H - y,
    u_y -> -u_y) reflects the solution: the two walls are treated alike."""
    n, lam = (12, 10), (2.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(11))
    rho = 1.0 + 0.01 * rng.standard_normal((n[1], n[0]))
    u = 0.05 * rng.standard_normal((2, n[1], n[0]))
    rho_m = rho[::-1].copy()
    u_m = np.stack([u[0][::-1], -u[1][::-1]])
    out = []
    for r, v in [(rho, u), (rho_m, u_m)]:
        o = oracle.Oracle(2, n, lam=lam + (1.0,), T=0.55, nu=0.02, walls_y=True, g=(1e-4, 0.0, 0.0))
        o.init(r, v)
        o.step(80)
        out.append(o.macros())
    (ra, ua), (rb, ub) = out
    np.testing.assert_allclose(rb, ra[::-1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(ub[0], ua[0][::-1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(ub[1], -ua[1][::-1], rtol=0, atol=1e-13)


def _poiseuille_error(ny, lam, T, nu, steps):
    g = 1e-6
    o = oracle.Oracle(2, (4, ny), lam=lam + (1.0,), T=T, nu=nu, walls_y=True, g=(g, 0.0, 0.0))
    rho, u = inputs.uniform((4, ny), (0.0, 0.0))
    o.init(rho, u)
    o.step(steps)
    prof = o.macros()[1][0, :, 0]
    H = ny * lam[1]
    y = (np.arange(ny) + 0.5) * lam[1]
    exact = g / (2 * nu) * y * (H - y)
    return np.abs(prof - exact).max() / exact.max()


@pytest.mark.parametrize("lam,T,nu", [((2.0, 1.0), 0.55, 0.1), ((1.0, 1.5), 0.5, 0.2)])
def test_poiseuille_converges_at_second_order(lam, T, nu):
    """Steady channel flow between the walls y = 0 and y = H (half a spacing
    outside the first and last nodes) under a constant force is the parabola
    u_x = g y (H - y) / (2 nu); its error falls about 4x per doubling of ny,
    on the channel's stretched lattice too."""
    e16 = _poiseuille_error(16, lam, T, nu, 12000)
    e32 = _poiseuille_error(32, lam, T, nu, 30000)
    assert e16 < 1e-2 and e32 < 3e-3
    assert 3.0 < e16 / e32 < 5.0
