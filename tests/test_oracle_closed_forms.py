"""Pins of the FP64 oracle against closed forms the paper fixes (Sec. II.B-C).

Every check builds its own velocity table and moment sums with numpy, so a
dropped term, a wrong sign or a transposed index in the oracle's triplet,
product, equilibrium or anomaly fails here.
"""
import itertools

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20210112)


def table(D):
    """c_i in the documented ordering i = (cx+1) + 3(cy+1) [+ 9(cz+1)]."""
    rows = []
    if D == 3:
        for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3):
            rows.append((cx, cy, cz))
    else:
        for cy, cx in itertools.product((-1, 0, 1), repeat=2):
            rows.append((cx, cy, 0))
    return np.array(rows, dtype=np.float64)


def random_state(D):
    lam = np.array([RNG.uniform(0.7, 2.2) for _ in range(3)])
    u = np.array([RNG.uniform(-0.3, 0.3) for _ in range(3)])
    P = np.array([RNG.uniform(0.2, 0.45) * lam[a] ** 2 for a in range(3)])
    if D == 2:
        u[2] = 0.0
    return u, P, lam


def test_velocity_ordering_matches_documentation():
    for D in (2, 3):
        np.testing.assert_array_equal(oracle.velocities(D), table(D).astype(np.int64))


@pytest.mark.parametrize("trial", range(5))
def test_triplet_moments(trial):
    """Eqs. phi0S/phiPlusS/phiMinusS: sum = 1, first moment u, second P, third lam^2 u."""
    u, P, lam = random_state(3)
    t = oracle.triplet(u[0], P[0], lam[0])
    v = lam[0] * np.array([-1.0, 0.0, 1.0])
    assert np.isclose(t.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.isclose((v * t).sum(), u[0], rtol=0, atol=1e-15)
    assert np.isclose((v ** 2 * t).sum(), P[0], rtol=0, atol=1e-15)
    assert np.isclose((v ** 3 * t).sum(), lam[0] ** 2 * u[0], rtol=0, atol=1e-14)


def closed_form_1d(k, u, P, lam):
    """M_k00 of the factorized moments (Sec. II.B): 1 for k = 0,
    lam^(k-1) u for odd k and lam^(k-2) P for even k >= 2."""
    if k == 0:
        return 1.0
    return lam ** (k - 1) * u if k % 2 else lam ** (k - 2) * P


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("trial", range(4))
def test_product_moments_factorize(D, trial):
    """Normalized moments of the product form equal M_l00 M_0m0 M_00n for
    l, m, n up to 4 (Sec. II.B, with the y and z cases read with m and n)."""
    u, P, lam = random_state(D)
    Psi = oracle.product(D, u, P, lam)
    c = table(D)
    v = c * lam
    orders = range(5)
    for l, m, n in itertools.product(orders, orders, orders if D == 3 else [0]):
        got = np.sum(v[:, 0] ** l * v[:, 1] ** m * v[:, 2] ** n * Psi)
        want = (closed_form_1d(l, u[0], P[0], lam[0]) * closed_form_1d(m, u[1], P[1], lam[1])
                * (closed_form_1d(n, u[2], P[2], lam[2]) if D == 3 else 1.0))
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (l, m, n, got, want)


@pytest.mark.parametrize("D", [2, 3])
def test_product_brute_force_solve(D):
    """The 3^D moments M_lmn, l,m,n in {0,1,2}, fix the 3^D populations: solve
    the moment matrix for the populations that have the closed-form moments and
    compare with the oracle's product form."""
    u, P, lam = random_state(D)
    c = table(D)
    v = c * lam
    rows, rhs = [], []
    for l, m, n in itertools.product(range(3), range(3), range(3) if D == 3 else [0]):
        rows.append(v[:, 0] ** l * v[:, 1] ** m * v[:, 2] ** n)
        rhs.append(closed_form_1d(l, u[0], P[0], lam[0]) * closed_form_1d(m, u[1], P[1], lam[1])
                   * (closed_form_1d(n, u[2], P[2], lam[2]) if D == 3 else 1.0))
    f = np.linalg.solve(np.array(rows), np.array(rhs))
    np.testing.assert_allclose(oracle.product(D, u, P, lam), f, rtol=0, atol=1e-13)


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("T", [1.0 / 3.0, 0.5])
def test_equilibrium_tensors(D, T):
    """Eq. Peq: P^eq = p I + rho u u.  Eqs. Qeq, QMB, Deviation: Q^eq minus the
    Maxwell-Boltzmann third moment vanishes off the diagonal and equals the
    anomaly rho u_a (lam_a^2 - 3T) - rho u_a^3 on it."""
    u, _, lam = random_state(D)
    lam = np.maximum(lam, 1.0)  # keep T + u^2 < lam^2 (positive rest population)
    rho = RNG.uniform(0.8, 1.2)
    feq = oracle.equilibrium(D, rho, u, T, lam)
    P, Qt = oracle.cell_tensors(D, feq, lam)
    p = rho * T
    dims = range(D)
    for a in dims:
        for b in dims:
            assert np.isclose(P[a, b], p * (a == b) + rho * u[a] * u[b], rtol=0, atol=1e-14)
            for g in dims:
                qmb = p * ((a == b) * u[g] + (a == g) * u[b] + (b == g) * u[a]) + rho * u[a] * u[b] * u[g]
                dev = Qt[a, b, g] - qmb
                if a == b == g:
                    want = rho * u[a] * (lam[a] ** 2 - 3 * T) - rho * u[a] ** 3
                    assert np.isclose(dev, want, rtol=0, atol=1e-14)
                    assert np.isclose(oracle.anomaly(rho, u[a], lam[a], T), want, rtol=0, atol=1e-15)
                else:
                    assert abs(dev) < 1e-14, (a, b, g, dev)


def test_anomaly_special_case_lattice_temperature():
    """Eq. TL: at T = 1/3 and lam = 1 the linear term vanishes, leaving -rho u^3."""
    for u in (-0.2, 0.05, 0.3):
        assert np.isclose(oracle.anomaly(1.3, u, 1.0, 1.0 / 3.0), -1.3 * u ** 3, rtol=1e-14, atol=0)


@pytest.mark.parametrize("D", [2, 3])
def test_conservation_of_equilibrium(D):
    """Eqs. density, momentum: the equilibrium carries rho and rho u."""
    u, _, lam = random_state(D)
    lam = np.maximum(lam, 1.0)
    rho = 0.93
    feq = oracle.equilibrium(D, rho, u, 0.4, lam)
    r, uu = oracle.cell_moments(D, feq, lam)
    assert np.isclose(r, rho, rtol=1e-15)
    np.testing.assert_allclose(uu[:D], u[:D], rtol=0, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_second_order_equilibrium_is_textbook_at_lattice_temperature(D):
    """At T = 1/3 and lam = 1 the product form truncated to second order is the
    standard polynomial w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u) with the
    product weights (2/3, 1/6, 1/6) per axis (Sec. III preamble)."""
    c = table(D)
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    u = np.array([0.07, -0.11, 0.05 if D == 3 else 0.0])
    rho = 1.07
    f2 = oracle.equilibrium(D, rho, u, 1.0 / 3.0, [1.0, 1.0, 1.0], second_order=True)
    for i, ci in enumerate(c):
        w = np.prod([w1[int(ci[a])] for a in range(D)])
        cu = ci @ u
        want = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
        assert np.isclose(f2[i], want, rtol=0, atol=1e-15), (i, f2[i], want)


def test_central_difference_second_order():
    """Eq. Paastar1 takes a second-order central difference with node spacing
    lam: on q = sin(k x) it gives cos(k x) sin(k lam)/lam exactly, and its
    error against the derivative falls 4x per halving of lam k."""
    errs = []
    for nx in (16, 32, 64):
        lam = 1.7
        o = oracle.Oracle(2, (nx, 3), lam=(lam, 1.0, 1.0), T=1 / 3, nu=0.1)
        x = np.arange(nx) * lam
        k = 2 * np.pi / (nx * lam)
        q = np.tile(np.sin(k * x), (3, 1))
        d = o.central_difference(q, 0)[0]
        np.testing.assert_allclose(d, np.cos(k * x) * np.sin(k * lam) / lam, rtol=0, atol=1e-14)
        errs.append(np.abs(d - k * np.cos(k * x)).max() / k)
        # along y the field is constant, the difference vanishes
        assert np.abs(o.central_difference(q, 1)).max() == 0.0
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def truncated_moment(orders, u, T, lam, D):
    """Moment sum_i rho^-1 prod_a (lam_a c_ia)^(l_a) f_i of the second-order
    equilibrium (Sec. III preamble) in closed form.  Per axis the product form
    has the moments 1, u_a, T + u_a^2 (Sec. II.B: M_100 = u, M_200 = P with
    P = T + u^2); a moment of the product is the product of the per-axis
    moments, and dropping every term above second order in u from the
    populations drops the same terms from each moment, because the moment sum
    does not mix powers of u.  So the moment is the product of the per-axis
    polynomials with every term of total degree above two removed."""
    # per-axis polynomial in u_a: coefficients of u_a^0, u_a^1, u_a^2
    per_axis = {0: (1.0, 0.0, 0.0), 1: (0.0, 1.0, 0.0), 2: (T, 0.0, 1.0)}
    total = 0.0
    for powers in itertools.product(range(3), repeat=D):
        if sum(powers) > 2:
            continue
        term = 1.0
        for a in range(D):
            term *= per_axis[orders[a]][powers[a]] * u[a] ** powers[a]
        total += term
    return total


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("trial", range(6))
def test_second_order_equilibrium_moments_general_T_lambda(D, trial):
    """The second-order equilibrium at random stretch lam in [0.7, 2.2] and
    T in (0.2, 0.6) (Sec. III preamble, Eqs. Peq, Qeq): all 3^D moments with
    orders <= 2 per axis -- which fix the 3^D populations -- equal their closed
    forms.  So rho, rho u and the pressure rho (T I + u u) are kept exactly,
    the diagonal third moment is rho lam_a^2 u_a (c^3 = c on the lattice), and
    the off-diagonal Q_abb loses exactly rho u_a u_b^2 against the product form."""
    rng = np.random.default_rng(1000 + 10 * D + trial)
    lam = np.array([rng.uniform(0.7, 2.2) for _ in range(3)])
    T = rng.uniform(0.2, 0.6) * min(1.0, float(np.min(lam[:D] ** 2)))
    u = np.array([rng.uniform(-0.2, 0.2) for _ in range(3)])
    if D == 2:
        u[2] = 0.0
    rho = rng.uniform(0.8, 1.2)
    c = table(D)
    v = c * lam
    f2 = oracle.equilibrium(D, rho, u, T, lam, second_order=True)
    for orders in itertools.product(range(3), repeat=D):
        m = (f2 * np.prod([v[:, a] ** orders[a] for a in range(D)], axis=0)).sum()
        want = rho * truncated_moment(orders, u, T, lam, D)
        assert abs(m - want) <= 1e-14 * max(1.0, abs(want)), (orders, m, want)
    # the named tensors, spelled out
    mom = lambda w: (f2 * w).sum()
    assert np.isclose(mom(np.ones(len(c))), rho, rtol=1e-15)
    for a in range(D):
        assert np.isclose(mom(v[:, a]), rho * u[a], rtol=0, atol=1e-15)
        assert np.isclose(mom(v[:, a] ** 3), rho * lam[a] ** 2 * u[a], rtol=0, atol=1e-14)
        for b in range(D):
            want_p = rho * ((T if a == b else 0.0) + u[a] * u[b])
            assert np.isclose(mom(v[:, a] * v[:, b]), want_p, rtol=0, atol=1e-14)
            if a != b:
                feq = oracle.equilibrium(D, rho, u, T, lam)
                q_full = (feq * v[:, a] * v[:, b] ** 2).sum()
                q_trunc = mom(v[:, a] * v[:, b] ** 2)
                assert np.isclose(q_full - q_trunc, rho * u[a] * u[b] ** 2, rtol=0, atol=1e-14)
