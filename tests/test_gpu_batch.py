"""Batched step: grids of different sizes, stretches, temperatures and
viscosities advanced together give bit for bit the states of stepping each
alone (the per-node arithmetic is the same), also for members that join at
the other streaming parity and that are stepped alone afterwards."""
import numpy as np
import pytest
import torch

from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()


SPECS3 = [((32, 32, 32), (1.0, 1.0, 1.0), 1 / 3, 0.02), ((48, 40, 36), (1.0, 2.0, 1.0), 0.5, 0.01),
          ((20, 12, 9), (1.5, 1.0, 2.0), 0.45, 0.05), ((64, 32, 64), (1.0, 2.0, 1.0), 0.6, 0.015)]
SPECS2 = [((64, 64, 1), (1.0, 1.0, 1.0), 1 / 3, 0.02), ((100, 37, 1), (2.0, 1.0, 1.0), 0.5, 0.03)]


def _fields(n, seed, D):
    if D == 3:
        return inputs.isotropic_turbulence(n, seed=seed, k0=3.0, u_rms=0.05)
    rho, u = inputs.double_shear_layer(n[:2], U=0.08)
    return rho, u


def _make(lattice, spec, storage, seed):
    n, lam, T, nu = spec
    D = 3 if lattice == elbm.D3Q27 else 2
    s = elbm.Solver(lattice, n, stretch=lam, T=T, nu=nu, storage=storage, kernel=1,
                    stream=torch.cuda.current_stream())
    rho, u = _fields(n, seed, D)
    s.init(rho, u)
    return s


@pytest.mark.parametrize("lattice,specs", [(elbm.D3Q27, SPECS3), (elbm.D2Q9, SPECS2)])
@pytest.mark.parametrize("storage", [elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_batch_matches_solo_bitwise(lattice, specs, storage):
    solo = [_make(lattice, sp, storage, k) for k, sp in enumerate(specs)]
    mixed = [_make(lattice, sp, storage, k) for k, sp in enumerate(specs)]
    # one member joins at the odd parity
    solo[1].step(1)
    mixed[1].step(1)
    for s in solo:
        s.step(23)
    with elbm.Batch(mixed) as b:
        b.step(3)      # two tuning steps, then one replayed step
        b.step(10)     # captured sequence of 10 steps
        b.step(10)     # replay
        info = b.info()
    assert info["block_size"] in (128, 256)
    for s, m in zip(solo, mixed):
        assert m.steps_done == s.steps_done
        assert np.array_equal(s.get_populations(), m.get_populations())
    # members keep stepping alone after the batch is gone
    for s, m in zip(solo, mixed):
        s.step(3)
        m.step(3)
        assert np.array_equal(s.get_populations(), m.get_populations())
    for s in solo + mixed:
        s.close()


def test_batch_rejects_mixed_storage():
    a = _make(elbm.D3Q27, SPECS3[0], elbm.F32_SHIFT, 0)
    b = _make(elbm.D3Q27, SPECS3[2], elbm.F16_SHIFT, 1)
    with pytest.raises(elbm.ElbmError):
        elbm.Batch([a, b])
    a.close()
    b.close()


def test_members_join_and_leave_a_running_batch():
    specs = SPECS3
    solo = [_make(elbm.D3Q27, sp, elbm.F32_SHIFT, k) for k, sp in enumerate(specs)]
    mixed = [_make(elbm.D3Q27, sp, elbm.F32_SHIFT, k) for k, sp in enumerate(specs)]
    with elbm.Batch(mixed[:2]) as b:
        b.step(10)
        b.add(mixed[2])          # joins mid-flight at step 0
        b.step(7)
        b.remove(mixed[0])       # leaves after 17 steps
        b.add(mixed[3])
        b.step(7)                # replays the graph of 7 steps with new members
        assert len(b) == 3
    counts = [17, 24, 14, 7]
    for s, m, k in zip(solo, mixed, counts):
        s.step(k)
        assert m.steps_done == k
        assert np.array_equal(s.get_populations(), m.get_populations())
    for s in solo + mixed:
        s.close()


# single-pass members (kernel 3): x a multiple of 32 nodes and y of 16 for the TMEM form
SPECS_SP = [((32, 32, 32), (1.0, 1.0, 1.0), 1 / 3, 0.02), ((64, 32, 64), (1.0, 2.0, 1.0), 0.6, 0.015),
            ((96, 48, 40), (1.0, 1.5, 2.0), 0.45, 0.01), ((64, 16, 7), (1.0, 1.0, 1.0), 0.5, 0.03)]


def _make_sp(spec, storage, seed, **kw):
    n, lam, T, nu = spec
    s = elbm.Solver(elbm.D3Q27, n, stretch=lam, T=T, nu=nu, storage=storage, kernel=3,
                    stream=torch.cuda.current_stream(), **kw)
    s.init(*_fields(n, seed, 3))
    return s


@pytest.mark.parametrize("storage", [elbm.F32_SHIFT, elbm.F16_SHIFT])
def test_single_pass_batch_matches_solo_bitwise(storage):
    """Single-pass members of different sizes and parameters, with an odd step
    count (the arrays swap) and a repeated one (the cached graphs replay):
    bit for bit the states of stepping each alone."""
    solo = [_make_sp(sp, storage, k) for k, sp in enumerate(SPECS_SP)]
    mixed = [_make_sp(sp, storage, k) for k, sp in enumerate(SPECS_SP)]
    for s in solo:
        s.step(27)
    with elbm.Batch(mixed) as b:
        b.step(7)
        b.step(10)
        b.step(10)
        info = b.info()
        tuning = b.tuning()
    # every candidate of the autotuner ran two real steps of these members
    assert info["block_size"] == 0 and tuning["tuned"] and min(tuning["ms"]) > 0
    for s, m in zip(solo, mixed):
        assert m.steps_done == s.steps_done == 27
        assert np.array_equal(s.get_populations(), m.get_populations())


@pytest.mark.parametrize("config", range(elbm.BATCH_CONFIGS))
def test_single_pass_batch_every_configuration_bitwise(config):
    """Each configuration of the single-pass batch -- the flattened launch on
    32 x 16 (TMEM) or 32 x 8 (TMA) tile columns with 32-, 16- or 8-plane
    segments, members one after another or interleaved, and per-member
    graphs -- pinned, over odd and even step counts, with a member whose grid
    only the 32 x 8 kernel takes beside them (per-member graphs under the
    TMEM configurations): bit for bit the solo states; a flattened
    configuration makes one launch per step."""
    specs = SPECS_SP + [((32, 8, 16), (1.0, 1.0, 1.0), 0.4, 0.02)]
    solo = [_make_sp(sp, elbm.F16_SHIFT, k) for k, sp in enumerate(specs)]
    mixed = [_make_sp(sp, elbm.F16_SHIFT, k) for k, sp in enumerate(specs)]
    assert mixed[-1].kernel_form == (3, 2)
    for s in solo:
        s.step(16)
    with elbm.Batch(mixed) as b:
        b.set_config(config)
        before = b.info()["launches"]
        b.step(5)
        b.step(11)
        launches = b.info()["launches"] - before
        t = b.tuning()
    assert t["config"] == config and t["tuned"]
    assert t["tile_rows"] == (16 if config < 6 else 8 if config < 12 else 0)
    if config < 6:
        want = 16 + 16          # one launch per step + the 32 x 8 member's own launches
    elif config < 12:
        want = 16               # every member in the 32 x 8 flattened launch
    else:
        want = 16 * len(specs)  # per-member graphs
    assert launches == want
    for s, m in zip(solo, mixed):
        assert np.array_equal(s.get_populations(), m.get_populations())


@pytest.mark.parametrize("lattice,specs", [(elbm.D3Q27, SPECS3), (elbm.D2Q9, SPECS2)])
def test_two_pass_batches_live_side_by_side(lattice, specs):
    """Two two-pass batches of the same lattice and storage mode at once (each
    keeps its member table in device memory of its own), stepped alternately
    with different step counts: bit for bit the solo states."""
    solo = [_make(lattice, sp, elbm.F32_SHIFT, k) for k, sp in enumerate(specs)]
    mixed = [_make(lattice, sp, elbm.F32_SHIFT, k) for k, sp in enumerate(specs)]
    half = len(specs) // 2
    for s in solo[:half]:
        s.step(9)
    for s in solo[half:]:
        s.step(12)
    with elbm.Batch(mixed[:half]) as b1, elbm.Batch(mixed[half:]) as b2:
        for k1, k2 in ((3, 5), (6, 7)):
            b1.step(k1)
            b2.step(k2)
    for s, m in zip(solo, mixed):
        assert np.array_equal(s.get_populations(), m.get_populations())
    for s in solo + mixed:
        s.close()


def test_single_pass_batches_live_side_by_side():
    """Two single-pass batches of the same storage mode at once (the member
    tables live in each batch's device memory), stepped alternately."""
    solo = [_make_sp(sp, elbm.F32_SHIFT, k) for k, sp in enumerate(SPECS_SP)]
    mixed = [_make_sp(sp, elbm.F32_SHIFT, k) for k, sp in enumerate(SPECS_SP)]
    for s in solo:
        s.step(9)
    with elbm.Batch(mixed[:2]) as b1, elbm.Batch(mixed[2:]) as b2:
        for k in (3, 6):
            b1.step(k)
            b2.step(k)
    for s, m in zip(solo, mixed):
        assert np.array_equal(s.get_populations(), m.get_populations())


def test_single_pass_batch_membership_and_bounded_members():
    """Members leave and join between steps (a leaving member's graphs are
    released), a wall-bounded, forced channel member runs beside periodic ones,
    and every state equals the solo run; two-pass and single-pass members do
    not share a batch."""
    chan = ((64, 32, 20), (2.0, 1.0, 2.0), 0.55, 0.02)
    rho_c, u_c = inputs.channel(chan[0], chan[1], u_center=0.05, perturbation=0.05, seed=3)

    def make_chan():
        s = elbm.Solver(elbm.D3Q27, chan[0], stretch=chan[1], T=chan[2], nu=chan[3], storage=elbm.F32, kernel=3,
                        walls_y=True, force=(2e-5, 0.0, 0.0), stream=torch.cuda.current_stream())
        s.init(rho_c, u_c)
        return s

    specs = SPECS_SP[:3]
    solo = [_make_sp(sp, elbm.F32, k) for k, sp in enumerate(specs)] + [make_chan()]
    mixed = [_make_sp(sp, elbm.F32, k) for k, sp in enumerate(specs)] + [make_chan()]
    steps = [0] * 4
    with elbm.Batch([mixed[0], mixed[3]]) as b:
        b.step(5)
        steps[0] += 5; steps[3] += 5
        b.add(mixed[1])
        b.add(mixed[2])
        b.step(4)
        for k in range(4):
            steps[k] += 4
        b.remove(mixed[0])
        b.step(5)
        for k in (1, 2, 3):
            steps[k] += 5
        b.add(mixed[0])
        b.step(4)
        for k in range(4):
            steps[k] += 4
        assert len(b) == 4
        with pytest.raises(elbm.ElbmError):
            b.add(_make(elbm.D3Q27, SPECS3[0], elbm.F32, 9))  # a two-pass member
    for s, k in zip(solo, steps):
        s.step(k)
    for s, m in zip(solo, mixed):
        assert m.steps_done == s.steps_done
        assert np.array_equal(s.get_populations(), m.get_populations())


def test_d2q9_single_pass_members_batch_bitwise():
    """D2Q9 solvers in the automatic form (the row-march single pass) batch
    together as per-member graphs: bit for bit the solo states, over an odd
    and an even step count (the arrays swap)."""
    specs = [((256, 128, 1), (1.0, 1.0, 1.0), 0.5, 0.01), ((300, 77, 1), (1.0, 2.0, 1.0), 0.5, 0.02),
             ((64, 64, 1), (2.0, 1.0, 1.0), 1 / 3, 0.02)]

    def make(spec, seed):
        n, lam, T, nu = spec
        s = elbm.Solver(elbm.D2Q9, n, stretch=lam, T=T, nu=nu, storage=elbm.F32_SHIFT,
                        stream=torch.cuda.current_stream())
        s.init(*_fields(n, seed, 2))
        return s

    solo = [make(sp, k) for k, sp in enumerate(specs)]
    mixed = [make(sp, k) for k, sp in enumerate(specs)]
    assert all(m.kernel_form == (3, 4) for m in mixed)
    for s in solo:
        s.step(12)
    with elbm.Batch(mixed) as b:
        b.step(5)
        b.step(7)
        assert b.tuning()["member_graphs"]
    for s, m in zip(solo, mixed):
        assert m.steps_done == 12
        assert np.array_equal(s.get_populations(), m.get_populations())
    for s in solo + mixed:
        s.close()
