"""Device-side failure detection on the GPU, without a fault: each bounded
wait of the library -- the mbarrier wait of the TMA-fed kernels, the
progress-counter wait of the fused in-place form -- run on something that
never happens, gives up after its bound with ELBM_ERR_TIMEOUT, and the context
stays usable (a solve in the same form afterwards still matches the oracle)."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2101_04550_gb300 import elbm, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("counter", [False, True])
def test_bounded_wait_gives_up_and_the_device_stays_usable(counter):
    """counter=False: the mbarrier wait of the TMA-fed kernels; True: the
    progress-counter wait of the fused in-place form."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    elbm.load()
    t0 = time.perf_counter()
    rc, msg = elbm.selftest_wait_timeout(50, counter=counter)
    dt = time.perf_counter() - t0
    assert rc == -6, msg                  # ELBM_ERR_TIMEOUT
    assert 0.045 <= dt < 2.0, dt          # gave up after its own bound, not a watchdog's
    # the same process and device still compute correctly, in the TMA-fed form
    n = (64, 32, 32)
    rho, u = inputs.isotropic_turbulence(n, seed=5, k0=3.0, u_rms=0.05)
    with elbm.Solver(elbm.D3Q27, n, T=0.4, nu=0.02, storage=elbm.F32_SHIFT, kernel=4 if counter else 3) as s:
        s.init(rho, u)
        s.step(20)
        _, ug = s.moments()
    o = oracle.Oracle(3, n, T=0.4, nu=0.02)
    o.init(rho, u)
    o.step(20)
    _, uo = o.macros()
    assert np.abs(ug - uo).max() / np.abs(uo).max() <= 1e-5
