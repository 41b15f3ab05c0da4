"""The allocation-free step (elbm_step_noalloc) against the solver's step.

Some callers cannot allocate device memory themselves: applications that route
every device allocation through their own pool, plugins whose host framework
forbids allocations on its threads, code that records CUDA work where
cudaMalloc is not allowed.  They hand the library their own population buffer
and the step uses a fixed scratch array inside the library.  This file is
collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2101_04550_gb300 import elbm

pytestmark = pytest.mark.gpu


def noalloc_step(lib, lattice, n, lam, T, nu, f_dev, nsteps, stream):
    fn = lib.elbm_step_noalloc
    fn.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    st = (ctypes.c_double * 3)(*[float(v) for v in lam])
    return fn(lattice, n[0], n[1], n[2], st, T, nu, ctypes.c_void_p(f_dev.data_ptr()), nsteps,
              ctypes.c_void_p(stream.cuda_stream))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return elbm.load()


@pytest.mark.parametrize("lattice,n,lam,T", [(elbm.D3Q27, (20, 12, 9), (1.0, 1.5, 2.0), 0.45),
                                             (elbm.D2Q9, (48, 40, 1), (2.0, 1.0, 1.0), 0.4)])
def test_noalloc_step_matches_solver_step_on_two_calls(lib, lattice, n, lam, T):
    D = 3 if lattice == elbm.D3Q27 else 2
    rng = np.random.default_rng(17)
    shape = (n[2], n[1], n[0]) if D == 3 else (n[1], n[0])
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.04 * rng.standard_normal((D,) + shape)
    stream = torch.cuda.current_stream()
    with elbm.Solver(lattice, n, stretch=lam, T=T, nu=0.03, storage=elbm.F32, kernel=1, stream=stream) as s:
        s.init(rho, u)
        f = torch.tensor(s.get_populations(dtype=np.float32), device="cuda").contiguous()
        # an odd then an even number of steps: the layout restore and a second
        # call on the scratch the first call left behind
        for nsteps in (7, 4):
            rc = noalloc_step(lib, lattice, n, lam, T, 0.03, f, nsteps, stream)
            assert rc == 0, lib.elbm_last_error().decode()
            torch.cuda.synchronize()
            s.step(nsteps)
            ref = s.get_populations(dtype=np.float32)
            got = f.cpu().numpy().reshape(ref.shape)
            np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7)


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    f = torch.zeros(27, device="cuda")
    rc = noalloc_step(lib, elbm.D3Q27, (128, 64, 64), (1.0, 1.0, 1.0), 1 / 3, 0.01, f,
                      1, torch.cuda.current_stream())
    assert rc == -1
    assert b"262144" in lib.elbm_last_error()
