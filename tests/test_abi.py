"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/elbm.h declares; argument checks that run before any CUDA call
return ELBM_ERR_ARG / ELBM_ERR_UNREALIZABLE without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2101_04550_gb300 import build as elbm_build
from paper_2101_04550_gb300 import elbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(elbm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    elbm_build.build()
    return elbm.load(build_if_missing=False)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert set(elbm.EXPORTS) <= set(names)


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(elbm_build.ARCH)


def _create(lib, lattice, n, stretch, T, nu, storage=0):
    h = ctypes.c_void_p()
    st = (ctypes.c_double * 3)(*stretch)
    rc = lib.elbm_create(lattice, n[0], n[1], n[2], st, T, nu, storage, None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("args,code", [
    ((5, (8, 8, 1), (1, 1, 1), 0.3, 0.01), -1),          # unknown lattice
    ((9, (8, 8, 2), (1, 1, 1), 0.3, 0.01), -1),          # D2Q9 with nz != 1
    ((27, (8, 2, 8), (1, 1, 1), 0.3, 0.01), -1),         # too few nodes for the central difference
    ((27, (8, 8, 8), (1, -1, 1), 0.3, 0.01), -1),        # negative stretch
    ((27, (8, 8, 8), (1, 1, 1), 0.3, 0.0), -1),          # nu = 0
    ((27, (8, 8, 8), (1, 1, 1), 1.0, 0.01), -2),         # T >= lam^2: rest population not positive
    ((9, (8, 8, 1), (2, 0.5, 1), 0.3, 0.01), -2),        # T >= lam_y^2 = 0.25
    ((27, (1024, 1024, 1024), (1, 1, 1), 0.3, 0.01), -1),  # nx*ny*nz*Q >= 2^31
    ((27, (8, 8, 8), (1, 1, 1), 0.3, 0.01, 7), -1),     # unknown storage
])
def test_argument_checks(lib, args, code):
    rc, h = _create(lib, *args)
    assert rc == code
    assert not h.value
    assert lib.elbm_last_error()


def test_null_handles(lib):
    lib.elbm_destroy(None)
    assert lib.elbm_step(None, 1) == -1
    assert lib.elbm_sync(None) == -1
    assert lib.elbm_cells(None) == 0


def test_selftest_rejects_a_bound_out_of_range(lib):
    """The failure-detection self-test checks its bound before any CUDA call."""
    for ms in (0, -5, 2001):
        assert lib.elbm_selftest_wait_timeout(ms, None) == -1
