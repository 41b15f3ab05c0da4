"""FP64 CPU oracle of the extended LBGK step (arXiv 2101.04550, Sec. II).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never does.  The
arithmetic lives in ``elbm_oracle.c`` (plain C, double precision, whole-grid
sub-steps in the paper's order); this module compiles it with gcc on first use
and marshals numpy arrays through ctypes.

Layouts (shared with the library only as a documented interface):
population ``f[i][z][y][x]`` with ``i = (cx+1) + 3(cy+1) + 9(cz+1)``;
``rho[z][y][x]``; ``u[alpha][z][y][x]``.  For D = 2 arrays keep ``nz = 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

EXTENDED, PRODUCT, SECOND_ORDER = 0, 1, 2


class Lattice(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lam", ctypes.c_double * 3),
        ("T", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("mode", ctypes.c_int),
        ("walls_y", ctypes.c_int),
        ("g", ctypes.c_double * 3),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(Lattice)
            L.ora_step.argtypes = [lp, dp, dp]
            L.ora_run.argtypes = [lp, dp, ctypes.c_int]
            L.ora_init.argtypes = [lp, dp, dp, dp]
            L.ora_macros.argtypes = [lp, dp, dp, dp]
            L.ora_central_difference.argtypes = [lp, dp, ctypes.c_int, dp]
            L.ora_triplet.argtypes = [ctypes.c_double] * 3 + [dp]
            L.ora_product.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            L.ora_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp, dp]
            L.ora_second_order_equilibrium.argtypes = L.ora_equilibrium.argtypes
            L.ora_cell_moments.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            L.ora_anomaly.argtypes = [ctypes.c_double] * 4
            L.ora_anomaly.restype = ctypes.c_double
            L.ora_cell_tensors.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            L.ora_velocity.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            _lib = L
        return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def omega_from_nu(nu: float, T: float) -> float:
    """Eq. nu with R = 1, delta t = 1: nu = (1/omega - 1/2) T."""
    return 1.0 / (nu / T + 0.5)


def velocities(D: int) -> np.ndarray:
    """c_i for the documented ordering, shape (Q, 3)."""
    Q = 9 if D == 2 else 27
    out = np.zeros((Q, 3), dtype=np.int64)
    c = (ctypes.c_int * 3)()
    for i in range(Q):
        lib().ora_velocity(D, i, c)
        out[i] = list(c)
    return out


class Oracle:
    """A periodic (or y-walled) grid advanced by the FP64 oracle step."""

    def __init__(self, D, n, lam=(1.0, 1.0, 1.0), T=1.0 / 3.0, nu=None, omega=None,
                 mode=EXTENDED, walls_y=False, g=(0.0, 0.0, 0.0)):
        n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        if D == 2:
            n = (n[0], n[1], 1)
        if omega is None:
            omega = omega_from_nu(nu, T)
        self.D, self.Q = D, (9 if D == 2 else 27)
        self.n = n
        self.N = n[0] * n[1] * n[2]
        self.L = Lattice(D, (ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*lam), T, omega,
                         mode, int(walls_y), (ctypes.c_double * 3)(*g))
        self.f = np.zeros((self.Q, self.N), dtype=np.float64)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (ny, nx) if self.D == 2 else (nz, ny, nx)

    def init(self, rho, u):
        """Populations set to the product-form equilibrium of (rho, u) (Eq. 27eq)."""
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.N))
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(self.D, self.N))
        lib().ora_init(ctypes.byref(self.L), _ptr(rho), _ptr(u), _ptr(self.f))

    def step(self, n=1):
        if lib().ora_run(ctypes.byref(self.L), _ptr(self.f), int(n)) != 0:
            raise MemoryError("oracle step could not allocate its work arrays")

    def macros(self):
        rho = np.zeros(self.N)
        u = np.zeros((self.D, self.N))
        lib().ora_macros(ctypes.byref(self.L), _ptr(self.f), _ptr(rho), _ptr(u))
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape)

    def central_difference(self, q, alpha):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(self.N))
        out = np.zeros(self.N)
        lib().ora_central_difference(ctypes.byref(self.L), _ptr(q), int(alpha), _ptr(out))
        return out.reshape(self.shape)


def triplet(u, P, lam):
    out = np.zeros(3)
    lib().ora_triplet(u, P, lam, _ptr(out))
    return out


def product(D, u, P, lam):
    Q = 9 if D == 2 else 27
    out = np.zeros(Q)
    lib().ora_product(D, _ptr(np.array(u, float)), _ptr(np.array(P, float)),
                      _ptr(np.array(lam, float)), _ptr(out))
    return out


def equilibrium(D, rho, u, T, lam, second_order=False):
    Q = 9 if D == 2 else 27
    out = np.zeros(Q)
    fn = lib().ora_second_order_equilibrium if second_order else lib().ora_equilibrium
    fn(D, float(rho), _ptr(np.array(u, float)), float(T), _ptr(np.array(lam, float)), _ptr(out))
    return out


def cell_moments(D, fc, lam):
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().ora_cell_moments(D, _ptr(np.ascontiguousarray(fc, dtype=np.float64)),
                           _ptr(np.array(lam, float)), _ptr(rho), _ptr(u))
    return rho[0], u


def cell_tensors(D, fc, lam):
    P = np.zeros(9)
    Qt = np.zeros(27)
    lib().ora_cell_tensors(D, _ptr(np.ascontiguousarray(fc, dtype=np.float64)),
                           _ptr(np.array(lam, float)), _ptr(P), _ptr(Qt))
    return P.reshape(3, 3), Qt.reshape(3, 3, 3)


def anomaly(rho, u, lam, T):
    return lib().ora_anomaly(float(rho), float(u), float(lam), float(T))
