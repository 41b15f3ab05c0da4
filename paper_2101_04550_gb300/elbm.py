"""ctypes binding of the elbm C ABI (include/elbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libelbm.so``.  Buffers may be numpy arrays (host) or torch
CUDA tensors (device, passed by pointer).  If the library is missing or
cannot be loaded the first call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

D2Q9, D3Q27 = 9, 27
F32, F16_SHIFT, BF16_SHIFT, F32_SHIFT = 0, 1, 2, 3
DTYPE_F32, DTYPE_F64 = 0, 1
OPT_EQUILIBRIUM, OPT_KERNEL, OPT_RHO_REF = 1, 2, 3
OPT_FORCE_X, OPT_FORCE_Y, OPT_FORCE_Z, OPT_WALLS_Y = 4, 5, 6, 7
OPT_U_REF_X, OPT_U_REF_Y, OPT_U_REF_Z, OPT_U_REF_AUTO = 8, 9, 10, 11
NRED = 13
BATCH_CONFIGS = 13   # single-pass batch configurations (ELBM_BATCH_CONFIGS)
ERRORS = {0: "OK", -1: "ARG", -2: "UNREALIZABLE", -3: "OOM", -4: "CUDA", -5: "NONFINITE",
          -6: "TIMEOUT", -7: "STATE"}
STORAGE_NAMES = {"f32": F32, "f16": F16_SHIFT, "bf16": BF16_SHIFT, "f32s": F32_SHIFT}
STORAGE_BYTES = {F32: 4, F16_SHIFT: 2, BF16_SHIFT: 2, F32_SHIFT: 4}
RED_NAMES = ["mass", "mom_x", "mom_y", "mom_z", "rho_u2", "u2", "curl2", "dxux2", "ux2", "fmin",
             "nonfinite", "umax", "wall_dudn"]

_lock = threading.Lock()
_lib = None
EXPORTS = ["elbm_create", "elbm_destroy", "elbm_set_option", "elbm_init", "elbm_step", "elbm_moments",
           "elbm_get_populations", "elbm_set_populations", "elbm_reduce", "elbm_sync", "elbm_cells",
           "elbm_steps_done", "elbm_omega", "elbm_device_bytes", "elbm_launch_count", "elbm_get_u_ref",
           "elbm_last_error", "elbm_batch_create", "elbm_batch_step", "elbm_batch_info", "elbm_batch_destroy",
           "elbm_batch_add", "elbm_batch_remove", "elbm_batch_size",
           "elbm_step_noalloc", "elbm_selftest_wait_timeout", "elbm_mode_sums", "elbm_kernel_form",
           "elbm_batch_tuning", "elbm_batch_set_config", "elbm_selftest_counter_timeout"]


class ElbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"elbm error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed and allowed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"elbm CUDA library not found at {path}; run build() first")
        L = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.elbm_create.argtypes = [ip, ip, ip, ip, ctypes.POINTER(dp), dp, dp, ip, vp, ctypes.POINTER(vp)]
        L.elbm_destroy.argtypes = [vp]
        L.elbm_destroy.restype = None
        L.elbm_set_option.argtypes = [vp, ip, dp]
        L.elbm_init.argtypes = [vp, vp, vp, ip, ip]
        L.elbm_step.argtypes = [vp, ip]
        L.elbm_moments.argtypes = [vp, vp, vp, ip, ip]
        L.elbm_get_populations.argtypes = [vp, vp, ip, ip]
        L.elbm_set_populations.argtypes = [vp, vp, ip, ip]
        L.elbm_reduce.argtypes = [vp, ctypes.POINTER(dp)]
        L.elbm_sync.argtypes = [vp]
        for name in ("elbm_cells", "elbm_steps_done", "elbm_device_bytes", "elbm_launch_count"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = ctypes.c_longlong
        L.elbm_omega.argtypes = [vp]
        L.elbm_omega.restype = dp
        L.elbm_get_u_ref.argtypes = [vp, ctypes.POINTER(dp)]
        L.elbm_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
        L.elbm_batch_step.argtypes = [vp, ip]
        L.elbm_selftest_wait_timeout.argtypes = [ip, vp]
        L.elbm_selftest_counter_timeout.argtypes = [ip, vp]
        L.elbm_mode_sums.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(dp)]
        L.elbm_kernel_form.argtypes = [vp, ctypes.POINTER(ip)]
        L.elbm_batch_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_longlong)]
        L.elbm_batch_tuning.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip),
                                         ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.elbm_batch_set_config.argtypes = [vp, ip]
        L.elbm_batch_add.argtypes = [vp, vp]
        L.elbm_batch_remove.argtypes = [vp, vp]
        L.elbm_batch_size.argtypes = [vp]
        L.elbm_batch_destroy.argtypes = [vp]
        L.elbm_batch_destroy.restype = None
        L.elbm_last_error.argtypes = []
        L.elbm_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc):
    if rc != 0:
        raise ElbmError(rc, load().elbm_last_error().decode(errors="replace"))


def _buffer(a, dtype):
    """(pointer, on_device, dtype code) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            code = {torch.float32: DTYPE_F32, torch.float64: DTYPE_F64}[a.dtype]
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), code
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype not in (np.float32, np.float64):
        arr = arr.astype(dtype)
    arr = np.ascontiguousarray(arr)
    code = DTYPE_F64 if arr.dtype == np.float64 else DTYPE_F32
    return arr, 0, code


class Solver:
    """One grid on the GPU, advanced by the extended LBGK step: periodic, or
    with half-way bounce-back walls in y (``walls_y``) and a constant body
    force ``force`` = (g_x, g_y, g_z)."""

    def __init__(self, lattice, n, stretch=(1.0, 1.0, 1.0), T=1.0 / 3.0, nu=0.01, storage=F32,
                 stream=None, kernel=0, equilibrium=0, u_ref=None, walls_y=False, force=None):
        L = load()
        self.lattice = lattice
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = lattice
        n = tuple(int(v) for v in n)
        if self.D == 2:
            n = (n[0], n[1], 1)
        self.n = n
        self.N = n[0] * n[1] * n[2]
        if isinstance(storage, str):
            storage = STORAGE_NAMES[storage]
        self.storage = storage
        st = (ctypes.c_double * 3)(*[float(v) for v in (list(stretch) + [1.0] * 3)[:3]])
        h = ctypes.c_void_p()
        if stream is None:
            stream_ptr = None
        elif isinstance(stream, int):
            stream_ptr = ctypes.c_void_p(stream)
        else:
            stream_ptr = ctypes.c_void_p(stream.cuda_stream)
        _check(L.elbm_create(lattice, n[0], n[1], n[2], st, float(T), float(nu), int(storage),
                             stream_ptr, ctypes.byref(h)))
        self._h = h
        self.stretch = tuple(st)
        self.T = T
        self.nu = nu
        if kernel:
            self.set_option(OPT_KERNEL, kernel)
        if equilibrium:
            self.set_option(OPT_EQUILIBRIUM, equilibrium)
        if walls_y:
            self.set_option(OPT_WALLS_Y, 1)
        if force is not None:
            for a, v in enumerate(force):
                self.set_option(OPT_FORCE_X + a, float(v))
        if isinstance(u_ref, str) and u_ref == "mean":
            self.set_option(OPT_U_REF_AUTO, 1)
        elif u_ref is not None:
            for a, v in enumerate(u_ref):
                self.set_option(OPT_U_REF_X + a, float(v))

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().elbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- shapes ---------------------------------------------------------
    @property
    def shape(self):
        nx, ny, nz = self.n
        return (ny, nx) if self.D == 2 else (nz, ny, nx)

    # -- calls ----------------------------------------------------------
    def set_option(self, key, value):
        _check(load().elbm_set_option(self._h, int(key), float(value)))

    def init(self, rho, u):
        r, on_r, code = _buffer(rho, np.float64)
        v, on_u, code_u = _buffer(u, np.float64)
        if on_r != on_u or code != code_u:
            raise ValueError("rho and u must live on the same side and share a dtype")
        _check(load().elbm_init(self._h, _addr(r), _addr(v), code, on_r))

    def step(self, n=1):
        _check(load().elbm_step(self._h, int(n)))

    def sync(self):
        _check(load().elbm_sync(self._h))

    def moments(self, rho=None, u=None, dtype=np.float64):
        """(rho, u) of the current state; into the given buffers if provided."""
        if rho is None:
            rho = np.empty(self.shape, dtype=dtype)
            u = np.empty((self.D,) + self.shape, dtype=dtype)
        r, on_r, code = _buffer(rho, dtype)
        v, on_u, _ = _buffer(u, dtype)
        _check(load().elbm_moments(self._h, _addr(r), _addr(v), code, on_r))
        return rho, u

    def get_populations(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty((self.Q,) + self.shape, dtype=dtype)
        b, on, code = _buffer(out, dtype)
        _check(load().elbm_get_populations(self._h, _addr(b), code, on))
        return out

    def set_populations(self, f):
        b, on, code = _buffer(f, np.float64)
        _check(load().elbm_set_populations(self._h, _addr(b), code, on))

    def mode_amplitude(self, k, direction):
        """Amplitude 2 |sum_x (u . s) exp(-i k . x)| / N of one Fourier mode of
        the velocity, accumulated in FP64 on the GPU (k in physical units)."""
        kk = (ctypes.c_double * 3)(*[float(v) for v in (list(k) + [0.0] * 3)[:3]])
        dd = (ctypes.c_double * 3)(*[float(v) for v in (list(direction) + [0.0] * 3)[:3]])
        out = (ctypes.c_double * 2)()
        _check(load().elbm_mode_sums(self._h, kk, dd, out))
        return 2.0 * float(np.hypot(out[0], out[1])) / self.N

    def reduce(self, raise_nonfinite=True):
        out = (ctypes.c_double * NRED)()
        rc = load().elbm_reduce(self._h, out)
        vals = dict(zip(RED_NAMES, list(out)))
        if rc != 0 and not (rc == -5 and not raise_nonfinite):
            _check(rc)
        return vals

    @property
    def u_ref(self):
        out = (ctypes.c_double * 3)()
        _check(load().elbm_get_u_ref(self._h, out))
        return tuple(out)[: self.D]

    @property
    def kernel_form(self):
        """(form, variant) of the next step: form 1 two-pass, 2 graph-pipelined,
        3 single pass; variant (form 3) 1 TMEM, 2 TMA, 3 cp.async-staged."""
        v = ctypes.c_int()
        form = load().elbm_kernel_form(self._h, ctypes.byref(v))
        if form < 0:
            _check(form)
        return form, v.value

    @property
    def omega(self):
        return load().elbm_omega(self._h)

    @property
    def steps_done(self):
        return load().elbm_steps_done(self._h)

    @property
    def device_bytes(self):
        return load().elbm_device_bytes(self._h)

    @property
    def launches(self):
        return load().elbm_launch_count(self._h)

    @property
    def handle(self):
        return self._h


class Batch:
    """Solvers of one lattice, storage mode, stream and kernel form advanced
    together.  Two-pass members: two launches per step for the whole batch,
    replayed from a CUDA graph.  Single-pass members (kernel=3): each member's
    step sequence is a CUDA graph of its own, replayed side by side with the
    others on private streams of the batch."""

    def __init__(self, solvers):
        L = load()
        self.solvers = list(solvers)  # the batch refers to them; keep them alive
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.handle.value for s in self.solvers])
        h = ctypes.c_void_p()
        _check(L.elbm_batch_create(arr, len(self.solvers), ctypes.byref(h)))
        self._h = h

    def step(self, n=1):
        _check(load().elbm_batch_step(self._h, int(n)))

    def add(self, solver):
        _check(load().elbm_batch_add(self._h, solver.handle))
        self.solvers.append(solver)

    def remove(self, solver):
        _check(load().elbm_batch_remove(self._h, solver.handle))
        self.solvers.remove(solver)

    def __len__(self):
        return load().elbm_batch_size(self._h)

    def info(self):
        bs = ctypes.c_int()
        ms = (ctypes.c_double * 2)()
        launches = ctypes.c_longlong()
        _check(load().elbm_batch_info(self._h, ctypes.byref(bs), ms, ctypes.byref(launches)))
        return {"block_size": bs.value, "tuned_ms": {128: ms[0], 256: ms[1]}, "launches": launches.value}

    def set_config(self, config):
        """Single-pass batches: pin the configuration (0..11 flattened launch,
        12 per-member graphs; see elbm_batch_tuning) or return to the
        autotuner (-1)."""
        _check(load().elbm_batch_set_config(self._h, int(config)))

    def tuning(self):
        """Single-pass batches: the configuration of the last step and the
        autotuner's two-step timings (ms, -1 for a candidate not yet timed)."""
        c, rows, seg, inter = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * BATCH_CONFIGS)()
        rc = load().elbm_batch_tuning(self._h, ctypes.byref(c), ctypes.byref(rows), ctypes.byref(seg),
                                      ctypes.byref(inter), ms)
        if rc < 0:
            _check(rc)
        return {"config": c.value, "tile_rows": rows.value, "seg_planes": seg.value,
                "interleaved": bool(inter.value), "member_graphs": c.value == BATCH_CONFIGS - 1,
                "tuned": rc == 0, "ms": list(ms)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().elbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _addr(b):
    if isinstance(b, np.ndarray):
        return ctypes.c_void_p(b.ctypes.data)
    return b


def selftest_wait_timeout(limit_ms=50, stream=None, counter=False):
    """Run one of the library's bounded device-side waits on something that
    never happens -- an mbarrier phase (the TMA-fed kernels' wait) or, with
    counter=True, a progress counter (the fused in-place form's wait);
    returns the error code (ELBM_ERR_TIMEOUT, -6, when it gave up as
    designed) and the library's message."""
    L = load()
    sp = None if stream is None else ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    fn = L.elbm_selftest_counter_timeout if counter else L.elbm_selftest_wait_timeout
    rc = fn(int(limit_ms), sp)
    return rc, L.elbm_last_error().decode()
