"""Test-side flow diagnostics (numpy, float64): Fourier amplitude of a shear
wave and exponential-decay fits.  Used for the oracle's physics pins and for
the GPU viscosity checks alike."""
import numpy as np


def mode_amplitude(u, k, s, lam):
    """A = (2/N) |sum_x (u . s) exp(-i k . x)| with x the physical node position."""
    D = u.shape[0]
    shape = u.shape[1:]
    n = shape[::-1]
    axes = [np.arange(n[a]) * lam[a] for a in range(D)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    phase = sum(k[a] * grids[a] for a in range(D))
    up = sum(u[a] * s[a] for a in range(D))
    return 2.0 * abs(np.sum(up * np.exp(-1j * phase))) / up.size


def decay_rate(ts, values, t_min=0):
    ts = np.asarray(ts, dtype=np.float64)
    values = np.asarray(values, dtype=np.float64)
    m = ts >= t_min
    return -np.polyfit(ts[m], np.log(values[m]), 1)[0]
