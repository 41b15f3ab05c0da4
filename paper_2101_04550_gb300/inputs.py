"""Seeded synthetic initial conditions of the paper's flows (Sec. III).

These generators hold none of the method's arithmetic: they only produce the
density and velocity fields that both the CUDA library and the FP64 oracle
start from.  Fields use the library layout: ``rho`` has shape ``(ny, nx)`` or
``(nz, ny, nx)``; ``u`` has shape ``(D,) + rho.shape``.  Node ``(i, j, k)`` sits
at the physical position ``(i lam_x, j lam_y, k lam_z)`` (node spacing equals
the stretch factor, Eq. d3q27velSTRETCHED with delta t = 1).
"""
from __future__ import annotations

import numpy as np


def _coords(n, lam):
    """Physical coordinates (x, y[, z]) broadcast to the field shape."""
    D = len(n)
    axes = [np.arange(n[a], dtype=np.float64) * lam[a] for a in range(D)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # (z,) y, x order
    return grids[::-1]  # x, y[, z]


def uniform(n, u0, rho0=1.0):
    D = len(n)
    shape = tuple(n[::-1])
    rho = np.full(shape, rho0)
    u = np.zeros((D,) + shape)
    for a in range(D):
        u[a] = u0[a]
    return rho, u


def shear_wave(n, lam=(1.0, 1.0, 1.0), k_dir=(1, 0, 0), shear_dir=(0, 1, 0),
               amplitude=1e-3, advection=0.0, rho0=1.0):
    """Plane shear wave u = U k_hat + a sin(k . x) s_hat (Sec. III.A).

    ``k_dir`` is an integer vector of periods per box along each axis, so the
    wave is periodic on the box; ``shear_dir`` must be orthogonal to the
    physical wave vector (it is normalised here).  The advection velocity U
    points along the wave vector, as in the axis-aligned setup of Sec. III.A.
    Returns (rho, u, k_phys, s_hat) with k_phys the physical wave vector.
    """
    D = len(n)
    L = [n[a] * lam[a] for a in range(D)]
    k = np.array([2.0 * np.pi * k_dir[a] / L[a] for a in range(D)])
    s = np.array(shear_dir[:D], dtype=np.float64)
    s = s - k * (s @ k) / (k @ k)  # keep it exactly transverse
    s /= np.linalg.norm(s)
    khat = k / np.linalg.norm(k)
    X = _coords(n, lam)
    phase = sum(k[a] * X[a] for a in range(D))
    shape = tuple(n[::-1])
    rho = np.full(shape, rho0)
    u = np.zeros((D,) + shape)
    for a in range(D):
        u[a] = advection * khat[a] + amplitude * np.sin(phase) * s[a]
    return rho, u, k, s


def taylor_green_2d(n, lam=(1.0, 1.0), U=0.01, advection=(0.0, 0.0), rho0=1.0):
    """u_x = U sin(kx) cos(ky), u_y = -U cos(kx) sin(ky) on a physically square box."""
    X = _coords(n, lam)
    Lx, Ly = n[0] * lam[0], n[1] * lam[1]
    kx, ky = 2 * np.pi / Lx, 2 * np.pi / Ly
    shape = tuple(n[::-1])
    rho = np.full(shape, rho0)
    u = np.zeros((2,) + shape)
    u[0] = U * np.sin(kx * X[0]) * np.cos(ky * X[1]) + advection[0]
    u[1] = -U * (kx / ky) * np.cos(kx * X[0]) * np.sin(ky * X[1]) + advection[1]
    return rho, u, (kx, ky)


def taylor_green_3d(n, lam=(1.0, 1.0, 1.0), U=0.01, rho0=1.0):
    """u = U (sin x cos y cos z, -cos x sin y cos z, 0) scaled to the box."""
    X = _coords(n, lam)
    k = [2 * np.pi / (n[a] * lam[a]) for a in range(3)]
    shape = tuple(n[::-1])
    rho = np.full(shape, rho0)
    u = np.zeros((3,) + shape)
    u[0] = U * np.sin(k[0] * X[0]) * np.cos(k[1] * X[1]) * np.cos(k[2] * X[2])
    u[1] = -U * (k[0] / k[1]) * np.cos(k[0] * X[0]) * np.sin(k[1] * X[1]) * np.cos(k[2] * X[2])
    return rho, u


def double_shear_layer(n, U=0.2, kappa=80.0, delta=0.05, rho0=1.0):
    """Periodic double shear layer (Sec. III.C) on a physically square domain.

    With normalised coordinates x/L = i/nx and y/L = j/ny the field is the
    same for a cubic and a stretched lattice of the same physical size.
    """
    nx, ny = n
    xs = np.arange(nx) / nx
    ys = np.arange(ny) / ny
    Y, Xg = np.meshgrid(ys, xs, indexing="ij")
    ux = np.where(Y <= 0.5, U * np.tanh(kappa * (Y - 0.25)), U * np.tanh(kappa * (0.75 - Y)))
    uy = delta * U * np.sin(2 * np.pi * (Xg + 0.25))
    rho = np.full((ny, nx), rho0)
    return rho, np.stack([ux, uy])


def isotropic_turbulence(n, seed=0, k0=4.0, u_rms=0.08, rho0=1.0):
    """Seeded solenoidal random field with E(k) ~ k^4 exp(-2 (k/k0)^2) (Sec. III.B).

    Gaussian white noise per component (numpy PCG64, ``seed``) is filtered in
    Fourier space by sqrt(E(k) / (4 pi k^2)) with k the integer box wavenumber,
    projected onto divergence-free modes, transformed back in float64 and
    scaled so that the per-component rms velocity sqrt(<u.u>/3) equals u_rms.
    """
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((3, nz, ny, nx))
    uh = np.fft.fftn(noise, axes=(1, 2, 3))
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    kk = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(kk > 0, np.sqrt(kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2) / (4 * np.pi * k2)), 0.0)
        kdotu = KX * uh[0] + KY * uh[1] + KZ * uh[2]
        proj = np.where(k2 > 0, kdotu / np.where(k2 > 0, k2, 1.0), 0.0)
    uh[0] = (uh[0] - KX * proj) * amp
    uh[1] = (uh[1] - KY * proj) * amp
    uh[2] = (uh[2] - KZ * proj) * amp
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    scale = u_rms / np.sqrt((u ** 2).sum(axis=0).mean() / 3.0)
    u *= scale
    rho = np.full((nz, ny, nx), rho0)
    return rho, u


def channel(n, lam=(2.0, 1.0, 2.0), u_center=0.1, perturbation=0.05, seed=0, rho0=1.0):
    """Laminar Poiseuille profile between walls at y = -1/2 and y = ny - 1/2
    (half-way bounce-back) plus a seeded uniform-random perturbation of
    relative size ``perturbation`` on every component (Sec. III.E)."""
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    yc = (np.arange(ny) + 0.5) / ny  # wall-to-wall coordinate in (0, 1)
    prof = 4.0 * u_center * yc * (1.0 - yc)
    u = np.zeros((3, nz, ny, nx))
    u[0] = prof[None, :, None]
    u += perturbation * u_center * (2.0 * rng.random((3, nz, ny, nx)) - 1.0)
    rho = np.full((nz, ny, nx), rho0)
    return rho, u
