"""Seeded synthetic inputs for the two-phase lattice Boltzmann workloads.

This module is shared by the library's users (tests, benchmark) and by the
CPU oracle's callers; it holds none of the method's arithmetic.  It only draws
density/velocity fields of the shapes the paper's experiments use (Sec. 3):
flat liquid slabs (Sec. 3.1.1), static drops (Sec. 3.1.2) and a drop falling
on a thin film (Secs. 3.2-3.3), with a tanh interface of width W and seeded
noise.  The coexistence densities are arguments; nothing here evaluates the
equation of state.

Arrays are float64, indexed [z, y, x] (a leading axis of length 1 in 2-D); a
velocity field has a further leading component axis of length D.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20220128


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def tanh_profile(dist, rho_l, rho_v, W):
    """Density across an interface; dist < 0 inside the liquid, dist = 0 on the
    interface, W the interface width."""
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * dist / W)


def liquid_fraction(dist, W):
    return 0.5 - 0.5 * np.tanh(2.0 * dist / W)


def drop(shape, center, R, rho_l, rho_v, W, D=2):
    """Static drop of radius R (circle in 2-D, sphere in 3-D)."""
    x, y, z = _grid(shape)
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    if D == 3:
        r2 = r2 + (z - center[2]) ** 2
    return tanh_profile(np.sqrt(r2) - R, rho_l, rho_v, W)


def slab(shape, axis, lo, hi, rho_l, rho_v, W):
    """Liquid between lo and hi along `axis` (0 = x, 1 = y, 2 = z), periodic-friendly."""
    coord = _grid(shape)[axis]
    dist = np.maximum(lo - coord, coord - hi)
    return tanh_profile(dist, rho_l, rho_v, W)


def drop_on_film(shape, D, R, h, U, rho_l, rho_v, W, gap=None):
    """A drop of radius R falling at speed U onto a liquid film of thickness h on
    the bottom wall (the last axis of the domain: y in 2-D, z in 3-D).  The drop
    centre sits at height h + R + gap over the film, horizontally centred.
    Returns (rho, u) with u of shape (D,) + shape."""
    nz, ny, nx = shape
    x, y, z = _grid(shape)
    vert = y if D == 2 else z
    gap = 2.0 * W if gap is None else gap
    cv = h + R + gap
    if D == 2:
        r = np.sqrt((x - 0.5 * (nx - 1)) ** 2 + (y - cv) ** 2)
    else:
        r = np.sqrt((x - 0.5 * (nx - 1)) ** 2 + (y - 0.5 * (ny - 1)) ** 2 + (z - cv) ** 2)
    d_drop = r - R
    d_film = vert - (h - 0.5)  # the wall is half-way below the first node
    dist = np.minimum(d_drop, d_film)
    rho = tanh_profile(dist, rho_l, rho_v, W)
    u = np.zeros((D,) + tuple(shape))
    u[D - 1] = -U * liquid_fraction(d_drop, W)
    return rho, u


def uniform_noise(shape, amplitude, seed):
    return rng(seed).uniform(-amplitude, amplitude, size=shape)


def shear_wave(shape, D, rho0, U, axis_u=0, axis_k=1):
    """u_{axis_u} = U sin(2 pi k / L) along axis_k, uniform density."""
    coord = _grid(shape)[axis_k]
    L = shape[::-1][axis_k]
    u = np.zeros((D,) + tuple(shape))
    u[axis_u] = U * np.sin(2.0 * np.pi * coord / L)
    return np.full(shape, rho0, dtype=np.float64), u


def perturbed_populations(base, rel_amplitude, seed):
    """Multiply each population by (1 + eps), eps uniform in +-rel_amplitude: a
    non-equilibrium state for single-step parity tests."""
    return base * (1.0 + rng(seed).uniform(-rel_amplitude, rel_amplitude, size=base.shape))
