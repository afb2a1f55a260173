"""Seeded synthetic initial conditions shared by the tests, the benchmark and
the oracle checks.

This module holds no arithmetic of the lattice-Boltzmann method: it only
builds initial fields (phi, and optionally rho and u) on the host, in float64,
with site order s = x + nx*(y + ny*z) and arrays shaped (nz, ny, nx). Both the
CUDA path and the oracle start from the same arrays.

Random numbers use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): U(s) = (splitmix64(seed XOR
s*GOLDEN) >> 11) * 2^-53, one draw per site.
"""

from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each uint64 state (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = state.astype(np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(n: int, seed: int) -> np.ndarray:
    """n doubles in [0, 1), one SplitMix64 draw per index."""
    s = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) ^ (s * GOLDEN)
    bits = splitmix64(state) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53)


def spinodal_phi(nx: int, ny: int, nz: int, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """phi = amplitude * (2U - 1): uniform noise in [-amplitude, amplitude)."""
    u = uniform01(nx * ny * nz, seed)
    return (amplitude * (2.0 * u - 1.0)).reshape(nz, ny, nx)


def droplet_phi(nx: int, ny: int, nz: int, radius: float, phi0: float, xi: float) -> np.ndarray:
    """phi0 * tanh((R - r)/xi), r the distance to the lattice centre (nx/2, ny/2, nz/2)."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - nz / 2.0) ** 2)
    return phi0 * np.tanh((radius - r) / xi)


def slab_phi(nx: int, ny: int, nz: int, phi0: float, width_fraction: float = 0.5) -> np.ndarray:
    """Sharp slab along x: +phi0 for x in [nx/4, nx/4 + width*nx), -phi0 elsewhere
    (two flat interfaces normal to x)."""
    x = np.arange(nx)
    lo = nx // 4
    hi = lo + int(round(width_fraction * nx))
    prof = np.where((x >= lo) & (x < hi), phi0, -phi0).astype(np.float64)
    return np.broadcast_to(prof, (nz, ny, nx)).copy()


def sine_phi(nx: int, ny: int, nz: int, amplitude: float, mode: int = 1) -> np.ndarray:
    """amplitude * sin(2 pi mode x / nx), constant in y and z."""
    x = np.arange(nx)
    prof = amplitude * np.sin(2.0 * math.pi * mode * x / nx)
    return np.broadcast_to(prof, (nz, ny, nx)).copy()


def shear_wave_u(nx: int, ny: int, nz: int, u0: float, mode: int = 1) -> np.ndarray:
    """Velocity (3, nz, ny, nx) with u_x = u0 sin(2 pi mode y / ny), u_y = u_z = 0."""
    y = np.arange(ny)
    ux = u0 * np.sin(2.0 * math.pi * mode * y / ny)
    u = np.zeros((3, nz, ny, nx))
    u[0] = ux[None, :, None]
    return u


def random_q(nx: int, ny: int, nz: int, seed: int, amplitude: float = 0.15) -> np.ndarray:
    """Five Q-tensor components (xx, xy, xz, yy, yz) per site, each uniform in
    [-amplitude, amplitude) from its own seed (seed, seed + 1, ...), shaped
    (5, nz, ny, nx): a disordered liquid-crystal start."""
    n = nx * ny * nz
    return np.stack([(amplitude * (2.0 * uniform01(n, seed + k) - 1.0)).reshape(nz, ny, nx) for k in range(5)])
