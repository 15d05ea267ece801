"""Seeded synthetic lattice inputs shared by the tests and the benchmark.

This module only draws field configurations (numpy, float64); it contains
none of the method's arithmetic (no kicks, drifts, windings or sums), so both
the FP64 oracle and the CUDA library can be fed from it without sharing code.

Every state is an array of shape (20, nz, ny, nx) in the field order used by
both sides: phi_re, phi_im, psi_re, psi_im, A_0..2, B_0..2, Pi_re, Pi_im,
Psi_re, Psi_im, E_0..2, H_0..2.

The shapes and value ranges follow the paper's workloads (Sec. III-V): unit
vacuum expectation values, dx = 0.5, random phases at every site, and gauge
fields of order one once the network has formed.
"""
from __future__ import annotations

import numpy as np

NFIELDS = 20


def _grid(shape):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return X.astype(np.float64), Y.astype(np.float64), Z.astype(np.float64)


def random_state(shape, seed, mod_lo=0.2, mod_hi=1.6, a_amp=1.5, mom_amp=1.0):
    """Generic rough state: |phi| uniform in [mod_lo, mod_hi), uniform phases,
    links uniform in [-a_amp, a_amp), momenta and electric fields uniform in
    [-mom_amp, mom_amp).  Used where the test needs every code path exercised
    (windings of all signs, large gradients, non-zero currents)."""
    rng = np.random.default_rng(seed)
    st = np.zeros((NFIELDS,) + tuple(shape))
    for s in range(2):
        r = rng.uniform(mod_lo, mod_hi, size=shape)
        th = rng.uniform(0.0, 2.0 * np.pi, size=shape)
        st[2 * s] = r * np.cos(th)
        st[2 * s + 1] = r * np.sin(th)
    st[4:10] = rng.uniform(-a_amp, a_amp, size=(6,) + tuple(shape))
    st[10:20] = rng.uniform(-mom_amp, mom_amp, size=(10,) + tuple(shape))
    return st


def smooth_state(shape, seed, kmax=2, amp=0.3, a_amp=0.2):
    """Long-wavelength state: vacuum modulus plus a few low-k Fourier modes in
    every field, zero momenta.  Used where time-step errors must be small."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _grid(shape)
    nz, ny, nx = shape
    st = np.zeros((NFIELDS,) + tuple(shape))
    st[0] = 1.0
    st[2] = 1.0
    for f in range(10):
        a = amp if f < 4 else a_amp
        for _ in range(3):
            kx, ky, kz = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            st[f] += a * rng.uniform(-1, 1) * np.cos(
                2 * np.pi * (kx * X / nx + ky * Y / ny + kz * Z / nz) + ph)
    return st


def vortex_map(shape, sigma=1.0):
    """phi = sigma [sin(2 pi (X + 1/2) / nx) + i sin(2 pi (Y + 1/2) / ny)]:
    four straight z-directed zero lines between lattice sites, at
    X + 1/2 in {0, nx/2} and Y + 1/2 in {0, ny/2}, with windings
    +1 at (0, 0), -1 at (nx/2, 0), -1 at (0, ny/2), +1 at (nx/2, ny/2).
    Returns the complex field (nz, ny, nx)."""
    X, Y, _ = _grid(shape)
    nz, ny, nx = shape
    return sigma * (np.sin(2 * np.pi * (X + 0.5) / nx) + 1j * np.sin(2 * np.pi * (Y + 0.5) / ny))


def crossing_vortices(shape, sigma=1.0):
    """Product of the four-string map in the (x, y) plane and the same map in
    the (y, z) plane: four z-directed and four x-directed straight strings,
    which pass through common cells at the 8 positions
    X + 1/2 in {0, nx/2}, Y + 1/2 in {0, ny/2}, Z + 1/2 in {0, nz/2}."""
    X, Y, Z = _grid(shape)
    nz, ny, nx = shape
    fxy = np.sin(2 * np.pi * (X + 0.5) / nx) + 1j * np.sin(2 * np.pi * (Y + 0.5) / ny)
    fyz = np.sin(2 * np.pi * (Y + 0.5) / ny) + 1j * np.sin(2 * np.pi * (Z + 0.5) / nz)
    return sigma * fxy * fyz


def gauge_parameter(shape, seed):
    """Uniform random gauge angle Lambda in [0, 2 pi) per site."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * np.pi, size=shape)


def site_sample(shape, count, seed):
    """Distinct random sites (z, y, x) of a box, as an int64 array (count, 3)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    flat = rng.choice(nz * ny * nx, size=min(count, nz * ny * nx), replace=False)
    z, rem = np.divmod(flat, ny * nx)
    y, x = np.divmod(rem, nx)
    return np.stack([z, y, x], axis=1).astype(np.int64)


def sparse_cells(shape, density, seed):
    """Random cell array (uint8, values 2 or 4) with the given occupancy."""
    rng = np.random.default_rng(seed)
    occ = rng.random(shape) < density
    return (occ * rng.choice([2, 4], size=shape, p=[0.9, 0.1])).astype(np.uint8)
