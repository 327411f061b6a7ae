"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds no arithmetic of the method: fields are built directly in conservative
variables from a few random Fourier modes (smooth) or per-cell noise (rough),
with amplitudes that keep density and internal energy positive.
"""
import numpy as np


def smooth_field(shape, rng, nmodes=4, lengths=(2 * np.pi,) * 3):
    """Sum of random low Fourier modes, periodic on the box, max |f| <= 1."""
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) / nz
    y = (np.arange(ny) + 0.5) / ny
    x = (np.arange(nx) + 0.5) / nx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros(shape)
    for _ in range(nmodes):
        k = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.uniform(-1, 1) * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
    m = np.abs(f).max()
    return f / m if m > 0 else f


def smooth_state(n, seed, e0=3.0):
    """Conservative state [5][nz][ny][nx] with smooth random perturbations."""
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    q = np.empty((5,) + shape)
    q[0] = 1.0 + 0.1 * smooth_field(shape, rng)
    for c in (1, 2, 3):
        q[c] = 0.3 * smooth_field(shape, rng)
    q[4] = e0 + 0.2 * smooth_field(shape, rng)
    return q


def rough_state(n, seed, e0=3.0):
    """Conservative state with independent per-cell noise (exercises the nonlinear WENO weights)."""
    rng = np.random.default_rng(seed)
    shape = (5, n[2], n[1], n[0])
    q = np.empty(shape)
    q[0] = 1.0 + 0.05 * rng.uniform(-1, 1, shape[1:])
    for c in (1, 2, 3):
        q[c] = 0.1 * rng.uniform(-1, 1, shape[1:])
    q[4] = e0 + 0.1 * rng.uniform(-1, 1, shape[1:])
    return q
