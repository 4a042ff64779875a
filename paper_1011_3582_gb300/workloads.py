"""Seeded synthetic initial fields shaped like the paper's workloads
(arXiv:1011.3582, Sec. 3 and Sec. 4): planar liquid-vapour slabs, circular
droplets, a triangular droplet and spinodal decomposition from noise.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  It holds none of the method's arithmetic: it only lays out
initial (rho, u_x, u_y, T) fields from numbers the caller supplies
(coexistence densities, temperatures, radii).  Random numbers come from
numpy's PCG64 generator (``numpy.random.default_rng(seed)``), drawn once on
the host; the same float64 arrays are handed to both implementations.

All fields are float64 arrays of shape (ny, nx), row-major, x fastest.
Lengths are in lattice units (sites).
"""
from __future__ import annotations

import numpy as np


def _grid(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def uniform(nx, ny, rho, T, ux=0.0, uy=0.0):
    """Spatially uniform state."""
    shape = (ny, nx)
    return (np.full(shape, float(rho)), np.full(shape, float(ux)),
            np.full(shape, float(uy)), np.full(shape, float(T)))


def slab(nx, ny, rho_v, rho_l, T, y1=None, y2=None, width=2.0,
         noise=0.0, seed=42, axis="y"):
    """Planar slab of liquid (rho_l) between y1 and y2 in vapour (rho_v):
        rho = rho_v + (rho_l - rho_v) [tanh((y - y1)/w) - tanh((y - y2)/w)] / 2
    plus additive uniform noise U(-noise, +noise) on rho.  Defaults put the
    liquid in the central half (y1 = n/4, y2 = 3n/4).  axis='x' lays the
    slab across x instead (the 512x4 geometry of Sec. 4.1)."""
    x, y = _grid(nx, ny)
    c, n = (y, ny) if axis == "y" else (x, nx)
    y1 = n / 4.0 if y1 is None else float(y1)
    y2 = 3.0 * n / 4.0 if y2 is None else float(y2)
    rho = rho_v + (rho_l - rho_v) * 0.5 * (np.tanh((c - y1) / width)
                                           - np.tanh((c - y2) / width))
    if noise:
        rng = np.random.default_rng(seed)
        rho = rho + rng.uniform(-noise, noise, size=rho.shape)
    z = np.zeros_like(rho)
    return rho, z, z.copy(), np.full_like(rho, float(T))


def droplet(nx, ny, R, rho_in, rho_out, T, width=2.0, center=None):
    """Circular drop of radius R: rho = rho_out + (rho_in - rho_out)
    [1 - tanh((r - R)/w)] / 2, centred on the grid by default."""
    x, y = _grid(nx, ny)
    cx, cy = (nx / 2.0, ny / 2.0) if center is None else center
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    rho = rho_out + (rho_in - rho_out) * 0.5 * (1.0 - np.tanh((r - R) / width))
    z = np.zeros_like(rho)
    return rho, z, z.copy(), np.full_like(rho, float(T))


def triangle(nx, ny, side, rho_in, rho_out, T):
    """Equilateral triangular drop with a sharp edge, centred (Sec. 4.2)."""
    x, y = _grid(nx, ny)
    cx, cy = nx / 2.0, ny / 2.0
    h = side * np.sqrt(3.0) / 2.0
    # vertices: apex up; inside = below both slanted edges and above the base
    yb = cy - h / 3.0
    inside = (y >= yb) & (y <= yb + h) \
        & (np.abs(x - cx) <= (yb + h - y) / np.sqrt(3.0))
    rho = np.where(inside, float(rho_in), float(rho_out))
    z = np.zeros_like(rho)
    return rho, z, z.copy(), np.full_like(rho, float(T))


def spinodal(nx, ny, rho_c, T, amp=0.01, seed=7):
    """Spinodal decomposition from noise: rho = rho_c (1 + amp N(0, 1))."""
    rng = np.random.default_rng(seed)
    rho = rho_c * (1.0 + amp * rng.standard_normal((ny, nx)))
    z = np.zeros_like(rho)
    return rho, z, z.copy(), np.full_like(rho, float(T))


def smooth_random(nx, ny, seed=0, rho0=1.0, T0=0.9, amp=0.05, umax=0.02, modes=3):
    """Smooth random periodic fields (a few low Fourier modes): used for
    identity and parity checks away from equilibrium."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)

    def field():
        g = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(-3, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            g += np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
        return g / modes

    rho = rho0 * (1.0 + amp * field())
    ux = umax * field()
    uy = umax * field()
    T = T0 * (1.0 + 0.5 * amp * field())
    return rho, ux, uy, T


def sweep_plan(nruns=64, seed=3, sizes=(128, 256, 384, 512), tr_range=(0.70, 0.99)):
    """Phase-diagram sweep: for each run a square grid drawn from `sizes` and
    a reduced temperature drawn uniformly from `tr_range` (numpy PCG64,
    one generator for the whole plan).  Returns [(n, T_r), ...]."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=nruns)
    trs = rng.uniform(tr_range[0], tr_range[1], size=nruns)
    return [(int(n), float(t)) for n, t in zip(ns, trs)]
