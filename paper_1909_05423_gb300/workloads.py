"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the solver: it only draws random fields and
samples manufactured solutions and their continuous Laplacians at cell centres.
Both the tests (GPU path and CPU oracle) and the benchmark draw their inputs
from here, so the two sides always see identical data.

Grids are real arrays of shape (nz, ny, nx), x fastest, cell centres at
x_i = (i + 1/2) * dx on the domain [0, nx*dx).
"""
from __future__ import annotations

import numpy as np


def cell_centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def uniform_source(shape, seed: int, remove_mean: bool = True) -> np.ndarray:
    """i.i.d. U[-1, 1] source (the random-source timing workloads), optionally mean-free."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, size=shape)
    if remove_mean:
        f -= f.mean()
    return np.ascontiguousarray(f)


def _axis_mode(kind: str, kappa: float, x: np.ndarray):
    """Per-axis factor and its second derivative factor (-kappa^2) for the MMS products."""
    if kind == "sin":
        return np.sin(kappa * x)
    if kind == "cos":
        return np.cos(kappa * x)
    raise ValueError(kind)


def manufactured(shape, spacing, terms):
    """u* = sum_t amp_t * fx(kx x) fy(ky y) fz(kz z) and f = Laplacian(u*) (continuous).

    ``terms`` is a list of (amp, (fx, kx), (fy, ky), (fz, kz)) with f. in {"sin", "cos"}.
    Returns (u_star, f) sampled at cell centres.  The paper's sign convention is used:
    the solver solves Laplacian(u) = f, so f = -(kx^2+ky^2+kz^2) u* for each term.
    """
    nz, ny, nx = shape
    dx, dy, dz = spacing
    x = cell_centres(nx, dx)[None, None, :]
    y = cell_centres(ny, dy)[None, :, None]
    z = cell_centres(nz, dz)[:, None, None]
    u = np.zeros(shape)
    f = np.zeros(shape)
    for amp, (fx, kx), (fy, ky), (fz, kz) in terms:
        t = amp * _axis_mode(fx, kx, x) * _axis_mode(fy, ky, y) * _axis_mode(fz, kz, z)
        u += t
        f += -(kx * kx + ky * ky + kz * kz) * t
    return np.ascontiguousarray(u), np.ascontiguousarray(f)


def gaussian_blobs(shape, spacing, seed: int, count: int = 16):
    """Parameters of `count` Gaussian blobs: amplitudes N(0,1), centres U(0.2,0.8)^3, widths U(0.03,0.1)."""
    rng = np.random.default_rng(seed)
    amp = rng.standard_normal(count)
    centre = rng.uniform(0.2, 0.8, size=(count, 3))
    width = rng.uniform(0.03, 0.1, size=count)
    return amp, centre, width


def blob_field(shape, spacing, amp, centre, width) -> np.ndarray:
    """f = sum_i A_i exp(-|x - c_i|^2 / (2 w_i^2)) at cell centres (numpy, fp64)."""
    nz, ny, nx = shape
    dx, dy, dz = spacing
    x = cell_centres(nx, dx)[None, None, :]
    y = cell_centres(ny, dy)[None, :, None]
    z = cell_centres(nz, dz)[:, None, None]
    f = np.zeros(shape)
    for a, c, w in zip(amp, centre, width):
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        f += a * np.exp(-r2 / (2.0 * w * w))
    return f


def batched_grids(seed: int, count: int = 64, sides=(32, 48, 64, 96, 128, 192, 256)):
    """Uneven batch: per grid, sides drawn from `sides` per axis and boundary conditions
    drawn per axis (periodic with probability 1/3, else each face from {N, D})."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = [int(rng.choice(sides)) for _ in range(3)]
        bc = ""
        for _a in range(3):
            if rng.random() < 1.0 / 3.0:
                bc += "PP"
            else:
                bc += "".join(rng.choice(["N", "D"], size=2))
        out.append(((n[2], n[1], n[0]), bc))
    return out


def manufactured_device(shape, spacing, terms, device="cuda"):
    """manufactured() evaluated with torch on a device (FP64), for grids too large to build on the
    host; the same products and the same sign convention."""
    import torch
    nz, ny, nx = shape
    dx, dy, dz = spacing
    ar = lambda n, h: (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * h
    x = ar(nx, dx)[None, None, :]
    y = ar(ny, dy)[None, :, None]
    z = ar(nz, dz)[:, None, None]
    fn = {"sin": torch.sin, "cos": torch.cos}
    u = torch.zeros(shape, dtype=torch.float64, device=device)
    f = torch.zeros(shape, dtype=torch.float64, device=device)
    for amp, (fx, kx), (fy, ky), (fz, kz) in terms:
        t = amp * fn[fx](kx * x) * fn[fy](ky * y) * fn[fz](kz * z)
        u += t
        f += -(kx * kx + ky * ky + kz * kz) * t
        del t
    return u, f

