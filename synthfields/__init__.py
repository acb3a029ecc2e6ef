"""Seeded synthetic scalar fields on regular grids.

This module only draws inputs.  It holds none of the segmentation's
arithmetic (no order keys, no neighbours, no integral lines), so that the
CPU oracle and the CUDA path can both be fed the exact same bytes from it
without sharing any part of the method.

Layout convention for every generator: a C-ordered numpy array of shape
``(nz, ny, nx)`` so that x is the fastest axis and the vertex with grid
coordinates (x, y, z) has linear index ``x + nx*(y + ny*z)``.  This is the
vertex numbering of the paper's 4x4 example grid (Fig. 1), which counts
nodes along x first.  A 2D field is returned with ``nz == 1``.

The workloads stand in for the paper's datasets, which are not available
here (Sec. 6: Miranda 512^3, Foot 256^3):

* ``gaussian_sum``      -- a sum of a few random Gaussians plus small noise
                           (64^3 small case);
* ``smoothed_noise``    -- white noise blurred by a separable periodic
                           Gaussian (512^3, sigma = 4: dense extrema);
* ``quantize_levels``   -- the same quantised to 256 levels, which creates
                           exact value ties;
* ``broad_gaussians_ramp`` -- two very broad Gaussians plus a linear ramp
                           (1024^3 and 32768^2: very long steepest paths);
* ``batch_specs`` / ``batch_field`` -- a seeded list of uneven grids for
                           many-field batches;
* analytic fields with known extrema (ramp, constant, paraboloid).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "FIG1_VALUES",
    "FIG1_DIMS",
    "rng_for",
    "gaussian_sum",
    "smoothed_noise",
    "quantize_levels",
    "broad_gaussians_ramp",
    "ramp",
    "constant",
    "paraboloid",
    "random_ties",
    "batch_specs",
    "batch_field",
    "serve_specs",
]

# Fig. 1 (a): the 4x4 input field, rows listed from y = 0 upwards, x fastest.
FIG1_DIMS = (4, 4, 1)
FIG1_VALUES = [14, 12, 2, 0, 13, 11, 3, 4, 5, 6, 7, 8, 1, 9, 10, 15]


def rng_for(seed: int) -> np.random.Generator:
    """The one random source of every generator: numpy PCG64 with ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _shape(dims: Sequence[int]) -> Tuple[int, int, int]:
    nx, ny, nz = (int(d) for d in dims)
    if nx < 1 or ny < 1 or nz < 1:
        raise ValueError(f"bad dims {dims}")
    return nz, ny, nx


def _axes(dims):
    nx, ny, nz = (int(d) for d in dims)
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    return x, y, z


def gaussian_sum(dims, seed: int, n_gauss: int = 8, sigma=(4.0, 12.0),
                 amp=(-1.0, 1.0), noise: float = 1e-3,
                 dtype=np.float32) -> np.ndarray:
    """Sum of ``n_gauss`` isotropic Gaussians (centres uniform in the box,
    sigma uniform in ``sigma``, amplitude uniform in ``amp``) plus uniform
    noise in [-noise, noise].  Evaluated in float64, then cast."""
    nx, ny, nz = (int(d) for d in dims)
    g = rng_for(seed)
    c = g.uniform(0.0, 1.0, size=(n_gauss, 3)) * np.array([nx - 1, ny - 1, nz - 1], dtype=np.float64)
    s = g.uniform(sigma[0], sigma[1], size=n_gauss)
    a = g.uniform(amp[0], amp[1], size=n_gauss)
    x, y, z = _axes(dims)
    f = np.zeros(_shape(dims), dtype=np.float64)
    for i in range(n_gauss):
        ex = np.exp(-((x - c[i, 0]) ** 2) / (2 * s[i] ** 2))
        ey = np.exp(-((y - c[i, 1]) ** 2) / (2 * s[i] ** 2))
        ez = np.exp(-((z - c[i, 2]) ** 2) / (2 * s[i] ** 2))
        f += a[i] * (ez * ey * ex)
    if noise:
        f += g.uniform(-noise, noise, size=f.shape)
    return np.ascontiguousarray(f.astype(dtype))


def smoothed_noise(dims, seed: int, sigma: float = 4.0, radius: int = 16,
                   dtype=np.float32) -> np.ndarray:
    """White noise N(0,1) (drawn in float32) filtered by a separable,
    periodic Gaussian of standard deviation ``sigma`` truncated at
    ``radius`` voxels, one axis after the other (axes of extent 1 are
    skipped)."""
    from scipy import ndimage

    g = rng_for(seed)
    f = g.standard_normal(_shape(dims), dtype=np.float32)
    if sigma > 0:
        trunc = radius / float(sigma)
        for ax in range(3):
            if f.shape[ax] > 1:
                f = ndimage.gaussian_filter1d(f, float(sigma), axis=ax, mode="wrap",
                                              truncate=trunc)
    return np.ascontiguousarray(f.astype(dtype))


def quantize_levels(f: np.ndarray, levels: int = 256) -> np.ndarray:
    """q = min(levels-1, floor(levels*(f-min)/(max-min))) stored in the
    input's dtype; a constant input maps to all zeros."""
    f64 = f.astype(np.float64)
    lo, hi = float(f64.min()), float(f64.max())
    if hi <= lo:
        return np.zeros_like(f)
    q = np.floor(levels * (f64 - lo) / (hi - lo))
    q = np.minimum(q, levels - 1)
    return np.ascontiguousarray(q.astype(f.dtype))


def broad_gaussians_ramp(dims, seed: int, sigma: float = 300.0,
                         dtype=np.float32, rows: int = 2048) -> np.ndarray:
    """Two broad Gaussians (amplitudes +1 and -1, centres uniform in the
    middle half of the box) plus a gentle linear ramp.  3D ramp:
    0.5*(x+2y+3z)/(6(n-1)); 2D (nz == 1): 0.5*(x+2y)/(3(n-1)), with n the
    largest extent.  Built in blocks of ``rows`` rows so that 1024^3 and
    32768^2 fit in float32 without large temporaries."""
    nx, ny, nz = (int(d) for d in dims)
    g = rng_for(seed)
    ext = np.array([nx - 1, ny - 1, nz - 1], dtype=np.float64)
    c = (0.25 + 0.5 * g.uniform(0.0, 1.0, size=(2, 3))) * ext
    amps = (1.0, -1.0)
    n = max(nx, ny, nz)
    x = np.arange(nx, dtype=np.float64)
    gx = [np.exp(-((x - c[i, 0]) ** 2) / (2 * sigma ** 2)) for i in range(2)]
    if nz > 1:
        cx, cy, cz = 0.5 / (6.0 * (n - 1)), 0.5 * 2.0 / (6.0 * (n - 1)), 0.5 * 3.0 / (6.0 * (n - 1))
    else:
        cx, cy, cz = 0.5 / (3.0 * max(n - 1, 1)), 0.5 * 2.0 / (3.0 * max(n - 1, 1)), 0.0
    out = np.empty((nz, ny, nx), dtype=dtype)
    for z in range(nz):
        gz = [math.exp(-((z - c[i, 2]) ** 2) / (2 * sigma ** 2)) if nz > 1 else 1.0 for i in range(2)]
        for y0 in range(0, ny, rows):
            y = np.arange(y0, min(ny, y0 + rows), dtype=np.float64)[:, None]
            acc = cx * x[None, :] + cy * y + cz * z
            for i in range(2):
                gy = np.exp(-((y - c[i, 1]) ** 2) / (2 * sigma ** 2))
                acc = acc + (amps[i] * gz[i]) * gy * gx[i][None, :]
            out[z, y0:y0 + y.shape[0]] = acc.astype(dtype)
    return out


def ramp(dims, dtype=np.float32) -> np.ndarray:
    """f = x + y + z: strictly increasing along every stencil edge."""
    x, y, z = _axes(dims)
    return np.ascontiguousarray((x + y + z).astype(dtype))


def constant(dims, value: float = 1.0, dtype=np.float32) -> np.ndarray:
    return np.full(_shape(dims), value, dtype=dtype)


def paraboloid(dims, centre, dtype=np.float32) -> np.ndarray:
    """f = -|p - centre|^2 (an inverted paraboloid)."""
    x, y, z = _axes(dims)
    cx, cy, cz = centre
    f = -((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
    return np.ascontiguousarray(f.astype(dtype))


def random_ties(dims, seed: int, levels: int = 3, dtype=np.float32) -> np.ndarray:
    """Integer values drawn uniformly from ``levels`` levels: many exact ties."""
    g = rng_for(seed)
    return np.ascontiguousarray(g.integers(0, levels, size=_shape(dims)).astype(dtype))


def batch_specs(n_fields: int = 256, seed: int = 0, lo: int = 32, hi: int = 256):
    """A seeded list of (dims, dtype_name, kind, sub_seed, sigma) for a
    many-field batch: each axis log-uniform in [lo, hi] (rounded), fp32 or
    fp16 with even odds, smoothed noise (sigma uniform in [2, 6]) or a
    Gaussian sum with even odds."""
    g = rng_for(seed)
    out = []
    for i in range(n_fields):
        d = np.exp(g.uniform(math.log(lo), math.log(hi), size=3))
        dims = tuple(int(round(v)) for v in d)
        dt = "f16" if g.uniform() < 0.5 else "f32"
        kind = "noise" if g.uniform() < 0.5 else "gauss"
        sigma = float(g.uniform(2.0, 6.0))
        out.append((dims, dt, kind, 1000 + 7919 * seed + i, sigma))
    return out


def batch_field(spec) -> np.ndarray:
    dims, dt, kind, sub_seed, sigma = spec
    dtype = np.float16 if dt == "f16" else np.float32
    if kind == "noise":
        f = smoothed_noise(dims, sub_seed, sigma=sigma, radius=int(4 * sigma), dtype=np.float32)
    else:
        f = gaussian_sum(dims, sub_seed, dtype=np.float32)
    return np.ascontiguousarray(f.astype(dtype))


def serve_specs(n_requests: int, seed: int = 0, two_d=(512, 16384), three_d=(64, 768)):
    """A seeded request mix: (dims, sub_seed); half 2D squares with side
    log-uniform in ``two_d``, half 3D cubes with side log-uniform in
    ``three_d``."""
    g = rng_for(seed)
    out: List = []
    for i in range(n_requests):
        if g.uniform() < 0.5:
            s = int(round(math.exp(g.uniform(math.log(two_d[0]), math.log(two_d[1])))))
            dims = (s, s, 1)
        else:
            s = int(round(math.exp(g.uniform(math.log(three_d[0]), math.log(three_d[1])))))
            dims = (s, s, s)
        out.append((dims, 5000 + 104729 * seed + i))
    return out
