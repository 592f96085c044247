"""Field recipes for the nabla workloads (all seeded, numpy PCG64).

Scalar   f(lon, lat) = cos(lat) cos(lon) + 0.5 sin(2 lat)
Vector   (u, v)      = (cos(lat), 0.1 sin(lon) cos(lat))

Multi-level fields: level k holds the base field scaled by (1 + 0.01 k) plus
independent N(0, sigma^2) noise, sigma = 1e-3, drawn from PCG64(seed) in
[node][level] order.  The scalar uses seed 0; u and v use seeds 10 and 11.
Single-level scalar fields keep the noise; the single-level vector is
noise-free.  Everything is built in float64 and rounded once to the requested
dtype, so a float32 array upcast to float64 is exactly what the float32 path
computed on.
"""
from __future__ import annotations

import numpy as np

NOISE_SIGMA = 1e-3
SEED_SCALAR = 0
SEED_U = 10
SEED_V = 11


def base_scalar(lon: np.ndarray, lat: np.ndarray) -> np.ndarray:
    return np.cos(lat) * np.cos(lon) + 0.5 * np.sin(2.0 * lat)


def base_vector(lon: np.ndarray, lat: np.ndarray):
    return np.cos(lat), 0.1 * np.sin(lon) * np.cos(lat)


def normal(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard normal draws from PCG64(seed), row-major over ``shape``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if dtype == np.float32:
        return rng.standard_normal(shape, dtype=np.float32)
    return rng.standard_normal(shape)


def _levels(base: np.ndarray, nlev: int, seed: int | None, dtype, chunk: int = 1 << 22) -> np.ndarray:
    V = base.shape[0]
    out = np.empty((V, nlev), dtype=dtype)
    scale = 1.0 + 0.01 * np.arange(nlev, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed)) if seed is not None else None
    rows = max(1, chunk // max(nlev, 1))
    for i0 in range(0, V, rows):
        i1 = min(V, i0 + rows)
        blk = base[i0:i1, None] * scale[None, :]
        if rng is not None:
            blk = blk + NOISE_SIGMA * rng.standard_normal((i1 - i0, nlev))
        out[i0:i1] = blk.astype(dtype)
    return out


def level_scalar(lon, lat, nlev: int, dtype=np.float64, seed: int = SEED_SCALAR, noise: bool = True):
    """[node][level] scalar field of the recipe above."""
    return _levels(base_scalar(lon, lat), nlev, seed if noise else None, dtype)


def level_vector(lon, lat, nlev: int, dtype=np.float64, seeds=(SEED_U, SEED_V), noise: bool | None = None):
    """[node][level] (u, v); noise defaults to on for nlev > 1, off for one level."""
    if noise is None:
        noise = nlev > 1
    bu, bv = base_vector(lon, lat)
    u = _levels(bu, nlev, seeds[0] if noise else None, dtype)
    v = _levels(bv, nlev, seeds[1] if noise else None, dtype)
    return u, v


def padded(x: np.ndarray, ld: int) -> np.ndarray:
    """Copy [node][nlev] into a zero-padded [node][ld] array (ld >= nlev)."""
    V, nlev = x.shape
    out = np.zeros((V, ld), dtype=x.dtype)
    out[:, :nlev] = x
    return out


def sample_nodes(nnodes: int, row_offsets: np.ndarray, count: int, seed: int = 7) -> np.ndarray:
    """Sorted sample of node ids: every node of the first and last two rows'
    first points, each row's first and last node, plus uniform random nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    picks = [row_offsets[:-1], row_offsets[1:] - 1]
    picks.append(np.arange(row_offsets[0], row_offsets[1]))
    picks.append(np.arange(row_offsets[-2], row_offsets[-1]))
    picks.append(rng.integers(0, nnodes, size=count))
    return np.unique(np.concatenate(picks).astype(np.int64))
