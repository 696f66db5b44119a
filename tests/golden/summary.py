"""Compact summaries of a long oracle run, for comparison with the GPU run.

A restored cube of a 500-iteration run is too large to store, and too slow
for the oracle to recompute inside a GPU test, so ``make_long_runs.py``
stores, per run: the values at a fixed set of voxels, the per-band norms and
32 projections <x, r_i> on Rademacher vectors r_i.  For an error e = x_gpu -
x_oracle, E[<e, r_i>^2] = ||e||^2, so the root mean square of the projection
differences estimates the relative L2 error of the whole cube (within about
+-25 % for 32 projections), and the sampled voxels bound it locally.

The Rademacher signs come from a counter-based hash (splitmix64 of the voxel
index and the projection number), so they do not depend on a NumPy random
stream and both sides regenerate them exactly.
"""
from __future__ import annotations

import numpy as np

N_PROJ = 32
N_SAMPLES = 2048
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014), uint64 wrap-around."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def rademacher(i: int, size: int) -> np.ndarray:
    """+-1 vector number i of length size (float64)."""
    j = np.arange(size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _splitmix64(j + np.uint64(i) * np.uint64(0x632BE59BD9B4E019))
    return np.where((h >> np.uint64(63)) == 1, 1.0, -1.0)


def sample_indices(size: int, seed: int) -> np.ndarray:
    """N_SAMPLES distinct voxel indices (hash order, no NumPy random stream)."""
    keys = _splitmix64(np.arange(size, dtype=np.uint64) ^ np.uint64(seed))
    return np.sort(np.argsort(keys, kind="stable")[:N_SAMPLES]).astype(np.int64)


def summarise(x: np.ndarray, seed: int) -> dict:
    x = np.asarray(x, np.float64)
    flat = x.ravel()
    idx = sample_indices(flat.size, seed)
    return dict(shape=list(x.shape), seed=seed, norm=float(np.linalg.norm(flat)),
                band_norms=[float(v) for v in np.linalg.norm(x.reshape(x.shape[0], -1), axis=1)],
                sample_index=[int(v) for v in idx], sample_value=[float(v) for v in flat[idx]],
                proj=[float(np.dot(flat, rademacher(i, flat.size))) for i in range(N_PROJ)])


def errors(x: np.ndarray, s: dict) -> dict:
    """Relative errors of x against a stored summary s: sampled voxels,
    projection estimate of the whole cube, per-band norms."""
    x = np.asarray(x, np.float64)
    flat = x.ravel()
    idx = np.asarray(s["sample_index"], np.int64)
    ref = np.asarray(s["sample_value"])
    samp = float(np.linalg.norm(flat[idx] - ref) / np.linalg.norm(ref))
    d = np.array([np.dot(flat, rademacher(i, flat.size)) for i in range(N_PROJ)]) - \
        np.asarray(s["proj"])
    proj = float(np.sqrt(np.mean(d * d)) / s["norm"])
    bn = np.linalg.norm(x.reshape(x.shape[0], -1), axis=1)
    band = float(np.max(np.abs(bn - np.asarray(s["band_norms"])) / np.asarray(s["band_norms"])))
    return dict(sampled=samp, projected=proj, band_norm=band)
