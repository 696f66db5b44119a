"""Periodised orthonormal 2D wavelet transforms and the union W_s (FP64).

Reading of Sec. 2.1 / Sec. 4.2.1 (the paper names the dictionary only): the
memory count 11LN of Sec. 4.2.1 means W_s stores 8N coefficients per band, so
each of the 8 Daubechies bases is a critically sampled, periodised,
orthonormal transform:

* 1D analysis on a length-M signal (M even):
    a[k] = sum_i h[i] x[(2k+i) mod M],  d[k] = sum_i g[i] x[(2k+i) mod M],
  k = 0 .. M/2-1; synthesis is its exact transpose.
* 2D level: the 1D analysis along x (rows), then along y (columns).  Layout
  of the M x M level output (Mallat): [:M/2, :M/2] approximation (low y, low
  x), [:M/2, M/2:] low y / high x, [M/2:, :M/2] high y / low x, [M/2:, M/2:]
  high y / high x.  Level j+1 transforms the approximation block of level j.
* J levels (J = 0 makes every basis the identity).
* W_s x = [W_1 x; ...; W_K x] unscaled, so W_s^T W_s = K I and ||W_s||^2 = K.
"""
from __future__ import annotations

import numpy as np


def _idx(M: int, taps: int) -> np.ndarray:
    return (2 * np.arange(M // 2)[:, None] + np.arange(taps)[None, :]) % M


def analysis_1d(x: np.ndarray, h: np.ndarray, g: np.ndarray):
    """Periodised one-level analysis along the last axis -> (a, d)."""
    M = x.shape[-1]
    xs = x[..., _idx(M, len(h))]          # [..., M/2, taps]
    return xs @ h, xs @ g


def synthesis_1d(a: np.ndarray, d: np.ndarray, h: np.ndarray, g: np.ndarray):
    """Transpose of ``analysis_1d`` along the last axis."""
    M = 2 * a.shape[-1]
    idx = _idx(M, len(h))
    x = np.zeros(a.shape[:-1] + (M,), dtype=np.result_type(a, d, h))
    for i in range(len(h)):
        # for fixed i the targets (2k+i) mod M are distinct over k
        x[..., idx[:, i]] += h[i] * a + g[i] * d
    return x


def analysis_level(x: np.ndarray, h, g) -> np.ndarray:
    """One 2D level on the trailing [M, M] block, Mallat layout."""
    M = x.shape[-1]
    m = M // 2
    lo_x, hi_x = analysis_1d(x, h, g)                       # along x
    ll, lh = analysis_1d(np.swapaxes(lo_x, -1, -2), h, g)   # along y
    hl, hh = analysis_1d(np.swapaxes(hi_x, -1, -2), h, g)
    out = np.empty_like(x, dtype=np.result_type(x, h))
    out[..., :m, :m] = np.swapaxes(ll, -1, -2)
    out[..., :m, m:] = np.swapaxes(hl, -1, -2)
    out[..., m:, :m] = np.swapaxes(lh, -1, -2)
    out[..., m:, m:] = np.swapaxes(hh, -1, -2)
    return out


def synthesis_level(c: np.ndarray, h, g) -> np.ndarray:
    """Transpose of ``analysis_level``."""
    M = c.shape[-1]
    m = M // 2
    ll = np.swapaxes(c[..., :m, :m], -1, -2)
    hl = np.swapaxes(c[..., :m, m:], -1, -2)
    lh = np.swapaxes(c[..., m:, :m], -1, -2)
    hh = np.swapaxes(c[..., m:, m:], -1, -2)
    lo_x = np.swapaxes(synthesis_1d(ll, lh, h, g), -1, -2)
    hi_x = np.swapaxes(synthesis_1d(hl, hh, h, g), -1, -2)
    return synthesis_1d(lo_x, hi_x, h, g)


def dwt2(x: np.ndarray, h, g, J: int) -> np.ndarray:
    """J-level periodised 2D DWT of the trailing [n, n] axes."""
    out = np.array(x, dtype=np.float64, copy=True)
    n = x.shape[-1]
    for j in range(J):
        M = n >> j
        out[..., :M, :M] = analysis_level(out[..., :M, :M], h, g)
    return out


def idwt2(c: np.ndarray, h, g, J: int) -> np.ndarray:
    """Adjoint (= inverse) of ``dwt2``."""
    out = np.array(c, dtype=np.float64, copy=True)
    n = c.shape[-1]
    for j in reversed(range(J)):
        M = n >> j
        out[..., :M, :M] = synthesis_level(out[..., :M, :M], h, g)
    return out


def Ws(x: np.ndarray, bank, J: int) -> np.ndarray:
    """W_s x for images x [..., n, n] -> coefficients [..., K, n, n]."""
    return np.stack([dwt2(x, h, g, J) for h, g in bank], axis=-3)


def WsT(u: np.ndarray, bank, J: int) -> np.ndarray:
    """W_s^T u for coefficients [..., K, n, n] -> images [..., n, n]."""
    out = np.zeros(u.shape[:-3] + u.shape[-2:], dtype=np.float64)
    for k, (h, g) in enumerate(bank):
        out += idwt2(u[..., k, :, :], h, g, J)
    return out
