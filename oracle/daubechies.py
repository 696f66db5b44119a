"""Daubechies extremal-phase scaling filters (FP64).

The spatial dictionary of Sec. 4.2.1 is "the union of the first 8 Daubechies
wavelet bases"; the paper gives no taps, so they are derived here from the
mathematics (Daubechies' spectral factorisation), not copied from a table:

  |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<p} C(p-1+k, k) y^k.

With y = (2 - z - 1/z)/4 every root y_j of P gives the pair z, 1/z solving
z + 1/z = 2 - 4 y_j; the minimum-phase ("extremal phase") factor keeps the
root inside the unit circle.  The scaling filter is the coefficient list, in
descending powers of z, of (z + 1)^p prod_j (z - z_j), scaled so sum(h) =
sqrt(2).  db1 is the Haar filter (1, 1)/sqrt(2).
"""
from __future__ import annotations

import math

import numpy as np


def daubechies_lowpass(p: int) -> np.ndarray:
    """Scaling filter h of db<p>, length 2p, h[0] the leading tap."""
    if p < 1:
        raise ValueError("p >= 1")
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]          # ascending
    zeros = [-1.0 + 0j] * p
    if p > 1:
        for y in np.roots(coeffs[::-1]):
            b = 2.0 - 4.0 * y                    # z^2 - b z + 1 = 0
            disc = np.sqrt(b * b - 4.0 + 0j)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            zeros.append(z1 if abs(z1) < 1.0 else z2)
    h = np.real(np.poly(np.asarray(zeros)))
    return h * (math.sqrt(2.0) / h.sum())


def daubechies_highpass(h: np.ndarray) -> np.ndarray:
    """Quadrature-mirror detail filter g[i] = (-1)^i h[2p-1-i]."""
    L = len(h)
    return np.array([(-1.0) ** i * h[L - 1 - i] for i in range(L)])


def filter_bank(n_wavelets: int = 8):
    """[(h, g)] for db1 .. db<n_wavelets>."""
    out = []
    for p in range(1, n_wavelets + 1):
        h = daubechies_lowpass(p)
        out.append((h, daubechies_highpass(h)))
    return out
