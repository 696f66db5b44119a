"""Spectral dictionary W_lambda: the orthonormal DCT-II along bands (FP64).

Sec. 4.2.1 sets W_lambda to "the DCT"; the reading taken is the orthonormal
DCT-II, C[k, l] = c_k cos(pi (2l+1) k / (2L)), c_0 = sqrt(1/L), c_k =
sqrt(2/L), so ||W_lambda|| = 1 and W_lambda^T = C^T (the DCT-III).
"""
from __future__ import annotations

import numpy as np


def dct_matrix(L: int) -> np.ndarray:
    k = np.arange(L)[:, None]
    l = np.arange(L)[None, :]
    C = np.cos(np.pi * (2 * l + 1) * k / (2.0 * L))
    C *= np.sqrt(2.0 / L)
    C[0, :] = np.sqrt(1.0 / L)
    return C


def apply_spectra(C: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Apply C to every pixel spectrum of a band-major cube X [L, ...]."""
    return np.tensordot(C, X, axes=(1, 0))
