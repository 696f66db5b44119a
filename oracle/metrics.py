"""Point metrics of Sec. 4.1: SNR (dB) and WMSE (the per-voxel PMSE)."""
from __future__ import annotations

import numpy as np

from . import convolution


def snr_db(x_true, x) -> float:
    x_true = np.asarray(x_true, np.float64)
    err = x_true - np.asarray(x, np.float64)
    return float(10.0 * np.log10(np.sum(x_true ** 2) / np.sum(err ** 2)))


def wmse(x_true, x, hhat) -> float:
    x_true = np.asarray(x_true, np.float64)
    r = convolution.H(x_true - np.asarray(x, np.float64), hhat)
    return float(np.sum(r * r) / x_true.size)
