"""Per-band noise level from the dirty cube by the median absolute deviation
(FP64, test infrastructure).

Sec. 3.1 assumes the noise variances known, or estimated in the image domain
with robust statistics such as the median absolute deviation (MAD).  The
paper names the estimator only; the reading taken (Donoho and Johnstone's
wavelet-domain MAD, applied identically by the CUDA path):

* the detail coefficients come from the finest diagonal (high-high) band of
  the orthonormal Haar transform (db1, one level) of each dirty image y_l:
  an orthonormal transform keeps white noise white with the same variance,
  and on the finest scale the sky contributes few large coefficients;
* sigma_l = MAD(d) / Phi^-1(3/4), MAD(d) = median(|d - median(d)|), with
  Phi^-1(3/4) = 0.6744897501960817 the normal consistency constant; the
  median of an even count is the mean of the two middle values;
* the output is sigma_l^2, the per-band variance PSURE and SUGAR use.
"""
from __future__ import annotations

import numpy as np

from . import wavelets
from .daubechies import filter_bank

PHI_INV_3_4 = 0.6744897501960817


def haar_hh(y_l: np.ndarray) -> np.ndarray:
    """The finest high-high Haar band of one image (Mallat block [m:, m:])."""
    (h, g), = filter_bank(1)
    out = wavelets.analysis_level(np.asarray(y_l, np.float64), h, g)
    m = out.shape[-1] // 2
    return out[m:, m:]


def mad_sigma(d: np.ndarray) -> float:
    d = np.asarray(d, np.float64).ravel()
    med = np.median(d)
    return float(np.median(np.abs(d - med)) / PHI_INV_3_4)


def noise_var_mad(y: np.ndarray) -> np.ndarray:
    """sigma_l^2 for every band of a dirty cube y [L, n, n]."""
    return np.array([mad_sigma(haar_hh(y_l)) ** 2 for y_l in np.asarray(y)])
