"""Forward operator H_l of Eq. (model) and its adjoint (FP64).

Eq. (model) says only that H_l is "a convolution by the PSF".  Reading taken:
circular convolution on the n x n grid with the PSF origin at pixel (0, 0),
H_l = F^-1 diag(h_hat_l) F, so H_l^T = F^-1 diag(conj h_hat_l) F and
||H_l||^2 = max_k |h_hat_l(k)|^2.  The Lipschitz constant of the gradient of
the least-squares term of Eq. (probopt) is beta = max_l ||H_l||^2.
"""
from __future__ import annotations

import numpy as np


def psf_spectrum(psf: np.ndarray) -> np.ndarray:
    return np.fft.fft2(np.asarray(psf, dtype=np.float64))


def H(x: np.ndarray, hhat: np.ndarray) -> np.ndarray:
    """H_l x_l for every band (x, hhat: [L, n, n])."""
    return np.fft.ifft2(hhat * np.fft.fft2(x)).real


def HT(r: np.ndarray, hhat: np.ndarray) -> np.ndarray:
    """H_l^T r_l for every band."""
    return np.fft.ifft2(np.conj(hhat) * np.fft.fft2(r)).real


def lipschitz(hhat: np.ndarray) -> float:
    """beta = max_l ||H_l||^2 = max_{l,k} |h_hat_l(k)|^2 (circulant H_l)."""
    return float(np.max(np.abs(hhat) ** 2))


def power_iteration(hhat_l: np.ndarray, iters: int = 500,
                    seed: int = 0) -> float:
    """||H_l||^2 by power iteration on H_l^T H_l (generic operator method)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(hhat_l.shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = HT(H(v[None], hhat_l[None]), hhat_l[None])[0]
        lam = float(np.vdot(v, w))
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return lam
