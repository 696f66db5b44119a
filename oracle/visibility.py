"""Visibility-domain data term (FP64, test infrastructure).

Sec. 1 notes that the method runs unchanged when the direct operator maps
the sky to the visibilities instead of the dirty images.  The paper defines
no gridding or weighting for that case; the reading taken here:

* visibilities sample the unitary 2D DFT U = F / n of each band image on the
  n x n grid (nearest cell), d_p = (U x_l)_{k(p)} + noise;
* the data term is 1/2 sum_p |d_p - (U x_l)_{k(p)}|^2 (natural weighting).
  Gridding the samples into per-cell sums D_l[k] = sum_{p in k} d_p and
  counts m_l[k] gives, for real x,
      grad = Re U^H (m_l * U x_l - D_l) = F^-1 (m~_l * F x_l) - Re U^H D_l,
  with m~_l[k] = (m_l[k] + m_l[-k]) / 2;
* so the Lipschitz constant of the gradient is max_{l,k} m~_l[k], and the
  data term is the image-domain one with |h_hat_l|^2 = m~_l and H^T y =
  Re U^H D_l.

``point_gradient`` and ``data_term`` sum over the samples one by one (the
definition); ``gradient`` is the gridded closed form above; ``solve`` runs
Algorithm 2 (oracle.muffin.solve) with that gradient.
"""
from __future__ import annotations

import numpy as np

from . import muffin as om


def grid(ky, kx, d, n: int):
    """Per-cell sums D and counts m of samples d at cells (ky, kx) mod n."""
    D = np.zeros((n, n), np.complex128)
    m = np.zeros((n, n), np.float64)
    np.add.at(D, (ky % n, kx % n), d)
    np.add.at(m, (ky % n, kx % n), 1.0)
    return D, m


def dft_row(ky: int, kx: int, n: int) -> np.ndarray:
    """Row (ky, kx) of the unitary 2D DFT as an n x n array: (U x)_k =
    sum_{j} row[j] x[j]."""
    j = np.arange(n)
    return np.exp(-2j * np.pi * (ky * j[:, None] + kx * j[None, :]) / n) / n


def data_term(x_l, ky, kx, d) -> float:
    """1/2 sum_p |d_p - (U x)_{k(p)}|^2 by explicit sums over the samples."""
    n = x_l.shape[-1]
    f = 0.0
    for a, b, dp in zip(ky, kx, d):
        r = np.sum(dft_row(a, b, n) * x_l) - dp
        f += 0.5 * abs(r) ** 2
    return f


def point_gradient(x_l, ky, kx, d) -> np.ndarray:
    """Gradient of data_term in x (real): sum_p Re(conj(row_p) (row_p . x - d_p))."""
    n = x_l.shape[-1]
    g = np.zeros((n, n))
    for a, b, dp in zip(ky, kx, d):
        row = dft_row(a, b, n)
        r = np.sum(row * x_l) - dp
        g += (np.conj(row) * r).real
    return g


def symmetrised(m) -> np.ndarray:
    """m~[k] = (m[k] + m[-k]) / 2 per band (m: [..., n, n])."""
    m = np.asarray(m, np.float64)
    mr = np.roll(np.flip(m, axis=(-2, -1)), 1, axis=(-2, -1))   # m[-k]
    return 0.5 * (m + mr)


def gradient(x, D, m) -> np.ndarray:
    """Re U^H (m * U x - D) for every band (x, D, m: [L, n, n])."""
    x = np.asarray(x, np.float64)
    Ux = np.fft.fft2(x, norm="ortho")
    return np.fft.ifft2(m * Ux - D, norm="ortho").real


def lipschitz(m) -> float:
    return float(np.max(symmetrised(m)))


def make_problem(D, m, n_wavelets=8, J=3, sigma=10.0, **kw) -> om.Problem:
    """An Algorithm-2 problem whose data term is the visibility one: the
    step sizes see |h_hat|^2 = m~ (h_hat = sqrt(m~)); y is unused."""
    D = np.asarray(D)
    L, n, _ = D.shape
    psf = np.zeros((L, n, n))
    psf[:, 0, 0] = 1.0
    prob = om.make_problem(np.zeros((L, n, n)), psf, n_wavelets=n_wavelets, J=J,
                           sigma=sigma, **kw)
    prob.hhat = np.sqrt(symmetrised(m)).astype(np.complex128)
    return prob


def solve(D, m, mu: float, gamma: float, n_iter: int, n_wavelets=8, J=3, sigma=10.0,
          tau=None):
    """Algorithm 2 on the visibility data term; returns (state, tau)."""
    D = np.asarray(D, np.complex128)
    m = np.asarray(m, np.float64)
    prob = make_problem(D, m, n_wavelets=n_wavelets, J=J, sigma=sigma)
    return om.solve(prob, mu, gamma, n_iter, tau=tau, grad_fn=lambda x: gradient(x, D, m))


def equivalent_image_problem(D, m):
    """(h_hat, y) of the image-domain data term with the same gradient:
    h_hat = sqrt(m~) and y with conj(h_hat) F y = n D where m~ > 0
    (y real when D is Hermitian and m symmetric)."""
    D = np.asarray(D, np.complex128)
    n = D.shape[-1]
    ms = symmetrised(m)
    hh = np.sqrt(ms)
    yhat = np.where(ms > 0, n * D / np.where(hh > 0, hh, 1.0), 0.0)
    return hh.astype(np.complex128), np.fft.ifft2(yhat)
