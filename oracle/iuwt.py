"""Isotropic undecimated wavelet transform (IUWT, "starlet"), the alternative
spatial dictionary W_s that Sec. 2.1 names beside unions of Daubechies bases
(FP64, test infrastructure).

Readings (the paper names the transform only):
* scaling kernel: the B3 spline h = [1, 4, 6, 4, 1] / 16 of the starlet,
  separable in x and y, dilated by 2^j at scale j ("a trous");
* boundaries: periodic, as the circular convolution read for Eq. (model);
* J scales give J + 1 coefficient planes per image: w_1 .. w_J with
  w_{j+1} = c_j - c_{j+1}, c_{j+1} = S_j c_j, c_0 = x, and the coarse c_J;
* the step condition of Sec. 2.2 needs ||W_s||^2, the largest eigenvalue of
  W_s^T W_s, which is diagonal in the 2D DFT: the maximum over the n x n
  grid of sum_j |A_j - A_{j+1}|^2 + |A_J|^2, with A_j the transfer function
  of S_{j-1} ... S_0.  The B3 symbol (1 + cos w)^2 / 4 lies in [0, 1], so
  the A_j decrease from 1 and the sum is at most A_0^2 = 1, reached at
  w = 0: the norm is 1 for every grid and J (the frame is not tight; its
  lower bound is below 1).  norm2 evaluates the maximum anyway.
"""
from __future__ import annotations

import numpy as np

H_B3 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def smooth(c: np.ndarray, j: int) -> np.ndarray:
    """S_j c: separable periodic convolution of the last two axes with h
    dilated by 2^j (taps at offsets (m - 2) 2^j)."""
    d = 1 << j
    out = np.zeros_like(c, dtype=np.float64)
    for m in range(5):                       # along y
        out += H_B3[m] * np.roll(c, -(m - 2) * d, axis=-2)
    res = np.zeros_like(out)
    for m in range(5):                       # along x
        res += H_B3[m] * np.roll(out, -(m - 2) * d, axis=-1)
    return res


def analysis(x: np.ndarray, J: int) -> np.ndarray:
    """W x: images [..., n, n] -> planes [..., J + 1, n, n]."""
    c = np.asarray(x, np.float64)
    planes = []
    for j in range(J):
        cn = smooth(c, j)
        planes.append(c - cn)
        c = cn
    planes.append(c)
    return np.stack(planes, axis=-3)


def _A_T(v: np.ndarray, j: int) -> np.ndarray:
    """(S_{j-1} ... S_0)^T v = S_0 ... S_{j-1} v (each S_i is symmetric)."""
    for i in reversed(range(j)):
        v = smooth(v, i)
    return v


def adjoint(u: np.ndarray, J: int) -> np.ndarray:
    """W^T u: planes [..., J + 1, n, n] -> images, from W = [A_j - A_{j+1}
    (j < J); A_J] term by term."""
    u = np.asarray(u, np.float64)
    out = _A_T(u[..., J, :, :], J)
    for j in range(J):
        out = out + _A_T(u[..., j, :, :], j) - _A_T(u[..., j, :, :], j + 1)
    return out


def norm2(n: int, J: int) -> float:
    """||W||^2 on the n x n periodic grid (max eigenvalue of W^T W)."""
    w = 2.0 * np.pi * np.arange(n) / n
    def h1(d):                                # 1D transfer function of S at dilation d
        return (6.0 + 8.0 * np.cos(d * w) + 2.0 * np.cos(2.0 * d * w)) / 16.0
    A = [np.ones((n, n))]
    for j in range(J):
        hj = h1(1 << j)
        A.append(A[-1] * np.outer(hj, hj))
    s = A[J] ** 2
    for j in range(J):
        s = s + (A[j] - A[j + 1]) ** 2
    return float(np.max(s))
