"""Pins of the oracle's linear operators (H, W_s, W_lambda) against dense
brute force, closed forms and library special cases."""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import convolution, spectral, wavelets
from oracle.daubechies import filter_bank


# ---------------------------------------------------------------- dense builds
def dense_dwt1(M, h, g):
    """Analysis matrix of one periodised level, written from its definition:
    row k < M/2 holds h at columns (2k+i) mod M, row M/2+k holds g."""
    A = np.zeros((M, M))
    for k in range(M // 2):
        for i in range(len(h)):
            A[k, (2 * k + i) % M] += h[i]
            A[M // 2 + k, (2 * k + i) % M] += g[i]
    return A


def dense_basis(n, h, g, J):
    """n^2 x n^2 matrix of a J-level 2D transform (row-major images): each
    level maps the leading M x M block B to A B A^T (A acts along y from the
    left and along x from the right)."""
    W = np.eye(n * n)
    for j in range(J):
        M = n >> j
        A = dense_dwt1(M, h, g)
        Lj = np.zeros((n * n, n * n))
        for col in range(n * n):
            e = np.zeros((n, n))
            e.flat[col] = 1.0
            out = e.copy()
            out[:M, :M] = A @ e[:M, :M] @ A.T
            Lj[:, col] = out.ravel()
        W = Lj @ W
    return W


def dense_circulant(psf):
    n = psf.shape[0]
    Hm = np.zeros((n * n, n * n))
    for iy in range(n):
        for ix in range(n):
            for jy in range(n):
                for jx in range(n):
                    Hm[iy * n + ix, jy * n + jx] = psf[(iy - jy) % n, (ix - jx) % n]
    return Hm


# ---------------------------------------------------------------- wavelets
@pytest.mark.parametrize("n,J", [(8, 1), (8, 2), (8, 3), (16, 3), (16, 2)])
@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_fast_dwt_equals_dense(n, J, p):
    h, g = filter_bank(8)[p - 1]
    W = dense_basis(n, h, g, J)
    rng = np.random.default_rng(p * 100 + n + J)
    x = rng.standard_normal((n, n))
    assert np.allclose(wavelets.dwt2(x, h, g, J).ravel(), W @ x.ravel(), atol=1e-12)
    c = rng.standard_normal((n, n))
    assert np.allclose(wavelets.idwt2(c, h, g, J).ravel(), W.T @ c.ravel(), atol=1e-12)


@pytest.mark.parametrize("n,J", [(8, 3), (16, 3), (4, 2), (2, 1)])
@pytest.mark.parametrize("p", range(1, 9))
def test_each_basis_orthonormal(n, J, p):
    h, g = filter_bank(8)[p - 1]
    W = dense_basis(n, h, g, J)
    assert np.allclose(W @ W.T, np.eye(n * n), atol=1e-11)
    rng = np.random.default_rng(p)
    x = rng.standard_normal((3, n, n))
    xr = wavelets.idwt2(wavelets.dwt2(x, h, g, J), h, g, J)
    assert np.allclose(xr, x, atol=1e-11)


def test_haar_level_closed_form():
    # one Haar level: pairwise (x0+x1)/sqrt2 along x then along y
    x = np.arange(16.0).reshape(4, 4) ** 1.5
    h, g = filter_bank(1)[0]
    c = wavelets.dwt2(x, h, g, 1)
    a = x[0::2, 0::2]; b = x[0::2, 1::2]; cc = x[1::2, 0::2]; d = x[1::2, 1::2]
    assert np.allclose(c[:2, :2], (a + b + cc + d) / 2)          # low y, low x
    assert np.allclose(c[:2, 2:], (a - b + cc - d) / 2)          # low y, high x
    assert np.allclose(c[2:, :2], (a + b - cc - d) / 2)          # high y, low x
    assert np.allclose(c[2:, 2:], (a - b - cc + d) / 2)


def test_phase_convention_impulse():
    # a[k] = sum_i h[i] x[(2k+i) mod M]: an impulse at x[j] gives a[k] = h[j-2k]
    h, g = filter_bank(8)[2]      # db3, 6 taps
    M = 16
    for j in range(M):
        x = np.zeros(M); x[j] = 1.0
        a, d = wavelets.analysis_1d(x, h, g)
        for k in range(M // 2):
            i = (j - 2 * k) % M
            assert a[k] == pytest.approx(h[i] if i < 6 else 0.0, abs=1e-15)
            assert d[k] == pytest.approx(g[i] if i < 6 else 0.0, abs=1e-15)


@pytest.mark.parametrize("K", [1, 3, 8])
def test_union_frame(K):
    bank = filter_bank(K)
    rng = np.random.default_rng(K)
    x = rng.standard_normal((2, 16, 16))
    u = wavelets.Ws(x, bank, 3)
    assert u.shape == (2, K, 16, 16)
    # W_s^T W_s = K I  (so ||W_s||^2 = K, the 8N coefficients of Sec. 4.2.1)
    assert np.allclose(wavelets.WsT(u, bank, 3), K * x, atol=1e-11)
    # adjointness <W_s x, u> = <x, W_s^T u>
    v = rng.standard_normal(u.shape)
    assert np.vdot(u, v) == pytest.approx(np.vdot(x, wavelets.WsT(v, bank, 3)), rel=1e-12)


def test_levels_zero_is_identity():
    bank = filter_bank(8)
    x = np.random.default_rng(0).standard_normal((16, 16))
    u = wavelets.Ws(x, bank, 0)
    assert np.array_equal(u, np.broadcast_to(x, (8, 16, 16)))


# ---------------------------------------------------------------- DCT
@pytest.mark.parametrize("L", [1, 2, 8, 13, 64])
def test_dct_orthonormal_and_scipy(L):
    C = spectral.dct_matrix(L)
    assert np.allclose(C @ C.T, np.eye(L), atol=1e-13)
    x = np.random.default_rng(L).standard_normal((L, 5))
    assert np.allclose(spectral.apply_spectra(C, x),
                       scipy.fft.dct(x, type=2, norm="ortho", axis=0), atol=1e-12)
    assert np.allclose(spectral.apply_spectra(C.T, x),
                       scipy.fft.idct(x, type=2, norm="ortho", axis=0), atol=1e-12)


# ---------------------------------------------------------------- H
@pytest.mark.parametrize("n", [4, 8])
def test_convolution_equals_dense_circulant(n):
    rng = np.random.default_rng(n)
    psf = rng.standard_normal((n, n))
    Hm = dense_circulant(psf)
    hh = convolution.psf_spectrum(psf[None])
    x = rng.standard_normal((1, n, n))
    assert np.allclose(convolution.H(x, hh).ravel(), Hm @ x.ravel(), atol=1e-12)
    assert np.allclose(convolution.HT(x, hh).ravel(), Hm.T @ x.ravel(), atol=1e-12)
    # ||H||^2 = largest eigenvalue of H^T H, equal to max |h_hat|^2
    lam = np.linalg.eigvalsh(Hm.T @ Hm).max()
    assert convolution.lipschitz(hh) == pytest.approx(lam, rel=1e-10)


def test_power_iteration_matches_closed_form():
    from synth import make_cube
    c = make_cube(16, 2, 5, 1, 300, seed=11, with_delta=False)
    hh = convolution.psf_spectrum(c.psf)
    for l in range(2):
        exact = float(np.max(np.abs(hh[l]) ** 2))
        assert convolution.power_iteration(hh[l], iters=3000) == pytest.approx(exact, rel=1e-8)
