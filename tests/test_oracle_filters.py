"""Pins of the oracle's Daubechies filters against their defining properties.

db1..db8 (Sec. 4.2.1) are fixed by: sum h = sqrt(2), double-shift
orthonormality, p vanishing moments of the wavelet, minimum phase, and the
closed forms of db1 and db2.
"""
import math

import numpy as np
import pytest

from oracle.daubechies import daubechies_highpass, daubechies_lowpass


@pytest.mark.parametrize("p", range(1, 9))
def test_sum_and_length(p):
    h = daubechies_lowpass(p)
    assert len(h) == 2 * p
    assert abs(h.sum() - math.sqrt(2.0)) < 1e-13


@pytest.mark.parametrize("p", range(1, 9))
def test_double_shift_orthonormal(p):
    h = daubechies_lowpass(p)
    for m in range(p):
        c = float(np.dot(h[: len(h) - 2 * m], h[2 * m:]))
        assert abs(c - (1.0 if m == 0 else 0.0)) < 1e-12, (m, c)


@pytest.mark.parametrize("p", range(1, 9))
def test_vanishing_moments(p):
    h = daubechies_lowpass(p)
    g = daubechies_highpass(h)
    i = np.arange(2 * p, dtype=np.float64)
    for r in range(p):
        w = i ** r
        assert abs(np.dot(w, g)) <= 1e-11 * np.dot(w, np.abs(g)), r
    # the p-th moment must NOT vanish (exactly p moments)
    w = i ** p
    assert abs(np.dot(w, g)) > 1e-6 * np.dot(w, np.abs(g))


@pytest.mark.parametrize("p", range(2, 9))
def test_minimum_phase(p):
    # zeros of H(z) = sum h[k] z^{-k}: all inside or on the unit circle
    h = daubechies_lowpass(p)
    # p-fold zero at z = -1 (deflate it exactly), the rest strictly inside
    q, rem = np.polydiv(h, np.poly([-1.0] * p))
    assert np.max(np.abs(rem)) < 1e-10
    assert np.all(np.abs(np.roots(q)) < 1.0)
    # energy concentrated at the start (partial energies dominate the reversal)
    e = np.cumsum(h ** 2)
    e_rev = np.cumsum(h[::-1] ** 2)
    assert np.all(e >= e_rev - 1e-12)


def test_db1_haar():
    assert np.allclose(daubechies_lowpass(1), [2 ** -0.5, 2 ** -0.5], atol=1e-15)


def test_db2_closed_form():
    s3 = math.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.allclose(daubechies_lowpass(2), ref, atol=1e-14)


def test_highpass_qmf():
    h = daubechies_lowpass(3)
    g = daubechies_highpass(h)
    assert np.allclose(g, [h[5], -h[4], h[3], -h[2], h[1], -h[0]])
    assert abs(g.sum()) < 1e-14
