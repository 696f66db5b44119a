"""Pins of the oracle's point metrics (Sec. 4.1), of the projections of
Sec. 2.2 (Eqs. projpos, sat) and of their weak derivatives used by
Algorithms 3/4 (Sec. 3.2), against closed forms and hand-worked cases."""
import numpy as np
import pytest

from oracle import convolution, metrics
from oracle import muffin as om
from oracle import sure as osure


def _cube(seed, L=3, n=16):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (L, n, n))


def test_snr_of_a_scaled_estimate_is_closed_form():
    x = _cube(1)
    # x - 0.9 x = 0.1 x: energy ratio 100, i.e. 20 dB
    assert metrics.snr_db(x, 0.9 * x) == pytest.approx(20.0, abs=1e-12)
    assert metrics.snr_db(x, 0.99 * x) == pytest.approx(40.0, abs=1e-10)


def test_snr_matches_its_definition_on_random_error():
    rng = np.random.default_rng(2)
    x = _cube(3)
    e = rng.normal(0.0, 0.05, x.shape)
    want = 10.0 * np.log10(np.sum(x * x) / np.sum(e * e))
    assert metrics.snr_db(x, x - e) == pytest.approx(want, rel=1e-12)


def test_wmse_with_identity_psf_is_the_mean_squared_error():
    x = _cube(4)
    y = _cube(5)
    psf = np.zeros_like(x)
    psf[:, 0, 0] = 1.0                       # H = I
    hh = convolution.psf_spectrum(psf)
    assert metrics.wmse(x, y, hh) == pytest.approx(np.mean((x - y) ** 2), rel=1e-12)


def test_wmse_with_a_shift_psf_is_unchanged_and_scales_quadratically():
    x, y = _cube(6), _cube(7)
    psf = np.zeros_like(x)
    psf[:, 3, 5] = 2.0                       # H = 2 x a circular shift
    hh = convolution.psf_spectrum(psf)
    # a shift preserves the norm, the factor 2 scales the squared error by 4
    assert metrics.wmse(x, y, hh) == pytest.approx(4.0 * np.mean((x - y) ** 2), rel=1e-10)


def test_projections_and_their_masks():
    u = np.array([-2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0])
    np.testing.assert_array_equal(om.sat(u), [-1.0, -1.0, -0.5, 0.0, 0.5, 1.0, 1.0])
    np.testing.assert_array_equal(om.pos(u), [0.0, 0.0, 0.0, 0.0, 0.5, 1.0, 2.0])
    # weak derivatives: U(m) = 1 where m > 0 (0 at the kink), Pi(p) = 1 on
    # the closed interval [-1, 1] (1 at the kinks)
    np.testing.assert_array_equal(osure.U_mask(u), [0, 0, 0, 0, 1, 1, 1])
    np.testing.assert_array_equal(osure.Pi_mask(u), [0, 1, 1, 1, 1, 1, 0])


def test_masks_are_the_derivatives_away_from_the_kinks():
    rng = np.random.default_rng(8)
    u = rng.uniform(-3.0, 3.0, 1000)
    u = u[(np.abs(u) > 1e-3) & (np.abs(np.abs(u) - 1.0) > 1e-3)]
    h = 1e-6
    d_pos = (om.pos(u + h) - om.pos(u - h)) / (2 * h)
    d_sat = (om.sat(u + h) - om.sat(u - h)) / (2 * h)
    np.testing.assert_allclose(osure.U_mask(u), d_pos, atol=1e-9)
    np.testing.assert_allclose(osure.Pi_mask(u), d_sat, atol=1e-9)
