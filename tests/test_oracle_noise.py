"""Pins of the oracle's MAD noise estimate (Sec. 3.1, read as the wavelet
MAD of Donoho and Johnstone on the finest Haar diagonal band)."""
import numpy as np
import pytest

from oracle import noise
from synth import make_cube


def test_haar_hh_is_the_two_by_two_difference():
    """The finest high-high Haar coefficient of pixels (2i, 2j)..(2i+1, 2j+1)
    is (a - b - c + d) / 2, written out element by element."""
    y = np.random.default_rng(0).standard_normal((8, 8))
    hh = noise.haar_hh(y)
    want = np.empty((4, 4))
    for i in range(4):
        for j in range(4):
            want[i, j] = (y[2 * i, 2 * j] - y[2 * i, 2 * j + 1] - y[2 * i + 1, 2 * j]
                          + y[2 * i + 1, 2 * j + 1]) / 2.0
    assert np.allclose(hh, want, atol=1e-14)


def test_mad_hand_cases():
    c = 0.6744897501960817
    assert noise.mad_sigma([1.0, 2.0, 3.0, 4.0, 100.0]) == pytest.approx(1.0 / c, rel=1e-15)
    assert noise.mad_sigma([4.0, 1.0, 3.0, 2.0]) == pytest.approx(1.0 / c, rel=1e-15)
    assert noise.mad_sigma([5.0]) == 0.0


def test_white_noise_level_is_recovered():
    rng = np.random.default_rng(1)
    sig = np.array([0.3, 1.7, 0.05])
    y = rng.standard_normal((3, 256, 256)) * sig[:, None, None]
    est = noise.noise_var_mad(y)
    assert np.allclose(np.sqrt(est), sig, rtol=0.03)


def test_constant_and_ramps_do_not_change_it_and_scale_does():
    rng = np.random.default_rng(2)
    y = rng.standard_normal((2, 32, 32))
    yy, xx = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    base = noise.noise_var_mad(y)
    assert np.allclose(noise.noise_var_mad(y + 5.0 + 0.3 * xx - 0.2 * yy), base, rtol=1e-12)
    assert np.allclose(noise.noise_var_mad(-3.0 * y), 9.0 * base, rtol=1e-12)


def test_noise_of_the_workload_recipe_is_recovered():
    """The noise the generator adds to a workload cube (dirty minus the
    convolved sky) has the per-band variance it reports: within 5 %."""
    from oracle import convolution
    c = make_cube(128, 4, 40, 4, 4000, seed=17)
    w = c.dirty.astype(np.float64) - convolution.H(c.sky.astype(np.float64),
                                                   convolution.psf_spectrum(c.psf))
    est = noise.noise_var_mad(w)
    assert np.allclose(est, c.noise_var, rtol=0.05), (est, c.noise_var)
