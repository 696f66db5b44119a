"""Properties of the seeded workload generator (inputs only, no method)."""
import numpy as np
import pytest

from synth import WORKLOADS, fdmc_eps, make_cube, make_workload, serve_stream


def test_deterministic_and_shapes():
    a = make_workload("c1_64x64x8")
    b = make_workload("c1_64x64x8")
    for f in ("sky", "psf", "dirty", "delta"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
        assert getattr(a, f).shape == (8, 64, 64)
        assert getattr(a, f).dtype == np.float32
    assert a.voxels == 64 * 64 * 8


def test_psf_real_even_peak_one():
    c = make_cube(32, 4, 10, 2, 800, seed=3)
    for l in range(4):
        p = c.psf[l].astype(np.float64)
        assert p[0, 0] == 1.0
        # Hermitian-mirrored gridding -> even PSF: p(-y, -x) = p(y, x)
        pr = np.roll(np.flip(p, (0, 1)), 1, axis=(0, 1))
        assert np.allclose(p, pr, atol=1e-6)
        assert np.max(np.abs(p)) <= 1.0 + 1e-6


def test_noise_at_requested_snr():
    c = make_cube(64, 3, 20, 3, 2000, seed=1, snr_db=20.0)
    for l in range(3):
        hx = np.fft.irfft2(np.fft.rfft2(c.psf[l].astype(np.float64)) *
                           np.fft.rfft2(c.sky[l].astype(np.float64)), s=(64, 64))
        assert c.noise_var[l] == pytest.approx(np.sum(hx ** 2) / (64 * 64 * 100.0))
        w = c.dirty[l] - hx
        assert np.var(w) == pytest.approx(c.noise_var[l], rel=0.1)
    assert fdmc_eps(c.noise_var) == pytest.approx(0.1 * np.sqrt(np.mean(c.noise_var)))


def test_sky_positive_and_spectra_power_law():
    c = make_cube(32, 5, 3, 0, 500, seed=4)
    assert np.all(c.sky >= 0)
    # point-source-only sky: ratios between bands follow (nu_l/nu_0)^alpha
    nz = np.argwhere(c.sky[0] > 0)
    y, x = nz[0]
    s = c.sky[:, y, x].astype(np.float64)
    alpha = np.log(s[-1] / s[0]) / np.log(c.nu[-1])
    assert np.allclose(s, s[0] * c.nu ** alpha, rtol=1e-5)
    assert np.allclose(c.nu, 1 + np.arange(5) / 4)


def test_registry_and_stream():
    assert WORKLOADS["c3_1024x1024x64"][:2] == (1024, 64)
    st = serve_stream()
    assert len(st) == 64
    assert all(n in (128, 256, 512) and L in (16, 32, 64) for _, n, L, _ in st)
    assert all(b[0] > a[0] for a, b in zip(st, st[1:]))
