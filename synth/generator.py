"""Synthetic radio-interferometric cubes shaped like the paper's workloads.

The paper (Sec. 4.1) deconvolves 256x256x256 sky cubes observed through a
per-channel SKA1-MID PSF with white Gaussian noise at a fixed SNR.  Those
cubes and PSFs are not distributable, so every workload here is drawn from a
documented recipe instead:

* sky: point sources at uniform integer pixels with log-uniform amplitudes in
  [0.1, 1], plus circular Gaussian blobs (width 2..5 px, peak 0.3 at nu0,
  periodic distance); every component has its own power-law spectrum
  S(nu) = S0 (nu/nu0)^alpha, alpha ~ U(-1, 1), bands nu_l = nu0 (1 + l/(L-1));
* PSF: uv points ~ N(0, 0.15^2) cycles/px drawn once, scaled by nu_l/nu0 per
  band, dropped when a scaled coordinate reaches 0.5 cycles/px, gridded to the
  nearest Fourier cell together with the Hermitian mirror cell, inverse FFT'd
  (real part) and normalised to 1 at the origin pixel (0, 0);
* dirty cube: circular convolution of sky and PSF plus noise with per-band
  variance sigma_l^2 = ||h_l * x_l||^2 / (N 10^(SNR/10));
* delta: the N(0, I) probe of the finite-difference Monte-Carlo risk estimate
  (Sec. 3.1), drawn once here so both implementations see the same vector;
* visibilities (make_visibilities, the same sky and uv points): each kept uv
  point samples the unitary 2D DFT of the band's sky at its nearest cell k,
  d = (U x_l)_k + complex white noise (per-sample variance set by the SNR
  against the mean |(U x_l)_k|^2 of the samples), and its Hermitian mirror
  cell -k receives conj(d); the samples are gridded into per-cell sums D_l
  and counts m_l (natural weights).

Draw order from ``numpy.random.default_rng(seed)``: source positions,
amplitudes, source indices, blob centres, blob widths, blob indices, uv
points, noise (band by band), delta (band by band); for visibilities the
noise is one (n_kept, 2) standard normal draw per band.

All returned images are float32 (the arrays both implementations consume);
noise variances are float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# name -> (n, L, n_src, n_blob, n_uv, seed).  Source, blob and uv counts of the
# 256x256x16 crop follow the 2048^2 x 256 cube's densities per pixel.
WORKLOADS = {
    "c1_64x64x8": (64, 8, 20, 3, 2000, 1),
    "c2_256x256x32": (256, 32, 200, 20, 20000, 2),
    "c3_1024x1024x64": (1024, 64, 2000, 100, 200000, 3),
    "c5_2048x2048x256": (2048, 256, 8000, 400, 1000000, 5),
    "c5crop_256x256x16": (256, 16, 125, 6, 15625, 5),
    # a mid-size cube for profiler captures (state ~2 GB, inputs > L2)
    "prof_512x512x32": (512, 32, 500, 25, 50000, 6),
    "prof_512x512x64": (512, 64, 500, 25, 50000, 7),
    "prof_256x256x64": (256, 64, 125, 6, 12500, 8),
    "prof_256x256x256": (256, 256, 125, 6, 12500, 9),
}


@dataclasses.dataclass
class Cube:
    """One synthetic deconvolution problem (all images band-major [L][n][n])."""
    n: int
    L: int
    sky: np.ndarray        # float32 [L, n, n], the true cube X*
    psf: np.ndarray        # float32 [L, n, n], peak 1 at pixel (0, 0)
    dirty: np.ndarray      # float32 [L, n, n], Y = H X* + W
    noise_var: np.ndarray  # float64 [L], sigma_l^2
    delta: np.ndarray      # float32 [L, n, n], N(0, 1) FDMC probe
    nu: np.ndarray         # float64 [L], nu_l / nu0

    @property
    def voxels(self) -> int:
        return self.n * self.n * self.L


def _wrapped_gauss(n: int, centre: float, width: float) -> np.ndarray:
    d = np.abs(np.arange(n, dtype=np.float64) - centre)
    d = np.minimum(d, n - d)
    return np.exp(-0.5 * (d / width) ** 2)


def fdmc_eps(noise_var: np.ndarray) -> float:
    """FDMC step: 0.1 x the rms noise standard deviation over bands."""
    return 0.1 * math.sqrt(float(np.mean(noise_var)))


def _draw_sky_uv(n: int, L: int, n_src: int, n_blob: int, n_uv: int, rng):
    """nu_l / nu0, the float32 sky cube and the uv points (the first draws)."""
    if n < 2 or n & (n - 1):
        raise ValueError("image side must be a power of two >= 2")
    if L < 1:
        raise ValueError("need at least one band")
    nu = (1.0 + np.arange(L, dtype=np.float64) / (L - 1)) if L > 1 \
        else np.ones(1)

    pos = rng.integers(0, n, size=(n_src, 2))                   # (y, x)
    amp = np.exp(rng.uniform(math.log(0.1), math.log(1.0), n_src))
    a_src = rng.uniform(-1.0, 1.0, n_src)
    centres = rng.uniform(0.0, n, size=(n_blob, 2))             # (y, x)
    widths = rng.uniform(2.0, 5.0, n_blob)
    a_blob = rng.uniform(-1.0, 1.0, n_blob)
    uv = rng.normal(0.0, 0.15, size=(n_uv, 2))                  # (u, v)

    gy = np.stack([_wrapped_gauss(n, c[0], w) for c, w in zip(centres, widths)]) \
        if n_blob else np.zeros((0, n))
    gx = np.stack([_wrapped_gauss(n, c[1], w) for c, w in zip(centres, widths)]) \
        if n_blob else np.zeros((0, n))
    sky = np.empty((L, n, n), np.float32)
    for l in range(L):
        s = np.zeros((n, n), np.float64)
        np.add.at(s, (pos[:, 0], pos[:, 1]), amp * nu[l] ** a_src)
        if n_blob:
            w = 0.3 * nu[l] ** a_blob
            s += (gy * w[:, None]).T @ gx
        sky[l] = s
    return nu, sky, uv


def _cells(uv: np.ndarray, nu_l: float, n: int, l: int):
    """Nearest Fourier cells (ky, kx) of the uv points kept in band l."""
    sc = uv * nu_l
    keep = np.all(np.abs(sc) < 0.5, axis=1)
    kx = np.rint(sc[keep, 0] * n).astype(np.int64)
    ky = np.rint(sc[keep, 1] * n).astype(np.int64)
    if kx.size == 0:
        raise ValueError(f"band {l} has an empty uv coverage")
    return ky, kx


def make_cube(n: int, L: int, n_src: int, n_blob: int, n_uv: int,
              seed: int, snr_db: float = 20.0,
              with_delta: bool = True) -> Cube:
    rng = np.random.default_rng(seed)
    nu, sky, uv = _draw_sky_uv(n, L, n_src, n_blob, n_uv, rng)

    psf = np.empty((L, n, n), np.float32)
    dirty = np.empty((L, n, n), np.float32)
    noise_var = np.empty(L, np.float64)
    clean = np.empty((L, n, n), np.float64)
    N = n * n
    for l in range(L):
        # uv coverage of band l, nearest-cell gridding plus Hermitian mirror
        ky, kx = _cells(uv, nu[l], n, l)
        g = np.zeros((n, n), np.float64)
        np.add.at(g, (ky % n, kx % n), 1.0)
        np.add.at(g, ((-ky) % n, (-kx) % n), 1.0)
        p = np.fft.ifft2(g).real
        p /= p[0, 0]
        psf[l] = p
        # forward model on the float32 sky and PSF that both sides consume
        hx = np.fft.irfft2(np.fft.rfft2(psf[l].astype(np.float64)) *
                           np.fft.rfft2(sky[l].astype(np.float64)), s=(n, n))
        clean[l] = hx
        noise_var[l] = float(np.sum(hx * hx)) / (N * 10.0 ** (snr_db / 10.0))
    for l in range(L):
        dirty[l] = clean[l] + math.sqrt(noise_var[l]) * rng.standard_normal((n, n))
    del clean
    if with_delta:
        delta = np.empty((L, n, n), np.float32)
        for l in range(L):
            delta[l] = rng.standard_normal((n, n))
    else:
        delta = np.zeros((0,), np.float32)
    return Cube(n=n, L=L, sky=sky, psf=psf, dirty=dirty, noise_var=noise_var,
                delta=delta, nu=nu)


@dataclasses.dataclass
class VisCube:
    """Gridded visibilities of a synthetic sky (band-major [L][n][n])."""
    n: int
    L: int
    sky: np.ndarray        # float32 [L, n, n], the true cube X*
    vis: np.ndarray        # complex64 [L, n, n], per-cell sums D_l of the samples
    weights: np.ndarray    # float32 [L, n, n], per-cell sample counts m_l
    noise_std: np.ndarray  # float64 [L], per-sample noise std (real and imaginary)
    nu: np.ndarray         # float64 [L]


def make_visibilities(n: int, L: int, n_src: int, n_blob: int, n_uv: int,
                      seed: int, snr_db: float = 20.0) -> VisCube:
    rng = np.random.default_rng(seed)
    nu, sky, uv = _draw_sky_uv(n, L, n_src, n_blob, n_uv, rng)
    vis = np.zeros((L, n, n), np.complex128)
    weights = np.zeros((L, n, n), np.float64)
    noise_std = np.empty(L, np.float64)
    for l in range(L):
        ky, kx = _cells(uv, nu[l], n, l)
        spec = np.fft.fft2(sky[l].astype(np.float64), norm="ortho")
        s = spec[ky % n, kx % n]
        var = float(np.mean(np.abs(s) ** 2)) / 10.0 ** (snr_db / 10.0)
        noise_std[l] = math.sqrt(var / 2.0)
        w = rng.standard_normal((kx.size, 2))
        d = s + noise_std[l] * (w[:, 0] + 1j * w[:, 1])
        np.add.at(vis[l], (ky % n, kx % n), d)
        np.add.at(vis[l], ((-ky) % n, (-kx) % n), np.conj(d))
        np.add.at(weights[l], (ky % n, kx % n), 1.0)
        np.add.at(weights[l], ((-ky) % n, (-kx) % n), 1.0)
    return VisCube(n=n, L=L, sky=sky, vis=vis.astype(np.complex64),
                   weights=weights.astype(np.float32), noise_std=noise_std, nu=nu)


def make_workload(name: str, **kw) -> Cube:
    n, L, n_src, n_blob, n_uv, seed = WORKLOADS[name]
    return make_cube(n, L, n_src, n_blob, n_uv, seed, **kw)


def serve_stream(seed: int = 4, n_requests: int = 64, rate_hz: float = 4.0,
                 sides=(128, 256, 512), bands=(16, 32, 64)):
    """Poisson arrivals of cubes with uneven side and band counts.

    Returns a list of (arrival_s, n, L, request_seed).  Per-request cubes are
    generated with ``make_cube`` from seed 4000 + i and source/blob/uv
    densities per pixel equal to the 256^2 x 32 workload's.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps)
    ns = rng.choice(np.asarray(sides), n_requests)
    Ls = rng.choice(np.asarray(bands), n_requests)
    return [(float(t[i]), int(ns[i]), int(Ls[i]), 4000 + i)
            for i in range(n_requests)]
