"""Pins of the visibility-domain data term (oracle/visibility.py) against
definitions it does not use itself: sums over the samples one by one,
finite differences, the image-domain convolution model, the stationarity
of the noise-free truth and a power iteration for the Lipschitz constant."""
import numpy as np

from oracle import convolution, muffin as om, visibility as vis
from synth import make_visibilities


def _samples(n, count, seed):
    rng = np.random.default_rng(seed)
    ky = rng.integers(-n // 2, n // 2, count)
    kx = rng.integers(-n // 2, n // 2, count)
    ky[: count // 4] = ky[count // 4: 2 * (count // 4)]     # repeated cells
    kx[: count // 4] = kx[count // 4: 2 * (count // 4)]
    d = rng.standard_normal(count) + 1j * rng.standard_normal(count)
    return ky, kx, d


def test_gridded_gradient_equals_sample_sums():
    for n, count, seed in [(4, 9, 1), (8, 30, 2)]:
        ky, kx, d = _samples(n, count, seed)
        x = np.random.default_rng(seed + 10).standard_normal((n, n))
        D, m = vis.grid(ky, kx, d, n)
        g = vis.gradient(x[None], D[None], m[None])[0]
        gp = vis.point_gradient(x, ky, kx, d)
        assert np.max(np.abs(g - gp)) <= 1e-12 * max(1.0, np.max(np.abs(gp)))


def test_sample_gradient_finite_differences():
    n = 4
    ky, kx, d = _samples(n, 11, 3)
    x = np.random.default_rng(4).standard_normal((n, n))
    g = vis.point_gradient(x, ky, kx, d)
    h = 1e-6
    for (i, j) in [(0, 0), (1, 3), (3, 2)]:
        e = np.zeros((n, n))
        e[i, j] = h
        fd = (vis.data_term(x + e, ky, kx, d) - vis.data_term(x - e, ky, kx, d)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(g[i, j]))


def test_equals_image_domain_gradient():
    """Hermitian samples of a real sky: the visibility gradient is the image-
    domain gradient H^T (H x - y) with |h_hat|^2 = m~ and H^T y = Re U^H D."""
    c = make_visibilities(16, 3, 6, 1, 300, seed=5)
    hh, y = vis.equivalent_image_problem(c.vis, c.weights)
    assert np.max(np.abs(y.imag)) <= 1e-10 * np.max(np.abs(y.real))
    x = np.random.default_rng(6).uniform(0, 1, (3, 16, 16))
    gv = vis.gradient(x, c.vis.astype(np.complex128), c.weights)
    gi = convolution.HT(convolution.H(x, hh) - y.real, hh)
    assert np.max(np.abs(gv - gi)) <= 1e-10 * np.max(np.abs(gi))


def test_noise_free_truth_is_stationary():
    c = make_visibilities(16, 2, 6, 1, 300, seed=7)
    x = c.sky.astype(np.float64)
    m = c.weights.astype(np.float64)
    D = m * np.fft.fft2(x, norm="ortho")       # every sample exact
    g = vis.gradient(x, D, m)
    assert np.max(np.abs(g)) <= 1e-12 * np.max(np.abs(D))


def test_lipschitz_by_power_iteration():
    c = make_visibilities(8, 2, 3, 1, 80, seed=8)
    m = c.weights.astype(np.float64)
    v = np.random.default_rng(9).standard_normal((2, 8, 8))
    lam = 0.0
    for _ in range(400):
        w = vis.gradient(v, np.zeros_like(m, complex), m)
        lam = float(np.sum(v * w) / np.sum(v * v))
        v = w / np.linalg.norm(w)
    assert abs(lam - vis.lipschitz(m)) <= 1e-6 * vis.lipschitz(m)


def test_visibility_solve_equals_image_solve():
    c = make_visibilities(16, 4, 6, 1, 300, seed=10)
    st, tau = vis.solve(c.vis, c.weights, 1e-2, 2e-2, 12)
    hh, y = vis.equivalent_image_problem(c.vis, c.weights)
    psf = np.zeros((4, 16, 16))
    psf[:, 0, 0] = 1
    prob = om.make_problem(y.real, psf)
    prob.hhat = hh
    st_i, tau_i = om.solve(prob, 1e-2, 2e-2, 12)
    assert tau == tau_i
    assert np.max(np.abs(st.x - st_i.x)) <= 1e-10 * np.max(np.abs(st_i.x))
    assert np.max(st.x) > 0


def test_generator_hermitian():
    c = make_visibilities(16, 3, 6, 1, 300, seed=11)
    for l in range(3):
        D, m = c.vis[l], c.weights[l]
        Dm = np.roll(np.flip(D), 1, axis=(0, 1))
        mm = np.roll(np.flip(m), 1, axis=(0, 1))
        assert np.allclose(D, np.conj(Dm), atol=1e-5)
        assert np.array_equal(m, mm)
        assert np.all(m == np.rint(m)) and m.sum() % 2 == 0
