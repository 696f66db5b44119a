"""The 2048 px side and the 256-band spectral step (the 2048^2 x 256
workload's shapes) against the FP64 oracle: the operators on sampled bands
in their production launch configuration, two fused plain iterations on
sampled bands, and the DCT of 256 bands (mma.sync kernel) on every pixel."""
import numpy as np
import pytest

from oracle import convolution, spectral, wavelets
from oracle.daubechies import filter_bank
from synth import make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def test_operators_2048_sampled():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 2048, 3
    c = make_cube(n, L, 500, 25, 60000, seed=55, with_delta=False)
    x = np.random.default_rng(6).uniform(0, 1, (L, n, n)).astype(np.float32)
    with pkg.Plan(n, L, c.psf) as plan:
        xd = dev(x, torch)
        g = torch.empty_like(xd)
        plan.op_gradient(xd, g, dirty=dev(c.dirty, torch))
        u = torch.empty((L, 8, n, n), device="cuda")
        plan.op_analysis(xd, u)
        s = torch.empty_like(xd)
        plan.op_synthesis(u, s)
    for l in (0, 2):
        hh = convolution.psf_spectrum(c.psf[l:l + 1])
        ref = convolution.HT(convolution.H(x[l:l + 1].astype(np.float64), hh)
                             - c.dirty[l:l + 1].astype(np.float64), hh)
        e = rel_l2(host(g[l:l + 1]), ref)
        print(f"2048 gradient band {l}: {e:.2e}")
        assert e <= 1e-6
        ub = wavelets.Ws(x[l:l + 1].astype(np.float64), filter_bank(8), 3)
        assert rel_l2(host(u[l:l + 1]), ub) <= 1e-6
        assert rel_l2(host(s[l]), 8.0 * x[l]) <= 1e-6


def test_two_iterations_2048_sampled_bands():
    """Two fused iterations of Algorithm 2 at 2048^2 x 4 from a random X0;
    bands 1 and 2 recomputed by the oracle's operators (the spectral step of
    the first iteration is computed exactly for every pixel)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, mu, gamma = 2048, 4, 1e-2, 1e-2
    c = make_cube(n, L, 500, 25, 60000, seed=56, with_delta=False)
    x0 = np.random.default_rng(9).uniform(0, 0.05, (L, n, n)).astype(np.float32)
    x = dev(x0, torch)
    with pkg.Plan(n, L, c.psf) as plan:
        info = plan.solve(dev(c.dirty, torch), x, 2, mu, gamma)
    tau, sig = info.tau, 10.0
    hh = convolution.psf_spectrum(c.psf)
    bank = filter_bank(8)
    C = spectral.dct_matrix(L)
    y = c.dirty.astype(np.float64)
    X0 = x0.astype(np.float64)
    g1 = convolution.HT(convolution.H(X0, hh) - y, hh)
    x1 = np.where(X0 - tau * g1 > 0, X0 - tau * g1, 0.0)
    z1 = 2 * x1 - X0
    v1 = np.clip(sig * gamma * spectral.apply_spectra(C, z1), -1, 1)
    t1 = gamma * spectral.apply_spectra(C.T, v1)
    xg = host(x)
    for l in (1, 2):
        u1 = np.clip(sig * mu * wavelets.Ws(z1[l:l + 1], bank, 3), -1, 1)
        g2 = convolution.HT(convolution.H(x1[l:l + 1], hh[l:l + 1]) - y[l:l + 1], hh[l:l + 1])
        s2 = mu * wavelets.WsT(u1, bank, 3)
        m2 = x1[l:l + 1] - tau * (g2 + s2 + t1[l:l + 1])
        x2 = np.where(m2 > 0, m2, 0.0)
        e = rel_l2(xg[l:l + 1], x2)
        assert e <= 1e-5, (l, e)


@pytest.mark.parametrize("inverse", [False, True])
def test_dct_256_bands(inverse):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 16, 256
    x = np.random.default_rng(10 + inverse).standard_normal((L, n, n)).astype(np.float32)
    C = spectral.dct_matrix(L)
    ref = spectral.apply_spectra(C.T if inverse else C, x.astype(np.float64))
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1
    with pkg.Plan(n, L, psf, n_wavelets=1, levels=1) as plan:
        v = torch.empty((L, n, n), device="cuda")
        plan.op_dct(dev(x, torch), v, inverse=inverse)
    assert rel_l2(host(v), ref) <= 2e-6


@pytest.mark.parametrize("n,L,sure", [(32, 256, False), (16, 128, True), (16, 100, True)])
def test_many_bands_iteration_matches_oracle(n, L, sure):
    """The spectral step with more than 64 bands (the wide-tile mma.sync
    kernel, one warp per 16-band tile of C) inside the iteration: plain
    MUFFIN and ADA-PT (three chains) against the oracle."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    from oracle import muffin as om, sure as osure
    from synth import fdmc_eps
    c = make_cube(n, L, 10, 1, 40 * n, seed=57 + L)
    prob = om.make_problem(c.dirty, c.psf)
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(n, L, c.psf, sure=sure) as plan:
        if sure:
            eps = fdmc_eps(c.noise_var)
            th, _, _ = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                      (1e-2, 1e-2), 8, window=4, eta=(1e-6, 1e-5), eps=eps)
            ref = osure.ada_pt(prob, c.delta, eps, c.noise_var, (1e-2, 1e-2), 8, Delta=4,
                               eta=(1e-6, 1e-5))
            assert np.allclose(th, ref.theta, rtol=1e-3, atol=0)
            ref_x = ref.x
        else:
            plan.solve(dev(c.dirty, torch), x, 20, 1e-2, 1e-2)
            ref_x = om.solve(prob, 1e-2, 1e-2, 20)[0].x
    assert rel_l2(host(x), ref_x) <= 1e-5
