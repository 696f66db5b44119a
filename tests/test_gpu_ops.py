"""Tier-1 parity: each CUDA operator against the FP64 oracle, element by
element, over sizes that span several tiles, partial tiles and degenerate
levels.  Tolerances (relative L2, FP32 kernels vs FP64): gradient 1e-6,
wavelet analysis/synthesis 1e-6, 3xTF32 DCT 2e-6."""
import numpy as np
import pytest

from oracle import convolution, spectral, wavelets
from oracle.daubechies import filter_bank
from synth import make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _plan(pkg, c, **kw):
    kw.setdefault("levels", min(3, int(np.log2(c.n))))
    return pkg.Plan(c.n, c.L, c.psf, **kw)


@pytest.mark.parametrize("n,L", [(2, 1), (4, 3), (8, 2), (64, 8), (256, 4)])
def test_gradient_matches_oracle(n, L):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(1, n // 4), 1 if n >= 8 else 0, 40 * n, seed=100 + n)
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, (L, n, n)).astype(np.float32)
    hh = convolution.psf_spectrum(c.psf)
    y = c.dirty.astype(np.float64)
    ref = convolution.HT(convolution.H(x.astype(np.float64), hh) - y, hh)
    ref_hth = convolution.HT(convolution.H(x.astype(np.float64), hh), hh)
    with _plan(pkg, c) as plan:
        g = torch.empty((L, n, n), device="cuda")
        plan.op_gradient(dev(x, torch), g, dirty=dev(c.dirty, torch))
        e1 = rel_l2(host(g), ref)
        plan.op_gradient(dev(x, torch), g)
        e2 = rel_l2(host(g), ref_hth)
        assert plan.lipschitz == pytest.approx(convolution.lipschitz(hh), rel=1e-12)
    print(f"gradient n={n}: {e1:.2e} (H^T H x - b), {e2:.2e} (H^T H x)")
    assert e1 <= 1e-6, e1
    assert e2 <= 1e-6, e2


def test_gradient_host_buffers_equal_device_buffers():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 3, 5, 1, 600, seed=7)
    x = np.random.default_rng(1).uniform(0, 1, (3, 32, 32)).astype(np.float32)
    with _plan(pkg, c) as plan:
        gd = torch.empty((3, 32, 32), device="cuda")
        plan.op_gradient(dev(x, torch), gd, dirty=dev(c.dirty, torch))
        gh = np.empty((3, 32, 32), np.float32)
        plan.op_gradient(x, gh, dirty=c.dirty)
    assert np.array_equal(host(gd), gh.astype(np.float64))


WAVE_CASES = [(2, 1, 1, 1), (4, 2, 8, 2), (8, 3, 8, 3), (16, 1, 8, 3), (64, 2, 3, 3),
              (128, 2, 8, 3), (256, 1, 8, 3), (64, 2, 8, 0), (32, 1, 8, 1), (128, 1, 2, 5)]


@pytest.mark.parametrize("n,L,K,J", WAVE_CASES)
def test_wavelet_analysis_matches_oracle(n, L, K, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    bank = filter_bank(K)
    rng = np.random.default_rng(n * 10 + K + J)
    x = rng.standard_normal((L, n, n)).astype(np.float32)
    ref = wavelets.Ws(x.astype(np.float64), bank, J)            # [L, K, n, n]
    psf = np.zeros((L, n, n), np.float32); psf[:, 0, 0] = 1
    with pkg.Plan(n, L, psf, n_wavelets=K, levels=J) as plan:
        u = torch.empty((L, K, n, n), device="cuda")
        plan.op_analysis(dev(x, torch), u)
        e = rel_l2(host(u), ref)
    assert e <= 1e-6, e


@pytest.mark.parametrize("n,L,K,J", WAVE_CASES)
def test_wavelet_synthesis_matches_oracle(n, L, K, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    bank = filter_bank(K)
    rng = np.random.default_rng(n * 7 + K + J)
    u = rng.standard_normal((L, K, n, n)).astype(np.float32)
    ref = wavelets.WsT(u.astype(np.float64), bank, J)
    psf = np.zeros((L, n, n), np.float32); psf[:, 0, 0] = 1
    with pkg.Plan(n, L, psf, n_wavelets=K, levels=J) as plan:
        x = torch.empty((L, n, n), device="cuda")
        plan.op_synthesis(dev(u, torch), x)
        e = rel_l2(host(x), ref)
    assert e <= 1e-6, e


@pytest.mark.parametrize("n,L", [(4, 1), (8, 5), (16, 16), (32, 64), (8, 100), (64, 33)])
@pytest.mark.parametrize("inverse", [False, True])
def test_dct_matches_oracle(n, L, inverse):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    rng = np.random.default_rng(L + n)
    x = rng.standard_normal((L, n, n)).astype(np.float32)
    C = spectral.dct_matrix(L)
    ref = spectral.apply_spectra(C.T if inverse else C, x.astype(np.float64))
    psf = np.zeros((L, n, n), np.float32); psf[:, 0, 0] = 1
    with pkg.Plan(n, L, psf, n_wavelets=1, levels=1) as plan:
        v = torch.empty((L, n, n), device="cuda")
        plan.op_dct(dev(x, torch), v, inverse=inverse)
        e = rel_l2(host(v), ref)
    assert e <= 2e-6, e


def test_full_size_operators_sampled():
    """1024^2 x 64 (the ADA-PT workload's shape): every operator on the full
    cube in its production launch configuration, checked on sampled bands
    (spatial operators) and sampled pixels (spectral operator)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 1024, 64
    c = make_cube(n, L, 2000, 100, 200000, seed=3, with_delta=False)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (L, n, n)).astype(np.float32)
    bands = [0, 37]
    with pkg.Plan(n, L, c.psf) as plan:
        xd = dev(x, torch)
        g = torch.empty_like(xd)
        plan.op_gradient(xd, g, dirty=dev(c.dirty, torch))
        u = torch.empty((L, 8, n, n), device="cuda")
        plan.op_analysis(xd, u)
        s = torch.empty_like(xd)
        plan.op_synthesis(u, s)
        v = torch.empty_like(xd)
        plan.op_dct(xd, v)
        for l in bands:
            hh = convolution.psf_spectrum(c.psf[l:l + 1])
            ref = convolution.HT(convolution.H(x[l:l + 1].astype(np.float64), hh)
                                 - c.dirty[l:l + 1].astype(np.float64), hh)
            eg = rel_l2(host(g[l:l + 1]), ref)
            print(f"gradient 1024 band {l}: {eg:.2e}")
            assert eg <= 1e-6
            ub = wavelets.Ws(x[l:l + 1].astype(np.float64), filter_bank(8), 3)
            assert rel_l2(host(u[l:l + 1]), ub) <= 1e-6
            # W_s^T W_s = 8 I: synthesis of the analysis returns 8 x
            assert rel_l2(host(s[l]), 8.0 * x[l]) <= 1e-6
        pix = rng.integers(0, n * n, 512)
        C = spectral.dct_matrix(L)
        xs = x.reshape(L, -1)[:, pix].astype(np.float64)
        vs = host(v).reshape(L, -1)[:, pix]
        assert rel_l2(vs, C @ xs) <= 2e-6
