"""Visibility-domain data term on the GPU (muffin_plan_load_visibilities):
Algorithm 2 from gridded visibilities against the FP64 oracle
(oracle/visibility.py), against the same GPU solve on the equivalent
image-domain problem, in batches, and its input checks."""
import numpy as np
import pytest

from oracle import visibility as ovis
from synth import make_visibilities
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _unit_psf(L, n):
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1
    return psf


def _vis_solve(pkg, torch, c, iters, mu=1e-2, gamma=2e-2, **kw):
    x = torch.zeros((c.L, c.n, c.n), device="cuda")
    with pkg.Plan(c.n, c.L, _unit_psf(c.L, c.n), **kw) as p:
        p.load_visibilities(c.vis, c.weights)
        info = p.solve(None, x, iters, mu, gamma)
    return host(x), info


@pytest.mark.parametrize("n,L,iters", [(16, 8, 30), (32, 64, 20), (64, 4, 25), (8, 16, 40)])
def test_visibility_solve_matches_oracle(n, L, iters):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_visibilities(n, L, max(2, n // 4), 1, 40 * n, seed=5000 + n + L)
    x, info = _vis_solve(pkg, torch, c, iters)
    st, tau = ovis.solve(c.vis, c.weights, 1e-2, 2e-2, iters)
    e = rel_l2(x, st.x)
    print(f"visibilities {n}^2 x {L}, {iters} iterations: {e:.1e}")
    assert info.lipschitz == pytest.approx(ovis.lipschitz(c.weights), rel=1e-12)
    assert info.tau == pytest.approx(tau, rel=1e-12)
    assert e <= 1e-5
    assert np.max(st.x) > 0


def test_visibility_equals_equivalent_image_problem():
    """The same data term as a convolution: PSF = F^-1 sqrt(m~), dirty y with
    H^T y = Re U^H D (both from the oracle), solved from the dirty cube."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 32, 8
    c = make_visibilities(n, L, 8, 1, 1200, seed=5100)
    xv, _ = _vis_solve(pkg, torch, c, 30)
    hh, y = ovis.equivalent_image_problem(c.vis, c.weights)
    psf = np.fft.ifft2(hh).real.astype(np.float32)
    x = torch.zeros((L, n, n), device="cuda")
    with pkg.Plan(n, L, psf) as p:
        p.solve(dev(y.real.astype(np.float32), torch), x, 30, 1e-2, 2e-2)
    assert rel_l2(xv, host(x)) <= 1e-5


def test_visibility_batch_equals_singles_and_device_inputs():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 16, 8
    cs = [make_visibilities(n, L, 4, 1, 600, seed=5200 + i) for i in range(2)]
    singles = [_vis_solve(pkg, torch, c, 15)[0] for c in cs]
    xb = torch.zeros((2, L, n, n), device="cuda")
    with pkg.Plan(n, L, np.stack([_unit_psf(L, n)] * 2), batch=2) as p:
        vis = torch.from_numpy(np.stack([c.vis for c in cs])).cuda()
        w = torch.from_numpy(np.stack([c.weights for c in cs])).cuda()
        p.load_visibilities(vis, w)
        p.solve(None, xb, 15, 1e-2, 2e-2)
    for i in range(2):
        assert np.array_equal(host(xb[i]), singles[i])


def test_visibility_input_checks():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 8, 4
    c = make_visibilities(n, L, 2, 1, 200, seed=5300)
    x = torch.zeros((L, n, n), device="cuda")
    with pkg.Plan(n, L, _unit_psf(L, n), sure=True) as p:
        with pytest.raises(pkg.MuffinError):
            p.solve(None, x, 5, 1e-2, 1e-2)           # no data term loaded
        w = c.weights.copy()
        w[1, 2, 3] = -1.0
        with pytest.raises(pkg.MuffinError):
            p.load_visibilities(c.vis, w)
        with pytest.raises(pkg.MuffinError):
            p.load_visibilities(c.vis, np.zeros_like(c.weights))
        v = c.vis.copy()
        v[0, 1, 1] = np.nan
        with pytest.raises(pkg.MuffinError):
            p.load_visibilities(v, c.weights)
        p.load_visibilities(c.vis, c.weights)
        p.solve(None, x, 5, 1e-2, 1e-2)
        assert torch.isfinite(x).all()
        with pytest.raises(pkg.MuffinError):         # ADA-PT needs a dirty cube
            p.sure_tune(None, dev(np.zeros((L, n, n), np.float32), torch), np.ones(L), x,
                        (1e-2, 1e-2), 5, window=5, eta=(0.0, 0.0), eps=1e-3)
