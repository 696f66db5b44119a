"""Tier-2 parity: the fused MUFFIN iteration (Algorithm 2) on the GPU against
the FP64 oracle after a fixed iteration count, plus warm continuation and
checkpoint/resume.  Cube tolerance: relative L2 1e-5 (FP32 state vs FP64)."""
import numpy as np
import pytest

from oracle import convolution, muffin as om, spectral, wavelets
from oracle.daubechies import filter_bank
from synth import make_cube, make_workload
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu

CUBE_TOL = 1e-5


def run_gpu(c, iters, mu, gamma, x0=None, **kw):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    x = dev(np.zeros_like(c.dirty) if x0 is None else x0, torch)
    with pkg.Plan(c.n, c.L, c.psf, **kw) as plan:
        info = plan.solve(dev(c.dirty, torch), x, iters, mu, gamma)
    return host(x), info


def run_oracle(c, iters, mu, gamma, x0=None, n_wavelets=8, levels=3, step_rule=0,
               positivity=True, alpha=None, beta=None):
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=n_wavelets, J=levels,
                           positivity=positivity, alpha_w=alpha, beta_w=beta)
    st, tau = om.solve(prob, mu, gamma, iters, x0=x0, step_rule=step_rule)
    return st.x, tau


def test_c1_200_iterations():
    """64x64x8, mu = gamma = 1e-2, 200 iterations (the FP64-vs-FP32 workload)."""
    c = make_workload("c1_64x64x8")
    xg, info = run_gpu(c, 200, 1e-2, 1e-2)
    xo, tau = run_oracle(c, 200, 1e-2, 1e-2)
    assert info.tau == pytest.approx(tau, rel=1e-12)
    e = rel_l2(xg, xo)
    print(f"c1 200 it: rel L2 {e:.3e}")
    assert e <= CUBE_TOL, e
    assert np.all(xg >= 0)


@pytest.mark.parametrize("case", [
    dict(n=16, L=3, n_wavelets=8, levels=3),
    dict(n=32, L=5, n_wavelets=3, levels=2, step_rule=1),
    dict(n=8, L=1, n_wavelets=8, levels=3),
    dict(n=16, L=4, n_wavelets=8, levels=0),
    dict(n=32, L=2, n_wavelets=2, levels=1, positivity=False),
    dict(n=128, L=2, n_wavelets=8, levels=3),
])
def test_small_variants(case):
    case = dict(case)
    n, L = case.pop("n"), case.pop("L")
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=n + L)
    mu, gamma, iters = 2e-2, 3e-2, 60
    xg, _ = run_gpu(c, iters, mu, gamma, **case)
    xo, _ = run_oracle(c, iters, mu, gamma, **case)
    e = rel_l2(xg, xo)
    assert e <= CUBE_TOL, e


def test_weights_and_initial_cube():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 800, seed=9)
    rng = np.random.default_rng(2)
    alpha = rng.uniform(0.5, 1.5, (32, 32)).astype(np.float32)
    beta = rng.uniform(0.5, 1.5, 4).astype(np.float32)
    x0 = rng.uniform(0, 0.1, (4, 32, 32)).astype(np.float32)
    x = dev(x0, torch)
    with pkg.Plan(32, 4, c.psf, alpha=alpha, beta=beta) as plan:
        plan.solve(dev(c.dirty, torch), x, 50, 3e-2, 2e-2)
    xo, _ = run_oracle(c, 50, 3e-2, 2e-2, x0=x0.astype(np.float64),
                       alpha=alpha.astype(np.float64), beta=beta.astype(np.float64))
    assert rel_l2(host(x), xo) <= CUBE_TOL


def test_zero_iterations_and_empty_regularisation():
    c = make_cube(16, 2, 4, 1, 300, seed=4)
    x0 = np.random.default_rng(0).uniform(0, 1, (2, 16, 16)).astype(np.float32)
    xg, _ = run_gpu(c, 0, 1e-2, 1e-2, x0=x0)
    assert np.array_equal(xg, x0.astype(np.float64))
    # mu = gamma = 0: projected gradient descent
    xg, _ = run_gpu(c, 30, 0.0, 0.0)
    xo, _ = run_oracle(c, 30, 0.0, 0.0)
    assert rel_l2(xg, xo) <= CUBE_TOL


def test_warm_continuation_and_checkpoint_resume_bitwise():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(64, 4, 10, 2, 1500, seed=21)
    d = dev(c.dirty, torch)
    x_full = torch.zeros_like(d)
    with pkg.Plan(64, 4, c.psf) as p:
        p.solve(d, x_full, 40, 1e-2, 1e-2)
    x_part = torch.zeros_like(d)
    with pkg.Plan(64, 4, c.psf) as p:
        p.solve(d, x_part, 15, 1e-2, 1e-2)
        blob = p.state_export()
        p.solve(None, x_part, 25, 1e-2, 1e-2, warm=True)
    assert torch.equal(x_full, x_part)
    x_res = torch.zeros_like(d)
    with pkg.Plan(64, 4, c.psf) as p:
        p.state_import(blob)
        p.solve(None, x_res, 25, 1e-2, 1e-2, warm=True)
    assert torch.equal(x_full, x_res)


def test_invalid_calls():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(16, 2, 4, 1, 300, seed=4)
    with pkg.Plan(16, 2, c.psf) as p:
        x = torch.zeros((2, 16, 16), device="cuda")
        with pytest.raises(pkg.MuffinError) as e:
            p.solve(None, x, 5, 1e-2, 1e-2, warm=True)
        assert e.value.status == 6
        with pytest.raises(pkg.MuffinError) as e:
            p.solve(dev(c.dirty, torch), x, -1, 1e-2, 1e-2)
        assert e.value.status == 1
        with pytest.raises(pkg.MuffinError) as e:
            p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                        (1e-2, 1e-2), 10, eps=0.1)
        assert e.value.status == 6
        with pytest.raises(pkg.MuffinError):
            p.state_import(b"\0" * 16)
    with pytest.raises(pkg.MuffinError) as e:
        pkg.Plan(16, 2, np.zeros((2, 16, 16), np.float32))
    assert e.value.status == 1


def test_full_size_two_iterations_sampled_bands():
    """1024^2 x 64: two fused iterations from a random X0; bands 3 and 50 are
    recomputed by the oracle's operators in Algorithm 2's order (the spectral
    step needs every band at every pixel, which the oracle computes exactly)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, mu, gamma = 1024, 64, 1e-2, 1e-2
    c = make_cube(n, L, 2000, 100, 200000, seed=3, with_delta=False)
    x0 = np.random.default_rng(8).uniform(0, 0.05, (L, n, n)).astype(np.float32)
    x = dev(x0, torch)
    with pkg.Plan(n, L, c.psf) as plan:
        info = plan.solve(dev(c.dirty, torch), x, 2, mu, gamma)
    tau, sig = info.tau, 10.0
    hh = convolution.psf_spectrum(c.psf)
    bank = filter_bank(8)
    C = spectral.dct_matrix(L)
    y = c.dirty.astype(np.float64)
    X0 = x0.astype(np.float64)
    # iteration 1 (U = V = T = 0): all bands for the gradient and prox
    g1 = convolution.HT(convolution.H(X0, hh) - y, hh)
    x1 = np.maximum(X0 - tau * g1, 0.0) * (X0 - tau * g1 > 0)
    z1 = 2 * x1 - X0
    v1 = np.clip(sig * gamma * spectral.apply_spectra(C, z1), -1, 1)
    t1 = gamma * spectral.apply_spectra(C.T, v1)
    xg = host(x)
    for l in (3, 50):
        u1 = np.clip(sig * mu * wavelets.Ws(z1[l:l + 1], bank, 3), -1, 1)
        g2 = convolution.HT(convolution.H(x1[l:l + 1], hh[l:l + 1]) - y[l:l + 1], hh[l:l + 1])
        s2 = mu * wavelets.WsT(u1, bank, 3)
        m2 = x1[l:l + 1] - tau * (g2 + s2 + t1[l:l + 1])
        x2 = np.where(m2 > 0, m2, 0.0)
        e = rel_l2(xg[l:l + 1], x2)
        assert e <= CUBE_TOL, (l, e)
    assert np.all(xg >= 0)
