"""Weights from an initial cube (Eq. 2regpar) and the global SUGAR descent
(Eq. globalgrad) through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import muffin as om
from oracle import weights as ow
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,K,J", [(32, 8, 8, 3), (16, 6, 4, 2), (8, 5, 8, 0), (64, 3, 2, 1)])
def test_weights_from_x0_match_oracle(n, L, K, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=900 + n + L)
    x0 = np.abs(c.dirty)                        # a positive coarse estimate
    with pkg.Plan(n, L, c.psf, n_wavelets=K, levels=J) as p:
        a, b = p.weights_from_x0(dev(x0, torch), 1e-2, 3e-3)
    ao, bo = ow.weights_from_x0(x0, K, J, 1e-2, 3e-3)
    assert rel_l2(a, ao) <= 1e-6 and rel_l2(b, bo) <= 1e-6
    assert np.max(np.abs(a / ao - 1)) <= 1e-6 and np.max(np.abs(b / bo - 1)) <= 1e-6


def test_weighted_solve_matches_oracle_and_set_weights():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 8, 10, 2, 1000, seed=910)
    d = dev(c.dirty, torch)
    with pkg.Plan(32, 8, c.psf) as p:
        x0 = torch.zeros_like(d)
        p.solve(d, x0, 10, 1e-2, 1e-2)          # coarse X0: ten plain iterations
        a, b = p.weights_from_x0(x0, 1e-3, 1e-3)
        x = torch.zeros_like(d)
        p.solve(d, x, 60, 0.5, 0.5)
    prob = om.make_problem(c.dirty, c.psf, alpha_w=a.astype(np.float64), beta_w=b.astype(np.float64))
    st, _ = om.solve(prob, 0.5, 0.5, 60)
    assert rel_l2(host(x), st.x) <= 1e-5
    # the same weights given explicitly give the same iterates, bit for bit
    with pkg.Plan(32, 8, c.psf) as p2:
        p2.set_weights(a.reshape(1, -1), b.reshape(1, -1))
        x2 = torch.zeros_like(d)
        p2.solve(d, x2, 60, 0.5, 0.5)
    assert torch.equal(x, x2)


def test_batched_weights_are_per_cube():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    cs = [make_cube(16, 4, 4, 1, 480, seed=920 + i) for i in range(3)]
    x0 = np.stack([np.abs(c.dirty) * (i + 1) for i, c in enumerate(cs)])
    with pkg.Plan(16, 4, np.stack([c.psf for c in cs]), batch=3) as p:
        a, b = p.weights_from_x0(x0, 1e-2, 1e-2)
    for i in range(3):
        ao, bo = ow.weights_from_x0(x0[i], 8, 3, 1e-2, 1e-2)
        assert rel_l2(a[i], ao) <= 1e-6 and rel_l2(b[i], bo) <= 1e-6


def _global_case():
    c = make_cube(16, 4, 6, 1, 300, seed=11)
    return c, fdmc_eps(c.noise_var)


def test_global_descent_matches_oracle():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c, eps = _global_case()
    eta = (2e-4, 2e-4)
    x = torch.zeros((4, 16, 16), device="cuda")
    with pkg.Plan(16, 4, c.psf, sure=True) as p:
        th, tr, info = p.sure_global(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                     (0.03, 0.02), n_c=8, outer=3, eta=eta, eps=eps)
    prob = om.make_problem(c.dirty, c.psf)
    xo, tho, recs = ow.global_descent(prob, c.delta, eps, c.noise_var, (0.03, 0.02), 3, 8, eta=eta)
    assert info.records == 3 and len(tr) == 3 and [r["k"] for r in tr] == [8, 8, 8]
    assert np.max(np.abs(np.array(th) / tho - 1)) <= 1e-3
    assert rel_l2(host(x), xo) <= 1e-5
    for r, ro in zip(tr, recs):
        np.testing.assert_allclose([r["mu"], r["gamma"]], ro["theta"], rtol=1e-3)
        np.testing.assert_allclose([r["sugar_mu"], r["sugar_gamma"]], ro["sugar"], rtol=2e-3)


def test_global_descent_zero_step_and_invalid():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c, eps = _global_case()
    d, de = dev(c.dirty, torch), dev(c.delta, torch)
    with pkg.Plan(16, 4, c.psf, sure=True) as p:
        x = torch.zeros((4, 16, 16), device="cuda")
        th, tr, _ = p.sure_global(d, de, c.noise_var, x, (0.03, 0.02), n_c=6, outer=3,
                                  eta=(0.0, 0.0), eps=eps)
        assert th == (0.03, 0.02)
        assert tr[0] == tr[1] == tr[2]
        y = torch.zeros_like(x)
        p.sure_tune(d, de, c.noise_var, y, (0.03, 0.02), 6, window=6, eta=(0.0, 0.0), eps=eps)
        assert torch.equal(x, y)
        with pytest.raises(pkg.MuffinError) as e:
            p.sure_global(d, de, c.noise_var, x, (0.03, 0.02), n_c=6, outer=-1, eps=eps)
        assert e.value.status == 1
        with pytest.raises(pkg.MuffinError) as e:
            p.weights_from_x0(x, -1.0, 0.0)
        assert e.value.status == 1
