"""Parity of ADA-PT'ed MUFFIN (Algorithm 5 with Algorithms 3/4 fused into
the primal kernels) against the FP64 oracle.  Tolerances: restored cube
relative L2 1e-5, tuned (mu, gamma) relative 1e-3, per-window SUGAR and
PSURE relative 1e-3."""
import numpy as np
import pytest

from oracle import muffin as om, sure as osure
from synth import fdmc_eps, make_cube, make_workload
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def gpu_tune(c, theta0, iters, window, eta, eps, x0=None, reset=True, **kw):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    x = dev(np.zeros_like(c.dirty) if x0 is None else x0, torch)
    with pkg.Plan(c.n, c.L, c.psf, sure=True, **kw) as plan:
        th, trace, info = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch),
                                         c.noise_var, x, theta0, iters, window=window,
                                         eta=eta, eps=eps, reset=reset)
    return host(x), np.array(th), trace, info


def oracle_tune(c, theta0, iters, window, eta, eps, reset=True, n_wavelets=8, levels=3):
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=n_wavelets, J=levels)
    return osure.ada_pt(prob, c.delta, eps, c.noise_var, theta0, iters, Delta=window,
                        eta=eta, reset=reset)


def check(c, theta0, iters, window, eta, reset=True, interior=True, **kw):
    """interior: theta stays well above theta_min in both components (checked
    on the oracle's run), so the theta comparison is not vacuous; the change
    of theta over the run is compared as well as its end point."""
    eps = fdmc_eps(c.noise_var)
    xg, th, trace, _ = gpu_tune(c, theta0, iters, window, eta, eps, reset=reset, **kw)
    ref = oracle_tune(c, theta0, iters, window, eta, eps, reset=reset, **kw)
    assert len(trace) == len(ref.trace) == iters // window
    for tg, to in zip(trace, ref.trace):
        assert tg["k"] == to["k"]
        assert tg["sugar_mu"] == pytest.approx(to["sugar"][0], rel=1e-3, abs=1e-6)
        assert tg["sugar_gamma"] == pytest.approx(to["sugar"][1], rel=1e-3, abs=1e-6)
        assert tg["psure"] == pytest.approx(to["psure"], rel=1e-3)
    th_rel = np.max(np.abs(th - ref.theta) / np.abs(ref.theta))
    e = rel_l2(xg, ref.x)
    print(f"theta gpu {th} oracle {ref.theta} rel {th_rel:.2e}; cube rel L2 {e:.2e}")
    assert th_rel <= 1e-3, th_rel
    assert e <= 1e-5, e
    if interior:
        for j in range(2):
            assert ref.theta[j] > 1e-6, f"theta[{j}] reached the clamp"
            d_ref, d_gpu = ref.theta[j] - theta0[j], th[j] - theta0[j]
            assert abs(d_ref) > 1e-3 * theta0[j], f"theta[{j}] did not move"
            assert abs(d_gpu - d_ref) <= 2e-2 * abs(d_ref), (j, d_gpu, d_ref)
    else:
        assert not np.allclose(ref.theta, theta0)    # the tuning moved theta
    return ref


def test_sure_small():
    c = make_cube(32, 8, 10, 2, 800, seed=12)
    check(c, (0.05, 0.05), 20, 5, (2e-5, 2e-4))


def test_sure_small_mu_clamped():
    """Large eta_mu drives mu to theta_min (the clamp of Eq. adaptgrad)."""
    c = make_cube(32, 8, 10, 2, 800, seed=12)
    ref = check(c, (0.05, 0.05), 20, 5, (2e-4, 2e-4), interior=False)
    assert ref.theta[0] == 1e-8


def test_sure_c1_workload():
    c = make_workload("c1_64x64x8")
    check(c, (1e-2, 1e-2), 60, 10, (1e-5, 5e-5))


def test_sure_no_reset_and_short_windows():
    c = make_cube(16, 4, 6, 1, 400, seed=13)
    check(c, (0.05, 0.02), 12, 3, (1e-4, 1e-4), reset=False, n_wavelets=3, levels=2)


def test_sure_crop_of_the_tuning_workload():
    """256^2 x 16 crop with the 1024^2 x 64 cube's densities, window 10."""
    c = make_cube(256, 16, 125, 6, 12500, seed=3)
    check(c, (1e-2, 1e-2), 20, 10, (3e-7, 3e-6))


def test_sure_512_size_specialised_kernels():
    """512^2 x 2: the analysis kernels compiled for a 512 px side (levels 1
    and 2) against the oracle, one window of two iterations."""
    c = make_cube(512, 2, 30, 2, 3000, seed=31)
    check(c, (1e-2, 1e-2), 2, 2, (2e-3, 2e-2))


def test_full_size_eta_zero_primal_equals_plain_solve():
    """1024^2 x 64 (the tuning workload's shape, size-specialised kernels):
    with eta = 0 the ADA-PT primal chain is the plain iteration, bit for bit
    (the plain iteration at this size is checked against the oracle in
    test_gpu_muffin)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 1024, 64
    c = make_cube(n, L, 2000, 100, 200000, seed=3)
    eps = fdmc_eps(c.noise_var)
    d = dev(c.dirty, torch)
    xs = torch.zeros_like(d)
    with pkg.Plan(n, L, c.psf, sure=True) as plan:
        th, _, _ = plan.sure_tune(d, dev(c.delta, torch), c.noise_var, xs, (1e-2, 1e-2), 4,
                                  window=2, eta=(0.0, 0.0), eps=eps)
    assert tuple(th) == (1e-2, 1e-2)
    x = torch.zeros_like(d)
    with pkg.Plan(n, L, c.psf) as plan:
        plan.solve(d, x, 4, 1e-2, 1e-2)
    torch.cuda.synchronize()
    assert torch.equal(xs, x)


def test_eta_zero_primal_equals_plain_solve():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(64, 4, 10, 2, 1500, seed=14)
    eps = fdmc_eps(c.noise_var)
    xs, th, _, _ = gpu_tune(c, (1e-2, 1e-2), 20, 5, (0.0, 0.0), eps)
    assert tuple(th) == (1e-2, 1e-2)
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(64, 4, c.psf) as plan:
        plan.solve(dev(c.dirty, torch), x, 20, 1e-2, 1e-2)
    assert np.array_equal(xs, host(x))


def test_sure_warm_and_resume_bitwise():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 700, seed=15)
    eps = fdmc_eps(c.noise_var)
    d, de = dev(c.dirty, torch), dev(c.delta, torch)
    args = dict(window=4, eta=(1e-4, 1e-4), eps=eps)
    x_full = torch.zeros_like(d)
    with pkg.Plan(32, 4, c.psf, sure=True) as p:
        th_full, tr_full, _ = p.sure_tune(d, de, c.noise_var, x_full, (0.03, 0.03), 24, **args)
    x_part = torch.zeros_like(d)
    with pkg.Plan(32, 4, c.psf, sure=True) as p:
        p.sure_tune(d, de, c.noise_var, x_part, (0.03, 0.03), 10, **args)
        blob = p.state_export()
    with pkg.Plan(32, 4, c.psf, sure=True) as p:
        p.state_import(blob)
        th_res, tr_res, _ = p.sure_tune(None, None, None, x_part, (0, 0), 14, warm=True, **args)
    assert torch.equal(x_full, x_part)
    assert th_full == th_res
    assert [t["k"] for t in tr_res] == [12, 16, 20, 24]
    assert tr_res[-1] == tr_full[-1]
