"""Convergence monitor, objective, numeric-failure scan and the n_c rule of
the global SUGAR descent, against the FP64 oracle.

* objective (Eqs. probopt, RegAll) of a given cube: <= 1e-6 relative;
* the monitor's checks during Algorithm 2: the objective at X^k <= 1e-6 of
  the oracle's at its X^k, and ||X^k - X^{k-1}|| / ||X^{k-1}|| within 1e-3
  relative (a difference of FP32 iterates);
* early exit at the first check at or below rel_tol (Sec. 2.1: run until
  the iterates settle);
* a NaN in the dirty cube returns MUFFIN_ENUMERIC and leaves the plan usable;
* the n_c rule after Eq. globalgrad: the same n_c as the oracle, theta
  within 1e-3, the cube within 1e-5.
"""
import numpy as np
import pytest

from oracle import muffin as om, sure as osure, weights as ow
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def weighted_problem(c, seed=5):
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.6, 1.4, (c.n, c.n))
    beta = rng.uniform(0.7, 1.3, c.L)
    prob = om.make_problem(c.dirty, c.psf, alpha_w=alpha, beta_w=beta)
    return prob, alpha.astype(np.float32), beta.astype(np.float32)


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
def test_objective_matches_oracle(precision):
    """Eqs. probopt + RegAll with weights; with precision fp32 the spectral
    term's DCT is the FP32 fast transform."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 8, 10, 2, 800, seed=71)
    prob, alpha, beta = weighted_problem(c)
    x = np.abs(np.random.default_rng(3).standard_normal(c.dirty.shape)).astype(np.float32) * 0.1
    with pkg.Plan(c.n, c.L, c.psf, alpha=alpha.ravel(), beta=beta, precision=precision) as plan:
        for mu, gamma in ((1e-2, 2e-2), (0.0, 0.0), (0.3, 0.0)):
            f = plan.objective(dev(c.dirty, torch), dev(x, torch), mu, gamma)
            ref = om.objective(x.astype(np.float64), prob, mu, gamma)
            assert f == pytest.approx(ref, rel=1e-6), (mu, gamma)
        x[0, 3, 4] = -1e-3
        assert plan.objective(dev(c.dirty, torch), dev(x, torch), 1e-2, 1e-2) == float("inf")


def oracle_checks(prob, mu, gamma, iters, every):
    mu_l, gamma_n = om.weights(prob, mu, gamma)
    tau = om.step_tau(prob, mu_l, gamma_n)
    st = om.zero_state(prob)
    out = []
    for k in range(1, iters + 1):
        prev = st.x.copy()
        om.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        if k % every == 0:
            d = np.linalg.norm(st.x - prev)
            p = np.linalg.norm(prev)
            out.append((k, d / p if p > 0 else np.inf, om.objective(st.x, prob, mu, gamma)))
    return out


def test_monitor_records_during_solve():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 8, 10, 2, 800, seed=72)
    prob, alpha, beta = weighted_problem(c, seed=6)
    mu, gamma, iters, every = 1e-2, 1e-2, 40, 5
    ref = oracle_checks(prob, mu, gamma, iters, every)
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, alpha=alpha.ravel(), beta=beta) as plan:
        plan.set_monitor(every=every, objective=True)
        info = plan.solve(dev(c.dirty, torch), x, iters, mu, gamma)
        recs = plan.monitor_records()
    assert info.checks == len(recs) == iters // every and info.stopped_early == 0
    assert info.iters_done == iters
    for r, (k, rel, obj) in zip(recs, ref):
        assert r["k"] == k and r["nonfinite"] == 0
        assert r["objective"] == pytest.approx(obj, rel=1e-6), k
        if np.isfinite(rel):
            assert r["rel_change"] == pytest.approx(rel, rel=1e-3), k
        else:
            assert r["rel_change"] == float("inf")
    assert info.objective == recs[-1]["objective"]
    assert rel_l2(host(x), om.solve(prob, mu, gamma, iters)[0].x) <= 1e-5


def test_monitor_early_exit():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 600, seed=73)
    prob = om.make_problem(c.dirty, c.psf)
    mu, gamma, every, cap = 1e-2, 1e-2, 5, 150
    ref = oracle_checks(prob, mu, gamma, cap, every)
    rels = [r[1] for r in ref]
    # a tolerance halfway (in log) between two successive checks, past the first
    i = next(i for i in range(4, len(rels)) if rels[i] < 0.9 * min(rels[:i]))
    tol = float(np.sqrt(rels[i] * min(rels[:i])))
    want = ref[i][0]
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf) as plan:
        plan.set_monitor(every=every, rel_tol=tol)
        info = plan.solve(dev(c.dirty, torch), x, cap, mu, gamma)
    assert info.stopped_early == 1 and info.iters_done == want, (info.iters_done, want)
    assert rel_l2(host(x), om.solve(prob, mu, gamma, want)[0].x) <= 1e-5


def test_nan_in_dirty_cube_is_reported_and_plan_stays_usable():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    from paper_1905_08468_gb300.native import MuffinError
    c = make_cube(32, 4, 8, 1, 600, seed=74)
    bad = c.dirty.copy()
    bad[2, 5, 7] = np.nan
    eps = fdmc_eps(c.noise_var)
    with pkg.Plan(c.n, c.L, c.psf, sure=True) as plan:
        x = dev(np.zeros_like(c.dirty), torch)
        with pytest.raises(MuffinError) as e:
            plan.solve(dev(bad, torch), x, 10, 1e-2, 1e-2)
        assert e.value.status == 5
        with pytest.raises(MuffinError) as e:
            plan.sure_tune(dev(bad, torch), dev(c.delta, torch), c.noise_var, x, (1e-2, 1e-2),
                           10, window=5, eta=(1e-5, 1e-5), eps=eps)
        assert e.value.status == 5
        # no state to continue from after the failure
        with pytest.raises(MuffinError) as e:
            plan.solve(None, x, 1, 1e-2, 1e-2, warm=True)
        assert e.value.status == 6
        x1 = dev(np.zeros_like(c.dirty), torch)
        plan.solve(dev(c.dirty, torch), x1, 10, 1e-2, 1e-2)
        x2 = dev(np.zeros_like(c.dirty), torch)
        th2, _, _ = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x2,
                                   (1e-2, 1e-2), 10, window=5, eta=(1e-5, 1e-5), eps=eps)
    with pkg.Plan(c.n, c.L, c.psf, sure=True) as fresh:
        y1 = dev(np.zeros_like(c.dirty), torch)
        fresh.solve(dev(c.dirty, torch), y1, 10, 1e-2, 1e-2)
        y2 = dev(np.zeros_like(c.dirty), torch)
        th3, _, _ = fresh.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, y2,
                                    (1e-2, 1e-2), 10, window=5, eta=(1e-5, 1e-5), eps=eps)
    assert torch.equal(x1, y1) and torch.equal(x2, y2) and th2 == th3


def test_overflow_inside_the_iteration_is_caught_by_the_scan():
    """Finite inputs whose H^T y overflows FP32: without the positivity
    projection (which would map the non-finite m to 0) X turns non-finite and
    the end-of-call scan returns MUFFIN_ENUMERIC."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    from paper_1905_08468_gb300.native import MuffinError
    n, L = 16, 2
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1.0
    psf[:, 0, 1] = 1.0              # |h_hat(0)| = 2: H^T y = 2 y = 6e38 > FP32 max
    dirty = np.full((L, n, n), 3e38, np.float32)
    x = dev(np.zeros((L, n, n)), torch)
    with pkg.Plan(n, L, psf, positivity=False, n_wavelets=2, levels=1) as plan:
        with pytest.raises(MuffinError) as e:
            plan.solve(dev(dirty, torch), x, 3, 1e-2, 1e-2)
        assert e.value.status == 5 and "after 3 iterations" in str(e.value)


def test_monitor_in_sure_tune_checks_at_window_ends():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 600, seed=75)
    eps = fdmc_eps(c.noise_var)
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, sure=True) as plan:
        plan.set_monitor(every=7, objective=True)
        th, trace, info = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var,
                                         x, (1e-2, 1e-2), 30, window=5, eta=(1e-5, 1e-5),
                                         eps=eps)
        recs = plan.monitor_records()
    # first window end at or after 7, 14, 21, 28: k = 10, 15, 25, 30
    assert [r["k"] for r in recs] == [10, 15, 25, 30]
    prob = om.make_problem(c.dirty, c.psf)
    ref = osure.ada_pt(prob, c.delta, eps, c.noise_var, (1e-2, 1e-2), 30, Delta=5,
                       eta=(1e-5, 1e-5))
    assert recs[-1]["objective"] == pytest.approx(
        om.objective(ref.x, prob, ref.theta[0], ref.theta[1]), rel=1e-5)


def test_global_descent_auto_n_c():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 600, seed=76)
    prob = om.make_problem(c.dirty, c.psf)
    eps = fdmc_eps(c.noise_var)
    th0, check, cap, eta = (0.03, 0.02), 4, 48, (1e-5, 1e-4)
    long = osure.ada_pt(prob, c.delta, eps, c.noise_var, th0, cap, Delta=check,
                        eta=(0.0, 0.0), reset=False)
    norms = [np.linalg.norm(t["sugar"]) for t in long.trace]
    rel = [abs(norms[i] - norms[i - 1]) / norms[i] for i in range(1, len(norms))]
    # a tolerance between two well separated successive values
    i = next(i for i in range(2, len(rel)) if rel[i] < 0.8 * min(rel[:i]))
    tol = float(np.sqrt(rel[i] * min(rel[:i])))
    xr, thr, recr = ow.global_descent_auto(prob, c.delta, eps, c.noise_var, th0, 2, check=check,
                                           tol=tol, n_cap=cap, eta=eta)
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, sure=True) as plan:
        th, trace, _ = plan.sure_global_auto(dev(c.dirty, torch), dev(c.delta, torch),
                                             c.noise_var, x, th0, cap, 2, check=check, tol=tol,
                                             eta=eta, eps=eps)
        assert [t["k"] for t in trace] == [r["k"] for r in recr]
        assert rel_l2(host(x), xr) <= 1e-5
        assert np.allclose(th, thr, rtol=1e-3, atol=0)
        # tol = 0: the fixed-n_c descent, up to tau's rounding
        x0 = dev(np.zeros_like(c.dirty), torch)
        tha, tra, _ = plan.sure_global_auto(dev(c.dirty, torch), dev(c.delta, torch),
                                            c.noise_var, x0, th0, cap, 2, check=check, tol=0.0,
                                            eta=eta, eps=eps)
        x1 = dev(np.zeros_like(c.dirty), torch)
        thf, trf, _ = plan.sure_global(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var,
                                       x1, th0, cap, 2, eta=eta, eps=eps)
    assert [t["k"] for t in tra] == [cap, cap]
    assert np.allclose(tha, thf, rtol=1e-9, atol=0)
    assert rel_l2(host(x0), host(x1)) <= 1e-6
