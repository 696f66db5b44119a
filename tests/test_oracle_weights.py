"""Pins of the oracle's weights from an initial cube (Eq. 2regpar) and of the
global SUGAR descent (Eq. globalgrad).  Each bases is orthonormal and the DCT
is orthonormal, so the weights have closed forms by Parseval:
    alpha_n = 1 / (||x^n||_2 + eps),   beta_l = 1 / (sqrt(K) ||x_l||_2 + eps),
which the oracle does not use (it applies the transforms)."""
import numpy as np
import pytest

from oracle import muffin as om
from oracle import sure as osu
from oracle import weights as ow
from synth import fdmc_eps, make_cube


@pytest.mark.parametrize("K,J,L,n", [(8, 3, 6, 16), (3, 2, 5, 8), (8, 0, 4, 8), (1, 1, 3, 4)])
def test_weights_match_parseval_closed_forms(K, J, L, n):
    rng = np.random.default_rng(7 + K + J)
    x0 = rng.normal(size=(L, n, n))
    ea, eb = 1e-2, 3e-3
    alpha, beta = ow.weights_from_x0(x0, K, J, ea, eb)
    assert alpha.shape == (n, n) and beta.shape == (L,)
    np.testing.assert_allclose(alpha, 1.0 / (np.sqrt((x0 ** 2).sum(axis=0)) + ea), rtol=1e-12)
    np.testing.assert_allclose(beta, 1.0 / (np.sqrt(K * (x0 ** 2).sum(axis=(1, 2))) + eb),
                               rtol=1e-12)


def test_weights_orientation_zero_cube_and_scaling():
    L, n = 5, 8
    x0 = np.zeros((L, n, n))
    a0, b0 = ow.weights_from_x0(x0, 8, 2, 0.5, 0.25)
    assert np.all(a0 == 2.0) and np.all(b0 == 4.0)
    # one pixel spectrum only: alpha changes at that pixel alone; beta in the
    # bands where the spectrum is non-zero alone
    spec = np.array([0.0, 3.0, 0.0, 4.0, 0.0])
    x0[:, 2, 5] = spec
    a, b = ow.weights_from_x0(x0, 8, 2, 0.5, 0.25)
    expect_a = np.full((n, n), 2.0)
    expect_a[2, 5] = 1.0 / (5.0 + 0.5)
    np.testing.assert_allclose(a, expect_a, rtol=1e-12)
    expect_b = np.where(spec != 0, 1.0 / (np.sqrt(8.0) * np.abs(spec) + 0.25), 4.0)
    np.testing.assert_allclose(b, expect_b, rtol=1e-12)
    # homogeneity with eps = 0
    rng = np.random.default_rng(3)
    x = rng.random((L, n, n)) + 0.1
    a1, b1 = ow.weights_from_x0(x, 4, 2, 0.0, 0.0)
    a2, b2 = ow.weights_from_x0(2.5 * x, 4, 2, 0.0, 0.0)
    np.testing.assert_allclose(a2, a1 / 2.5, rtol=1e-12)
    np.testing.assert_allclose(b2, b1 / 2.5, rtol=1e-12)


def _small():
    c = make_cube(16, 4, 6, 1, 300, seed=11)
    return c, om.make_problem(c.dirty, c.psf, n_wavelets=4, J=2)


def test_global_descent_with_zero_step_is_a_cold_solve_each_time():
    c, prob = _small()
    eps = fdmc_eps(c.noise_var)
    x, theta, recs = ow.global_descent(prob, c.delta, eps, c.noise_var, (0.03, 0.02),
                                       outer=3, n_c=6, eta=(0.0, 0.0))
    assert np.all(theta == np.array([0.03, 0.02]))
    st, _ = om.solve(prob, 0.03, 0.02, 6)
    np.testing.assert_allclose(x, st.x, rtol=0, atol=1e-12)
    assert len(recs) == 3
    for r in recs[1:]:
        assert r["k"] == 6
        np.testing.assert_allclose(r["sugar"], recs[0]["sugar"], rtol=1e-12)
        assert r["psure"] == pytest.approx(recs[0]["psure"], rel=1e-12)


def test_global_descent_restarts_unlike_adapt():
    c, prob = _small()
    eps = fdmc_eps(c.noise_var)
    eta = (2e-4, 2e-4)
    x, theta, recs = ow.global_descent(prob, c.delta, eps, c.noise_var, (0.03, 0.02),
                                       outer=2, n_c=5, eta=eta)
    # step 1: theta after one window of length n_c
    r1 = osu.ada_pt(prob, c.delta, eps, c.noise_var, (0.03, 0.02), 5, Delta=5, eta=eta)
    np.testing.assert_allclose(recs[0]["theta"], [0.03, 0.02])
    np.testing.assert_allclose(recs[1]["theta"], r1.theta, rtol=1e-12)
    # step 2 starts from zero again with the new theta: its x equals a cold
    # 5-iteration solve at r1.theta, not ADA-PT's continued iterate
    st, _ = om.solve(prob, r1.theta[0], r1.theta[1], 5)
    np.testing.assert_allclose(x, st.x, rtol=0, atol=1e-12)
    r2 = osu.ada_pt(prob, c.delta, eps, c.noise_var, (0.03, 0.02), 10, Delta=5, eta=eta)
    assert np.max(np.abs(r2.x - x)) > 1e-6
    # the update is the descent step of Eq. globalgrad with SUGAR of that run
    expect = np.maximum(r1.theta - np.asarray(eta) * recs[1]["sugar"], 1e-8)
    np.testing.assert_allclose(theta, expect, rtol=1e-12)


def test_iuwt_weights_are_below_parseval():
    # the starlet has ||W|| = 1 but is not tight: ||W x|| <= ||x||, with
    # equality only for constant images
    rng = np.random.default_rng(4)
    x0 = rng.normal(size=(3, 16, 16))
    _, b = ow.weights_from_x0(x0, J=3, eps_alpha=0.0, eps_beta=0.0, dictionary="iuwt")
    norms = np.sqrt((x0 ** 2).sum(axis=(1, 2)))
    assert np.all(1.0 / b < norms)
    const = np.full((2, 16, 16), 3.0)
    _, bc = ow.weights_from_x0(const, J=3, eps_alpha=0.0, eps_beta=0.0, dictionary="iuwt")
    np.testing.assert_allclose(bc, 1.0 / (3.0 * 16), rtol=1e-12)


def test_auto_n_c_with_zero_tolerance_is_the_fixed_descent():
    """tol = 0 never settles: n_c = the cap, as the fixed-n_c descent."""
    c = make_cube(16, 3, 5, 1, 300, seed=61)
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=2, J=2)
    eps = fdmc_eps(c.noise_var)
    args = (prob, c.delta, eps, c.noise_var, (0.03, 0.02), 2)
    x, th, recs = ow.global_descent(*args, n_c=12, eta=(1e-4, 1e-4))
    xa, tha, reca = ow.global_descent_auto(*args, check=4, tol=0.0, n_cap=12, eta=(1e-4, 1e-4))
    assert [r["k"] for r in reca] == [12, 12]
    assert np.allclose(xa, x, rtol=0, atol=1e-13 * np.max(np.abs(x)))
    assert np.allclose(tha, th, rtol=1e-13, atol=0)
    for a, b in zip(reca, recs):
        assert np.allclose(a["sugar"], b["sugar"], rtol=1e-10, atol=0)


def test_auto_n_c_stops_where_the_norm_settles():
    """The chosen n_c is the first k >= 2 check where ||SUGAR_{0:k}|| moved by
    at most tol of itself since k - check, read off one long run of the
    derivative chains with theta fixed (Algorithm 5 with eta = 0 and the
    derivatives carried); the step is Eq. globalgrad with that SUGAR."""
    c = make_cube(16, 3, 5, 1, 300, seed=62)
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=2, J=2)
    eps = fdmc_eps(c.noise_var)
    th0, check, cap, eta = np.array([0.03, 0.02]), 3, 60, np.array([1e-4, 1e-4])
    long = osu.ada_pt(prob, c.delta, eps, c.noise_var, th0, cap, Delta=check,
                        eta=(0.0, 0.0), reset=False)
    norms = [np.linalg.norm(t["sugar"]) for t in long.trace]
    rel = [abs(norms[i] - norms[i - 1]) / norms[i] for i in range(1, len(norms))]
    tol = float(np.sort(rel)[len(rel) // 2])           # fires somewhere inside
    want = next(check * (i + 1) for i in range(1, len(norms)) if rel[i - 1] <= tol)
    assert want < cap
    x, th, recs = ow.global_descent_auto(prob, c.delta, eps, c.noise_var, th0, 1, check=check,
                                         tol=tol, n_cap=cap, eta=eta)
    assert recs[0]["k"] == want
    g = long.trace[want // check - 1]["sugar"]
    assert np.allclose(recs[0]["sugar"], g, rtol=1e-12, atol=0)
    assert np.allclose(th, np.maximum(th0 - eta * g, 1e-8), rtol=1e-14, atol=0)
    ref = osu.ada_pt(prob, c.delta, eps, c.noise_var, th0, want, Delta=check,
                       eta=(0.0, 0.0), reset=False)
    assert np.allclose(x, ref.x, rtol=0, atol=1e-13 * np.max(np.abs(ref.x)))
