"""Pins of the oracle's SURE machinery (Algorithms 3-5, Eqs. PSURE0, SUGAR).

* the derivative iterates of Algorithms 3/4 equal central finite differences
  of the FP64 primal (the iteration is piecewise linear in theta, so the two
  agree to rounding wherever no mask flips);
* SUGAR equals the finite-difference derivative of PSURE-FDMC in theta;
* PSURE-FDMC is unbiased for the PMSE and SUGAR for its gradient (Monte Carlo,
  Eq. PSURE1 and the limit stated after Eq. SUGAR);
* ADA-PT bookkeeping: eta = 0 keeps theta and reproduces plain MUFFIN; a
  hand-unrolled two-window run matches.
"""
import numpy as np
import pytest

from oracle import convolution, muffin, sure
from synth import make_cube


def problem(n=8, L=3, K=2, J=2, seed=7, weighted=True):
    c = make_cube(n, L, 6, 1, 300, seed=seed)
    prob = muffin.make_problem(c.dirty, c.psf, n_wavelets=K, J=J)
    if weighted:
        prob.beta_w = np.linspace(0.7, 1.3, L)
        prob.alpha_w = np.random.default_rng(seed).uniform(0.6, 1.4, (n, n))
    return c, prob


def run_primal(prob, y, mu, gamma, tau, k):
    st = muffin.zero_state(prob)
    mu_l, gamma_n = muffin.weights(prob, mu, gamma)
    for _ in range(k):
        muffin.iteration(st, prob, y, mu_l, gamma_n, tau)
    return st


def run_with_derivs(prob, y, mu, gamma, tau, k):
    st = muffin.zero_state(prob)
    dm, dg = sure.zero_dstate(prob), sure.zero_dstate(prob)
    mu_l, gamma_n = muffin.weights(prob, mu, gamma)
    st.masked = 0
    for _ in range(k):
        rec = muffin.iteration(st, prob, y, mu_l, gamma_n, tau)
        st.masked += int(np.sum(rec["m"] <= 0))
        sure.dmu_iteration(dm, rec, prob, mu, gamma, tau)
        sure.dgamma_iteration(dg, rec, prob, mu, gamma, tau)
    return st, dm, dg


MU, GAMMA = 0.08, 0.05


@pytest.mark.parametrize("which", ["mu", "gamma"])
def test_derivative_iterates_equal_finite_differences(which):
    c, prob = problem()
    tau = muffin.step_tau(prob, *muffin.weights(prob, MU, GAMMA))
    k = 25
    st, dm, dg = run_with_derivs(prob, prob.y, MU, GAMMA, tau, k)
    d = dm if which == "mu" else dg
    th = MU if which == "mu" else GAMMA
    h = 1e-7 * th
    if which == "mu":
        sp = run_primal(prob, prob.y, MU + h, GAMMA, tau, k)
        sm = run_primal(prob, prob.y, MU - h, GAMMA, tau, k)
    else:
        sp = run_primal(prob, prob.y, MU, GAMMA + h, tau, k)
        sm = run_primal(prob, prob.y, MU, GAMMA - h, tau, k)
    for name in ("x", "u", "v", "t"):
        fd = (getattr(sp, name) - getattr(sm, name)) / (2 * h)
        an = getattr(d, name)
        scale = max(np.max(np.abs(fd)), 1e-30)
        assert np.max(np.abs(fd - an)) <= 2e-5 * scale, name
    assert np.max(np.abs(d.x)) > 0
    # the masks were exercised: some clipping and some projected pixels
    assert np.any(np.abs(st.u) == 1.0) and st.masked > 0


def test_sugar_is_derivative_of_psure():
    c, prob = problem(seed=9)
    eps = 0.5 * np.sqrt(np.mean(c.noise_var))
    delta = c.delta.astype(np.float64)
    ybar = prob.y + eps * delta
    tau = muffin.step_tau(prob, *muffin.weights(prob, MU, GAMMA))
    k = 20
    s, dm, dg = run_with_derivs(prob, prob.y, MU, GAMMA, tau, k)
    sb, dmb, dgb = run_with_derivs(prob, ybar, MU, GAMMA, tau, k)
    g_mu = sure.sugar(prob.y, s.x, dm.x, dmb.x, delta, eps, c.noise_var, prob.hhat)
    g_ga = sure.sugar(prob.y, s.x, dg.x, dgb.x, delta, eps, c.noise_var, prob.hhat)

    def R(mu, gamma):
        a = run_primal(prob, prob.y, mu, gamma, tau, k)
        b = run_primal(prob, ybar, mu, gamma, tau, k)
        return sure.psure(prob.y, a.x, b.x, delta, eps, c.noise_var, prob.hhat)

    h = 1e-6 * MU
    fd_mu = (R(MU + h, GAMMA) - R(MU - h, GAMMA)) / (2 * h)
    h = 1e-6 * GAMMA
    fd_ga = (R(MU, GAMMA + h) - R(MU, GAMMA - h)) / (2 * h)
    assert g_mu == pytest.approx(fd_mu, rel=1e-5, abs=1e-9)
    assert g_ga == pytest.approx(fd_ga, rel=1e-5, abs=1e-9)


def _mc_draws(M, with_sugar):
    n, L = 8, 2
    c = make_cube(n, L, 4, 1, 200, seed=21, with_delta=False)
    prob = muffin.make_problem(c.dirty, c.psf, n_wavelets=2, J=1)
    x_true = c.sky.astype(np.float64)
    clean = convolution.H(x_true, prob.hhat)
    tau = muffin.step_tau(prob, *muffin.weights(prob, MU, GAMMA))
    rng = np.random.default_rng(99)
    sig = np.sqrt(c.noise_var)[:, None, None]
    eps = 0.05 * float(np.sqrt(np.mean(c.noise_var)))
    out = []
    for _ in range(M):
        y = clean + sig * rng.standard_normal(clean.shape)
        delta = rng.standard_normal(clean.shape)
        ybar = y + eps * delta
        if with_sugar:
            s, dm, _ = run_with_derivs(prob, y, MU, GAMMA, tau, 12)
            sb, dmb, _ = run_with_derivs(prob, ybar, MU, GAMMA, tau, 12)
            est = sure.sugar(y, s.x, dm.x, dmb.x, delta, eps, c.noise_var, prob.hhat)
            # pathwise derivative of the true PMSE at the same noise draw
            r = convolution.H(s.x - x_true, prob.hhat)
            truth = 2.0 * np.sum(r * convolution.H(dm.x, prob.hhat))
        else:
            s = run_primal(prob, y, MU, GAMMA, tau, 12)
            sb = run_primal(prob, ybar, MU, GAMMA, tau, 12)
            est = sure.psure(y, s.x, sb.x, delta, eps, c.noise_var, prob.hhat)
            truth = sure.pmse(x_true, s.x, prob.hhat)
        out.append((est, truth))
    return np.array(out)


def test_psure_unbiased_monte_carlo():
    a = _mc_draws(400, with_sugar=False)
    diff = a[:, 0] - a[:, 1]
    se = diff.std(ddof=1) / np.sqrt(len(diff))
    assert abs(diff.mean()) <= 3 * se, (diff.mean(), se, a[:, 1].mean())
    # power: halving the divergence term moves the mean by ~24 SE here
    assert se < 0.05 * a[:, 1].mean()


def test_sugar_unbiased_monte_carlo():
    a = _mc_draws(300, with_sugar=True)
    diff = a[:, 0] - a[:, 1]
    se = diff.std(ddof=1) / np.sqrt(len(diff))
    assert abs(diff.mean()) <= 3 * se, (diff.mean(), se, a[:, 1].mean())


def test_ada_pt_eta_zero_is_plain_muffin():
    c, prob = problem(seed=3)
    eps = 0.1 * np.sqrt(np.mean(c.noise_var))
    res = sure.ada_pt(prob, c.delta, eps, c.noise_var, (MU, GAMMA), 30,
                      Delta=10, eta=(0.0, 0.0))
    st, _ = muffin.solve(prob, MU, GAMMA, 30)
    assert np.array_equal(res.x, st.x)
    assert np.array_equal(res.theta, [MU, GAMMA])
    assert [t["k"] for t in res.trace] == [10, 20, 30]


def test_ada_pt_two_windows_hand_unrolled():
    c, prob = problem(seed=4)
    eps = 0.1 * np.sqrt(np.mean(c.noise_var))
    eta = np.array([2e-4, 1e-4])
    delta = c.delta.astype(np.float64)
    res = sure.ada_pt(prob, delta, eps, c.noise_var, (MU, GAMMA), 4, Delta=2,
                      eta=eta)
    # unrolled: two windows of two iterations, derivatives restarted per window
    y, yb = prob.y, prob.y + eps * delta
    th = np.array([MU, GAMMA])
    S, Sb = muffin.zero_state(prob), muffin.zero_state(prob)
    thetas = []
    for w in range(2):
        mu_l, gamma_n = muffin.weights(prob, *th)
        tau = muffin.step_tau(prob, mu_l, gamma_n)
        D = [sure.zero_dstate(prob) for _ in range(4)]
        for _ in range(2):
            r = muffin.iteration(S, prob, y, mu_l, gamma_n, tau)
            rb = muffin.iteration(Sb, prob, yb, mu_l, gamma_n, tau)
            sure.dmu_iteration(D[0], r, prob, th[0], th[1], tau)
            sure.dgamma_iteration(D[1], r, prob, th[0], th[1], tau)
            sure.dmu_iteration(D[2], rb, prob, th[0], th[1], tau)
            sure.dgamma_iteration(D[3], rb, prob, th[0], th[1], tau)
        g = np.array([sure.sugar(y, S.x, D[0].x, D[2].x, delta, eps, c.noise_var, prob.hhat),
                      sure.sugar(y, S.x, D[1].x, D[3].x, delta, eps, c.noise_var, prob.hhat)])
        thetas.append(th.copy())
        th = np.maximum(th - eta * g, 1e-8)
    assert np.array_equal(res.x, S.x)
    assert np.allclose(res.theta, th, rtol=0, atol=0)
    assert np.allclose([t["theta"] for t in res.trace], thetas, rtol=0, atol=0)
    assert not np.allclose(th, [MU, GAMMA])


def test_theta_clamped_at_minimum():
    c, prob = problem(seed=5)
    eps = 0.1 * np.sqrt(np.mean(c.noise_var))
    res = sure.ada_pt(prob, c.delta, eps, c.noise_var, (MU, GAMMA), 4, Delta=2,
                      eta=(1e9, 1e9), theta_min=1e-8)
    assert np.all(res.theta >= 1e-8)
