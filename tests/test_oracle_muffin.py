"""Pins of the oracle's MUFFIN iteration (Algorithm 2) and step sizes.

* an independent dense-matrix implementation of Algorithm 1 (X as an N x L
  matrix, explicit H_l, W_s, W_lambda matrices) must agree with the fast
  per-band / per-pixel Algorithm 2 to rounding;
* closed-form special cases: one step with H = I; soft thresholding fixed
  points; separability for gamma = 0 (Sec. 2.1);
* convergence theory: monotone objective for projected gradient, Condat's
  metric residual non-increasing, invariants X >= 0, |U|, |V| <= 1.
"""
import numpy as np
import pytest

from oracle import convolution, muffin, spectral, wavelets
from oracle.daubechies import filter_bank
from synth import make_cube
from tests.test_oracle_operators import dense_basis, dense_circulant


def small_problem(n=8, L=4, K=3, J=2, seed=5, **kw):
    c = make_cube(n, L, 6, 1, 400, seed=seed, with_delta=False)
    prob = muffin.make_problem(c.dirty, c.psf, n_wavelets=K, J=J, **kw)
    return c, prob


def identity_psf(n, L):
    p = np.zeros((L, n, n))
    p[:, 0, 0] = 1.0
    return p


# ---------------------------------------------------------------- Alg. 1
def alg1_dense(prob, mu_l, gamma_n, tau, iters):
    """Algorithm 1 with matrices: X is N x L (column l = band image)."""
    L, n = prob.L, prob.n
    N = n * n
    Hs = [dense_circulant(np.fft.ifft2(prob.hhat[l]).real) for l in range(L)]
    Wk = [dense_basis(n, h, g, prob.J) for h, g in prob.bank]
    Ws = np.vstack(Wk)                                      # KN x N
    C = spectral.dct_matrix(L)
    Y = prob.y.reshape(L, N).T                              # N x L
    Dmu = np.diag(mu_l)
    Dg = np.diag(gamma_n.ravel())
    X = np.zeros((N, L)); U = np.zeros((len(Wk) * N, L)); V = np.zeros((N, L))
    for _ in range(iters):
        G = np.column_stack([Hs[l].T @ (Hs[l] @ X[:, l] - Y[:, l]) for l in range(L)])
        Xt = X - tau * (G + Ws.T @ U @ Dmu + Dg @ V @ C)
        Xt = np.where(Xt > 0, Xt, 0.0)
        U = np.clip(U + prob.sigma * Ws @ (2 * Xt - X) @ Dmu, -1, 1)
        V = np.clip(V + prob.sigma * Dg @ (2 * Xt - X) @ C.T, -1, 1)
        X = Xt
    return X.T.reshape(L, n, n)


@pytest.mark.parametrize("n,L,K,J", [(4, 2, 2, 1), (8, 4, 3, 2)])
def test_alg2_equals_dense_alg1(n, L, K, J):
    c, prob = small_problem(n, L, K, J)
    mu_l, gamma_n = muffin.weights(prob, 3e-2, 2e-2)
    prob.beta_w = np.linspace(0.5, 1.5, L)
    prob.alpha_w = np.random.default_rng(1).uniform(0.5, 1.5, (n, n))
    mu_l, gamma_n = muffin.weights(prob, 3e-2, 2e-2)
    tau = muffin.step_tau(prob, mu_l, gamma_n)
    st, _ = muffin.solve(prob, 3e-2, 2e-2, 50, tau=tau)
    Xd = alg1_dense(prob, mu_l, gamma_n, tau, 50)
    assert np.max(np.abs(st.x - Xd)) <= 1e-12 * max(1.0, np.max(np.abs(Xd)))
    assert np.max(np.abs(st.x)) > 0


# ---------------------------------------------------------------- closed forms
def test_one_step_identity_operator():
    rng = np.random.default_rng(0)
    y = rng.standard_normal((2, 8, 8))
    prob = muffin.make_problem(y, identity_psf(8, 2), n_wavelets=2, J=1)
    st, _ = muffin.solve(prob, 0.0, 0.0, 1, tau=1.0)
    assert np.allclose(st.x, np.where(y > 0, y, 0.0), atol=0)


def test_identity_bases_soft_threshold_fixed_point():
    # J = 0, H = I, L = 1: argmin 1/2||y-x||^2 + (K mu + gamma)||x||_1, x >= 0
    rng = np.random.default_rng(1)
    y = rng.standard_normal((1, 4, 4))
    prob = muffin.make_problem(y, identity_psf(4, 1), n_wavelets=8, J=0)
    mu, gamma = 0.05, 0.1
    st, _ = muffin.solve(prob, mu, gamma, 3000, step_rule=1)
    assert np.allclose(st.x, np.maximum(y - 8 * mu - gamma, 0.0), atol=1e-9)


def test_single_basis_soft_threshold_fixed_point():
    # one orthonormal basis, gamma = 0, H = I, positivity off:
    # x = W^T soft(W y, mu)
    rng = np.random.default_rng(2)
    y = rng.standard_normal((1, 8, 8))
    prob = muffin.make_problem(y, identity_psf(8, 1), n_wavelets=2, J=2,
                               positivity=False)
    prob.bank = prob.bank[1:]          # db2 only
    mu = 0.3
    st, _ = muffin.solve(prob, mu, 0.0, 4000, step_rule=1)
    h, g = prob.bank[0]
    w = wavelets.dwt2(y[0], h, g, 2)
    ref = wavelets.idwt2(np.sign(w) * np.maximum(np.abs(w) - mu, 0.0), h, g, 2)
    assert np.allclose(st.x[0], ref, atol=1e-9)


def test_gamma_zero_is_separable():
    c, prob = small_problem(8, 3, 2, 2)
    tau = 0.01
    st, _ = muffin.solve(prob, 0.05, 0.0, 40, tau=tau)
    for l in range(3):
        p1 = muffin.make_problem(c.dirty[l:l + 1], c.psf[l:l + 1], n_wavelets=2, J=2)
        s1, _ = muffin.solve(p1, 0.05, 0.0, 40, tau=tau)
        assert np.allclose(s1.x[0], st.x[l], atol=1e-14)


def test_step_rules():
    c, prob = small_problem()
    mu_l, gamma_n = muffin.weights(prob, 1e-2, 2e-2)
    beta = convolution.lipschitz(prob.hhat)
    t0 = muffin.step_tau(prob, mu_l, gamma_n, rule=0)
    t1 = muffin.step_tau(prob, mu_l, gamma_n, rule=1)
    N = prob.n ** 2
    assert t0 == pytest.approx(0.99 / (beta / 2 + 10 * (3 * prob.L * 1e-4 + N * 4e-4)))
    assert t1 == pytest.approx(0.99 / (beta / 2 + 10 * (3 * 1e-4 + 4e-4)))
    assert t0 < t1


# ---------------------------------------------------------------- convergence
def test_projected_gradient_monotone():
    c, prob = small_problem(16, 4, 2, 2)
    st = muffin.zero_state(prob)
    mu_l, gamma_n = muffin.weights(prob, 0.0, 0.0)
    tau = muffin.step_tau(prob, mu_l, gamma_n)
    prev = muffin.objective(st.x, prob, 0.0, 0.0)
    for _ in range(60):
        muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        f = muffin.objective(st.x, prob, 0.0, 0.0)
        assert f <= prev + 1e-12 * abs(prev)
        prev = f


def test_condat_metric_residual_nonincreasing():
    c, prob = small_problem(8, 4, 3, 2)
    mu, gamma = 0.2, 0.3
    mu_l, gamma_n = muffin.weights(prob, mu, gamma)
    tau = muffin.step_tau(prob, mu_l, gamma_n, rule=1)
    sig = prob.sigma

    def Lop(x):
        return (mu_l[:, None, None, None] * wavelets.Ws(x, prob.bank, prob.J),
                gamma_n[None] * spectral.apply_spectra(prob.C, x))

    def pnorm2(dx, du, dv):
        lu, lv = Lop(dx)
        return (np.sum(dx * dx) / tau - 2 * (np.sum(lu * du) + np.sum(lv * dv))
                + (np.sum(du * du) + np.sum(dv * dv)) / sig)

    st = muffin.zero_state(prob)
    prev_state = st.copy()
    muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
    prev = pnorm2(st.x - prev_state.x, st.u - prev_state.u, st.v - prev_state.v)
    clipped = 0
    for _ in range(80):
        old = st.copy()
        muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        r = pnorm2(st.x - old.x, st.u - old.u, st.v - old.v)
        assert r >= -1e-12
        assert r <= prev * (1 + 1e-9) + 1e-15
        prev = r
        clipped += int(np.sum(np.abs(st.u) == 1.0))
        # invariants of the iterates
        assert np.all(st.x >= 0)
        assert np.all(np.abs(st.u) <= 1) and np.all(np.abs(st.v) <= 1)
    assert clipped > 0          # the dual clipping was exercised


def test_objective_converges_to_long_run_value():
    # well-conditioned blur (spectrum in [0.6, 1.4]) so the iterates settle
    rng = np.random.default_rng(3)
    psf = np.zeros((2, 8, 8))
    psf[:, 0, 0] = 1.0
    psf[:, 0, 1] = psf[:, 1, 0] = psf[:, 0, -1] = psf[:, -1, 0] = 0.1
    y = np.abs(rng.standard_normal((2, 8, 8)))
    prob = muffin.make_problem(y, psf, n_wavelets=2, J=1)
    st, tau = muffin.solve(prob, 0.02, 0.02, 4000, step_rule=1)
    f_long = muffin.objective(st.x, prob, 0.02, 0.02)
    x_long = st.x.copy()
    st, _ = muffin.solve(prob, 0.02, 0.02, 500, step_rule=1, state=st)
    assert np.max(np.abs(st.x - x_long)) < 1e-7
    assert muffin.objective(st.x, prob, 0.02, 0.02) == pytest.approx(f_long, rel=1e-10)
    # the fixed point minimises the objective among nearby feasible points
    for _ in range(20):
        xp = np.maximum(st.x + 1e-3 * rng.standard_normal(st.x.shape), 0)
        assert muffin.objective(xp, prob, 0.02, 0.02) >= f_long - 1e-10
