"""Pins of the oracle's IUWT (starlet) dictionary and of MUFFIN / ADA-PT run
with it (Sec. 2.1 names the IUWT as an alternative W_s).

* the planes sum back to the image (w_{j+1} = c_j - c_{j+1} telescopes);
* W and W^T are adjoint; a dense matrix built from a separate loop
  implementation of the definition matches W;
* ||W||^2 from the DFT symbol equals the largest eigenvalue of the dense
  W^T W and a power iteration;
* a constant image has zero detail planes; J = 0 is the identity;
* the MUFFIN fixed point with the IUWT minimises the objective, the
  fixed-point residual in Condat's metric is non-increasing, and the
  derivative chains of Algorithms 3/4 equal central finite differences.
"""
import numpy as np
import pytest

from oracle import iuwt, muffin, spectral, sure
from synth import make_cube


def dense_W(n, J):
    """W as a dense ((J+1) n^2) x n^2 matrix from explicit index loops."""
    h = [1 / 16, 4 / 16, 6 / 16, 4 / 16, 1 / 16]
    N = n * n

    def S(j):
        d = 1 << j
        M = np.zeros((N, N))
        for y in range(n):
            for x in range(n):
                for a in range(5):
                    for b in range(5):
                        yy = (y + (a - 2) * d) % n
                        xx = (x + (b - 2) * d) % n
                        M[y * n + x, yy * n + xx] += h[a] * h[b]
        return M

    A = [np.eye(N)]
    for j in range(J):
        A.append(S(j) @ A[-1])
    rows = [A[j] - A[j + 1] for j in range(J)] + [A[J]]
    return np.vstack(rows)


@pytest.mark.parametrize("n,J", [(8, 1), (8, 2), (16, 3), (32, 3)])
def test_planes_sum_to_image_and_adjoint(n, J):
    rng = np.random.default_rng(n + J)
    x = rng.normal(size=(3, n, n))
    w = iuwt.analysis(x, J)
    assert w.shape == (3, J + 1, n, n)
    np.testing.assert_allclose(w.sum(axis=-3), x, atol=1e-12)
    u = rng.normal(size=w.shape)
    lhs = np.sum(w * u)
    rhs = np.sum(x * iuwt.adjoint(u, J))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("n,J", [(8, 1), (8, 2), (4, 2)])
def test_dense_bruteforce_and_exact_norm(n, J):
    D = dense_W(n, J)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(n, n))
    np.testing.assert_allclose(iuwt.analysis(x, J).reshape(-1), D @ x.reshape(-1), atol=1e-13)
    u = rng.normal(size=(J + 1, n, n))
    np.testing.assert_allclose(iuwt.adjoint(u, J).reshape(-1), D.T @ u.reshape(-1), atol=1e-13)
    ev = np.linalg.eigvalsh(D.T @ D)
    assert iuwt.norm2(n, J) == pytest.approx(ev.max(), rel=1e-12)
    # the B3 symbol (1 + cos w)^2 / 4 lies in [0, 1]: ||W||^2 = 1 (at DC),
    # while the frame is not tight (smallest eigenvalue below 1)
    assert ev.max() == pytest.approx(1.0, abs=1e-12) and ev.min() < 0.9


def test_norm_by_power_iteration_and_special_cases():
    n, J = 32, 3
    rng = np.random.default_rng(2)
    v = rng.normal(size=(n, n))
    for _ in range(400):
        v = iuwt.adjoint(iuwt.analysis(v, J), J)
        lam = np.linalg.norm(v)
        v /= lam
    # eigenvalues crowd towards the top one near DC: the power iteration
    # approaches it from below
    assert iuwt.norm2(n, J) == 1.0
    assert 0.999 <= lam <= 1.0 + 1e-12
    c = np.full((n, n), 2.5)
    w = iuwt.analysis(c, J)
    assert np.max(np.abs(w[:J])) <= 1e-14 and np.allclose(w[J], 2.5)
    x = rng.normal(size=(n, n))
    np.testing.assert_array_equal(iuwt.analysis(x, 0)[0], x)
    assert iuwt.norm2(n, 0) == 1.0


def _prob(n=8, L=3, J=2, seed=7):
    c = make_cube(n, L, 6, 1, 300, seed=seed)
    return c, muffin.make_problem(c.dirty, c.psf, J=J, dictionary="iuwt")


def test_muffin_iuwt_fixed_point_minimises_objective():
    rng = np.random.default_rng(3)
    psf = np.zeros((2, 8, 8))
    psf[:, 0, 0] = 1.0
    psf[:, 0, 1] = psf[:, 1, 0] = psf[:, 0, -1] = psf[:, -1, 0] = 0.1
    y = np.abs(rng.standard_normal((2, 8, 8)))
    prob = muffin.make_problem(y, psf, J=2, dictionary="iuwt")
    assert prob.planes == 3 and prob.ws_norm2 == pytest.approx(iuwt.norm2(8, 2))
    st, _ = muffin.solve(prob, 0.02, 0.02, 4000, step_rule=1)
    f = muffin.objective(st.x, prob, 0.02, 0.02)
    for _ in range(20):
        xp = np.maximum(st.x + 1e-3 * rng.standard_normal(st.x.shape), 0)
        assert muffin.objective(xp, prob, 0.02, 0.02) >= f - 1e-10


def test_muffin_iuwt_condat_residual_nonincreasing():
    c, prob = _prob(8, 4, 2)
    mu_l, gamma_n = muffin.weights(prob, 0.2, 0.3)
    tau = muffin.step_tau(prob, mu_l, gamma_n, rule=1)

    def pnorm2(dx, du, dv):
        lu = mu_l[:, None, None, None] * prob.Ws(dx)
        lv = gamma_n[None] * spectral.apply_spectra(prob.C, dx)
        return (np.sum(dx * dx) / tau - 2 * (np.sum(lu * du) + np.sum(lv * dv))
                + (np.sum(du * du) + np.sum(dv * dv)) / prob.sigma)

    st = muffin.zero_state(prob)
    old = st.copy()
    muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
    prev = pnorm2(st.x - old.x, st.u - old.u, st.v - old.v)
    for _ in range(60):
        old = st.copy()
        muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        r = pnorm2(st.x - old.x, st.u - old.u, st.v - old.v)
        assert -1e-12 <= r <= prev * (1 + 1e-9) + 1e-15
        prev = r


@pytest.mark.parametrize("which", ["mu", "gamma"])
def test_iuwt_derivative_chains_equal_finite_differences(which):
    c, prob = _prob()
    MU, GAMMA = 0.08, 0.05
    tau = muffin.step_tau(prob, *muffin.weights(prob, MU, GAMMA))

    def primal(mu, gamma, k=25):
        st = muffin.zero_state(prob)
        mu_l, gamma_n = muffin.weights(prob, mu, gamma)
        for _ in range(k):
            muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        return st

    st = muffin.zero_state(prob)
    d = sure.zero_dstate(prob)
    mu_l, gamma_n = muffin.weights(prob, MU, GAMMA)
    for _ in range(25):
        rec = muffin.iteration(st, prob, prob.y, mu_l, gamma_n, tau)
        (sure.dmu_iteration if which == "mu" else sure.dgamma_iteration)(d, rec, prob, MU, GAMMA, tau)
    th = MU if which == "mu" else GAMMA
    h = 1e-7 * th
    sp = primal(MU + h, GAMMA) if which == "mu" else primal(MU, GAMMA + h)
    sm = primal(MU - h, GAMMA) if which == "mu" else primal(MU, GAMMA - h)
    for name in ("x", "u", "v", "t"):
        fd = (getattr(sp, name) - getattr(sm, name)) / (2 * h)
        an = getattr(d, name)
        assert np.max(np.abs(fd - an)) <= 2e-5 * max(np.max(np.abs(fd)), 1e-30), name
    assert np.max(np.abs(d.x)) > 0
