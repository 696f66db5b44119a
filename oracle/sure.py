"""SURE-based tuning of (mu, gamma): Algorithms 3-5, Eqs. PSURE0 and SUGAR.

Readings where the paper is silent or inconsistent (applied identically by
the CUDA path):

* noise: Eq. (model) assumes one variance; the workloads fix the SNR per band,
  so every band l uses its own sigma_l^2 in PSURE/SUGAR (each per-band term
  stays unbiased);
* windows: Algorithm 5 tests k = (q+1) Delta before incrementing k, which
  would make the first window Delta+1 iterations long; the notation
  grad R_{q Delta : k} reads as windows of exactly Delta iterations, so theta
  is updated after every Delta completed iterations;
* derivatives "m steps ahead of k" (Sec. 3.2) restart from zero at every
  window start: x', u', v', t' = 0 (the carried state X, U, V, T is treated as
  independent of theta); ``reset=False`` carries them over instead;
* step: separate step sizes eta_mu, eta_gamma (the two parameters differ by
  orders of magnitude, Sec. 4.2), theta clamped below at theta_min;
* tau is recomputed from the step condition after every theta update and held
  fixed within a window (Algorithms 3/4 differentiate with tau constant).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import convolution, spectral
from .muffin import Problem, State, iteration, step_tau, weights, zero_state


def U_mask(m):
    """Weak derivative of (.)_+ : 1 where m > 0 (Sec. 3.2)."""
    return (m > 0.0).astype(np.float64)


def Pi_mask(p):
    """Weak derivative of sat: 1 where -1 <= p <= 1 (Sec. 3.2)."""
    return (np.abs(p) <= 1.0).astype(np.float64)


def zero_dstate(prob: Problem) -> State:
    return zero_state(prob)


def dmu_iteration(d: State, rec: dict, prob: Problem, mu, gamma, tau):
    """Algorithm 3: one update of x' = dx/dmu alongside the primal update
    whose intermediates are ``rec``."""
    b = prob.beta_w[:, None, None]
    a = prob.alpha_w[None]
    x_d = d.x                                                # eq. updatenode_mu
    grad_d = convolution.HT(convolution.H(x_d, prob.hhat), prob.hhat)
    s_d = mu * b * prob.WsT(d.u) + \
        b * prob.WsT(rec["u_old"])    # eq. adjointspat_mu
    m_d = x_d - tau * (grad_d + s_d + d.t)
    xt_d = (U_mask(rec["m"]) if prob.positivity else 1.0) * m_d   # eq. U_mu
    w = 2.0 * rec["xt"] - rec["x"] + mu * (2.0 * xt_d - x_d)
    p_d = d.u + prob.sigma * b[:, None] * prob.Ws(w)
    u_d = Pi_mask(rec["p"]) * p_d                            # eq. pi_mu
    vt_d = d.v + prob.sigma * gamma * a * \
        spectral.apply_spectra(prob.C, 2.0 * xt_d - x_d)
    v_d = Pi_mask(rec["vt"]) * vt_d
    t_d = gamma * a * spectral.apply_spectra(prob.C.T, v_d)
    d.x, d.u, d.v, d.t = xt_d, u_d, v_d, t_d


def dgamma_iteration(d: State, rec: dict, prob: Problem, mu, gamma, tau):
    """Algorithm 4: one update of x' = dx/dgamma."""
    b = prob.beta_w[:, None, None]
    a = prob.alpha_w[None]
    x_d = d.x                                                # eq. updatenode
    grad_d = convolution.HT(convolution.H(x_d, prob.hhat), prob.hhat)  # grad
    s_d = mu * b * prob.WsT(d.u)      # eq. adjointspat
    m_d = x_d - tau * (grad_d + s_d + d.t)
    xt_d = (U_mask(rec["m"]) if prob.positivity else 1.0) * m_d
    p_d = d.u + prob.sigma * mu * b[:, None] * \
        prob.Ws(2.0 * xt_d - x_d)
    u_d = Pi_mask(rec["p"]) * p_d                            # eq. updateu
    w = 2.0 * rec["xt"] - rec["x"] + gamma * (2.0 * xt_d - x_d)
    vt_d = d.v + prob.sigma * a * spectral.apply_spectra(prob.C, w)
    v_d = Pi_mask(rec["vt"]) * vt_d
    t_d = gamma * a * spectral.apply_spectra(prob.C.T, v_d) + \
        a * spectral.apply_spectra(prob.C.T, rec["v_new"])
    d.x, d.u, d.v, d.t = xt_d, u_d, v_d, t_d


def psure(y, x, xbar, delta, eps, noise_var, hhat) -> float:
    """Eq. (PSURE) summed over bands of Eq. (PSURE0), per-band variance."""
    N = y.shape[-1] * y.shape[-2]
    d = convolution.H(x, hhat)
    db = convolution.H(xbar, hhat)
    r = np.sum((y - d) ** 2, axis=(1, 2)) - N * noise_var + \
        noise_var * (2.0 / eps) * np.sum((db - d) * delta, axis=(1, 2))
    return float(np.sum(r))


def sugar(y, x, dx, dxbar, delta, eps, noise_var, hhat) -> float:
    """Eq. (SUGAR) summed over bands: derivative of PSURE-FDMC."""
    d = convolution.H(x, hhat)
    dd = convolution.H(dx, hhat)
    ddb = convolution.H(dxbar, hhat)
    r = 2.0 * np.sum((d - y) * dd, axis=(1, 2)) + \
        (2.0 * noise_var / eps) * np.sum((ddb - dd) * delta, axis=(1, 2))
    return float(np.sum(r))


def pmse(x_true, x, hhat) -> float:
    """Eqs. (prisk0)/(prisk) for one realisation: sum ||H (x* - x)||^2."""
    r = convolution.H(np.asarray(x_true, np.float64) - x, hhat)
    return float(np.sum(r * r))


@dataclasses.dataclass
class AdaptResult:
    x: np.ndarray
    xbar: np.ndarray
    theta: np.ndarray
    tau: float
    trace: list        # per window: dict(k, theta, sugar, psure, tau)
    states: tuple      # (S, Sbar, Dmu, Dg, Dmubar, Dgbar)


def ada_pt(prob: Problem, delta, eps: float, noise_var, theta0, n_iter: int,
           Delta: int = 10, eta=(1e-3, 1e-3), theta_min: float = 1e-8,
           reset: bool = True, step_rule: int = 0, safety: float = 0.99,
           states=None) -> AdaptResult:
    """Algorithm 5 (ADA-PT'ed MUFFIN), theta = (mu, gamma) (Eq. adaptgrad)."""
    y = prob.y
    delta = np.asarray(delta, np.float64)
    noise_var = np.asarray(noise_var, np.float64)
    ybar = y + eps * delta
    theta = np.array(theta0, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    if states is None:
        S, Sb = zero_state(prob), zero_state(prob)
        D = [zero_dstate(prob) for _ in range(4)]
    else:
        S, Sb, *D = states
    mu_l, gamma_n = weights(prob, theta[0], theta[1])
    tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
    trace = []
    for k in range(n_iter):
        mu, gamma = theta
        mu_l, gamma_n = weights(prob, mu, gamma)
        rec = iteration(S, prob, y, mu_l, gamma_n, tau)          # primal on y
        recb = iteration(Sb, prob, ybar, mu_l, gamma_n, tau)     # primal on y + eps delta
        dmu_iteration(D[0], rec, prob, mu, gamma, tau)           # derivatives, both primals
        dgamma_iteration(D[1], rec, prob, mu, gamma, tau)
        dmu_iteration(D[2], recb, prob, mu, gamma, tau)
        dgamma_iteration(D[3], recb, prob, mu, gamma, tau)
        if (k + 1) % Delta == 0:
            g = np.array([
                sugar(y, S.x, D[0].x, D[2].x, delta, eps, noise_var, prob.hhat),
                sugar(y, S.x, D[1].x, D[3].x, delta, eps, noise_var, prob.hhat)])
            r = psure(y, S.x, Sb.x, delta, eps, noise_var, prob.hhat)
            trace.append(dict(k=k + 1, theta=theta.copy(), sugar=g, psure=r,
                              tau=tau))
            theta = np.maximum(theta - eta * g, theta_min)       # eq. adaptgrad
            mu_l, gamma_n = weights(prob, theta[0], theta[1])
            tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
            if reset:
                D = [zero_dstate(prob) for _ in range(4)]
    return AdaptResult(x=S.x, xbar=Sb.x, theta=theta, tau=tau, trace=trace,
                       states=(S, Sb, *D))
