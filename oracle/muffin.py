"""MUFFIN primal-dual iteration (Algorithm 2), step sizes and objective (FP64).

Follows Sec. 2.2-2.3: the first Vu-Condat algorithm without relaxation
applied to Eqs. (probopt)/(RegAll), written in the per-band / per-pixel form
of Algorithm 2, which is Algorithm 1 regrouped.

Readings where the paper is silent (applied identically by the CUDA path):

* start from X = 0, U = 0, V = 0, T = 0 unless an initial cube is given;
* step condition of Sec. 2.2 in the paper's sum form, with ||W_s||^2 = K
  (number of bases) and ||W_lambda||^2 = 1:
      tau = safety / (beta/2 + sigma (K sum_l mu_l^2 + sum_n gamma_n^2)),
  safety = 0.99; the max form K max mu_l^2 + max gamma_n^2 (= ||L||^2
  exactly, because L^T L is diagonal) is step rule 1;
* mu_l = mu beta_l, gamma_n = gamma alpha_n (Eq. 2regpar), weights default 1;
* positivity can be switched off only to test closed forms.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import convolution, iuwt, spectral, wavelets


@dataclasses.dataclass
class Problem:
    y: np.ndarray            # dirty cube [L, n, n]
    hhat: np.ndarray         # PSF spectra [L, n, n] complex
    bank: list               # [(h, g)] for db1..dbK
    J: int                   # wavelet levels
    C: np.ndarray            # DCT-II matrix [L, L]
    sigma: float = 10.0      # dual step (Sec. 4.2.1)
    alpha_w: np.ndarray = None   # pixel weights alpha_n [n, n]
    beta_w: np.ndarray = None    # band weights beta_l [L]
    positivity: bool = True
    dictionary: str = "daubechies"   # or "iuwt" (Sec. 2.1)

    @property
    def L(self):
        return self.y.shape[0]

    @property
    def n(self):
        return self.y.shape[-1]

    @property
    def K(self):
        """Number of Daubechies bases of the union."""
        return len(self.bank)

    @property
    def planes(self):
        """Coefficient planes per image: K bases, or J + 1 IUWT planes."""
        return self.J + 1 if self.dictionary == "iuwt" else self.K

    @property
    def ws_norm2(self):
        """||W_s||^2: K for the unscaled union of K orthonormal bases, the
        exact starlet norm for the IUWT."""
        if self.dictionary == "iuwt":
            return iuwt.norm2(self.n, self.J)
        return float(self.K)

    def Ws(self, x):
        """W_s x: images [..., n, n] -> [..., planes, n, n]."""
        if self.dictionary == "iuwt":
            return iuwt.analysis(x, self.J)
        return wavelets.Ws(x, self.bank, self.J)

    def WsT(self, u):
        """W_s^T u: [..., planes, n, n] -> images."""
        if self.dictionary == "iuwt":
            return iuwt.adjoint(u, self.J)
        return wavelets.WsT(u, self.bank, self.J)


def make_problem(dirty, psf, n_wavelets=8, J=3, sigma=10.0, alpha_w=None,
                 beta_w=None, positivity=True, dictionary="daubechies") -> Problem:
    from .daubechies import filter_bank
    y = np.asarray(dirty, dtype=np.float64)
    L, n, _ = y.shape
    return Problem(
        y=y, hhat=convolution.psf_spectrum(psf), bank=filter_bank(n_wavelets),
        J=J, C=spectral.dct_matrix(L), sigma=sigma,
        alpha_w=np.ones((n, n)) if alpha_w is None else np.asarray(alpha_w, np.float64),
        beta_w=np.ones(L) if beta_w is None else np.asarray(beta_w, np.float64),
        positivity=positivity, dictionary=dictionary)


def weights(prob: Problem, mu: float, gamma: float):
    """mu_l = mu beta_l (per band) and gamma_n = gamma alpha_n (per pixel)."""
    return mu * prob.beta_w, gamma * prob.alpha_w


def step_tau(prob: Problem, mu_l, gamma_n, rule: int = 0,
             safety: float = 0.99) -> float:
    """tau from the convergence condition of Sec. 2.2 given sigma."""
    beta = convolution.lipschitz(prob.hhat)
    if rule == 0:
        Lnorm2 = prob.ws_norm2 * np.sum(mu_l ** 2) + np.sum(gamma_n ** 2)
    else:
        Lnorm2 = prob.ws_norm2 * np.max(mu_l ** 2) + np.max(gamma_n ** 2)
    return safety / (beta / 2.0 + prob.sigma * Lnorm2)


def sat(u):
    """Eq. (sat): clip to [-1, 1]."""
    return np.clip(u, -1.0, 1.0)


def pos(u):
    """Eq. (projpos): u if u > 0 else 0."""
    return np.where(u > 0.0, u, 0.0)


@dataclasses.dataclass
class State:
    x: np.ndarray   # current primal X [L, n, n]
    u: np.ndarray   # spatial dual U [L, K, n, n]
    v: np.ndarray   # spectral dual V [L, n, n] (index 0 = DCT coefficient)
    t: np.ndarray   # spectral back-projection T [L, n, n]

    def copy(self):
        return State(self.x.copy(), self.u.copy(), self.v.copy(), self.t.copy())


def zero_state(prob: Problem, x0=None) -> State:
    L, n, K = prob.L, prob.n, prob.planes
    x = np.zeros((L, n, n)) if x0 is None else np.array(x0, dtype=np.float64)
    return State(x=x, u=np.zeros((L, K, n, n)), v=np.zeros((L, n, n)),
                 t=np.zeros((L, n, n)))


def iteration(st: State, prob: Problem, y, mu_l, gamma_n, tau, grad_fn=None) -> dict:
    """One Algorithm-2 update in place; returns the intermediates that the
    derivative iterates of Algorithms 3/4 need (m, p, v-tilde, pre-update u,
    updated v, x and x-tilde).  grad_fn(x), when given, replaces the
    gradient of the image-domain data term (another direct operator, Sec. 1)."""
    x = st.x                                               # eq. updatenode2
    if grad_fn is None:
        grad = convolution.HT(convolution.H(x, prob.hhat) - y, prob.hhat)  # grad2
    else:
        grad = grad_fn(x)
    s = mu_l[:, None, None] * prob.WsT(st.u)               # eq. adjointspat2
    m = x - tau * (grad + s + st.t)                         # eq. stpm
    xt = pos(m) if prob.positivity else m                   # eq. stpx
    z = 2.0 * xt - x
    p = st.u + prob.sigma * mu_l[:, None, None, None] * prob.Ws(z)  # eq. stpp
    u_new = sat(p)                                          # eq. stpu
    # master step, every pixel spectrum n
    vt = st.v + prob.sigma * gamma_n[None] * spectral.apply_spectra(prob.C, z)  # vt
    v_new = sat(vt)                                         # eq. v
    t_new = gamma_n[None] * spectral.apply_spectra(prob.C.T, v_new)  # eq. upt
    rec = dict(x=x, xt=xt, m=m, p=p, vt=vt, u_old=st.u, v_new=v_new, grad=grad)
    st.x, st.u, st.v, st.t = xt, u_new, v_new, t_new
    return rec


def solve(prob: Problem, mu: float, gamma: float, n_iter: int, x0=None,
          tau=None, step_rule: int = 0, safety: float = 0.99, state=None, grad_fn=None):
    """Run n_iter Algorithm-2 iterations; returns (state, tau)."""
    mu_l, gamma_n = weights(prob, mu, gamma)
    if tau is None:
        tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
    st = zero_state(prob, x0) if state is None else state
    for _ in range(n_iter):
        iteration(st, prob, prob.y, mu_l, gamma_n, tau, grad_fn)
    return st, tau


def objective(X, prob: Problem, mu: float, gamma: float) -> float:
    """Eq. (probopt) with h of Eq. (RegAll); +inf outside the orthant."""
    mu_l, gamma_n = weights(prob, mu, gamma)
    if prob.positivity and np.any(X < 0):
        return float("inf")
    r = prob.y - convolution.H(X, prob.hhat)
    f = 0.5 * np.sum(r * r)
    f += np.sum(mu_l * np.sum(np.abs(prob.Ws(X)),
                              axis=(1, 2, 3)))
    f += np.sum(gamma_n * np.sum(np.abs(spectral.apply_spectra(prob.C, X)),
                                 axis=0))
    return float(f)
