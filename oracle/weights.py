"""Regularisation weights from an initial cube and the global SUGAR descent
(FP64, test infrastructure).

* Eq. (2regpar) and the weights defined right after it: mu_l = mu beta_l and
  gamma_n = gamma alpha_n with
      alpha_n = 1 / (||W_lambda (x^n)_0||_2 + eps),
      beta_l  = 1 / (||W_s (x_l)_0||_2 + eps),
  where (x^n)_0 is pixel n's spectrum and (x_l)_0 band l's image of the cube
  used to initialise the algorithm (Sec. 2.1).  The paper leaves eps open;
  it is an input here, one value for the alphas and one for the betas.
* Eq. (globalgrad), Sec. 3.3: theta^(i+1) = theta^(i) - eta grad R_{0:n_c},
  where n_c is either given or, as the paragraph after Eq. (globalgrad)
  suggests, found by watching k -> ||grad R_{0:k}(theta^(i))||: reading
  taken, n_c is the first multiple k >= 2 check of the check interval at
  which that norm changed by at most tol times itself since k - check (or
  the cap, if reached first);
  where grad R_{0:n_c} is SUGAR after running MUFFIN and its derivative
  iterates for n_c iterations from the same initialisation with theta^(i)
  held fixed.  One such outer step is ADA-PT (Algorithm 5) with a single
  window of length n_c started cold, so it is computed as that; theta is
  kept above theta_min as in ADA-PT.
"""
from __future__ import annotations

import numpy as np

from . import iuwt, spectral, wavelets
from .daubechies import filter_bank
from .muffin import Problem
from .sure import ada_pt


def weights_from_x0(x0, n_wavelets: int = 8, J: int = 3, eps_alpha: float = 1e-3,
                    eps_beta: float = 1e-3, dictionary: str = "daubechies"):
    """alpha [n, n] and beta [L] of the initial cube x0 [L, n, n] (Eq.
    2regpar), with the transforms applied explicitly: the DCT of every
    pixel spectrum and W_s (the union of Daubechies bases, or the IUWT) of
    every band image."""
    x0 = np.asarray(x0, np.float64)
    L, n, _ = x0.shape
    C = spectral.dct_matrix(L)
    spectra = x0.reshape(L, n * n).T                 # row n = pixel spectrum x^n
    coef_lambda = spectra @ C.T                       # W_lambda x^n for every n
    alpha = 1.0 / (np.sqrt(np.sum(coef_lambda ** 2, axis=1)) + eps_alpha)
    bank = filter_bank(n_wavelets)
    beta = np.empty(L)
    for l in range(L):
        if dictionary == "iuwt":
            u = iuwt.analysis(x0[l], J)                # [J + 1, n, n]
        else:
            u = wavelets.Ws(x0[l], bank, J)           # [K, n, n]
        beta[l] = 1.0 / (np.sqrt(np.sum(u ** 2)) + eps_beta)
    return alpha.reshape(n, n), beta


def global_descent(prob: Problem, delta, eps: float, noise_var, theta0, outer: int,
                   n_c: int, eta=(1e-3, 1e-3), theta_min: float = 1e-8,
                   step_rule: int = 0, safety: float = 0.99):
    """Eq. (globalgrad): `outer` gradient steps, each after n_c iterations of
    MUFFIN and its derivative chains from the zero initialisation with theta
    fixed.  Returns (x of the last run, theta, records) with one record per
    outer step (the theta used, SUGAR, PSURE, tau)."""
    theta = np.array(theta0, np.float64)
    records, x = [], None
    for _ in range(outer):
        r = ada_pt(prob, delta, eps, noise_var, theta, n_c, Delta=n_c, eta=eta,
                   theta_min=theta_min, reset=True, step_rule=step_rule,
                   safety=safety)
        records.append(r.trace[-1])
        theta, x = r.theta, r.x
    return x, theta, records


def global_descent_auto(prob: Problem, delta, eps: float, noise_var, theta0, outer: int,
                        check: int, tol: float, n_cap: int, eta=(1e-3, 1e-3),
                        theta_min: float = 1e-8, step_rule: int = 0, safety: float = 0.99):
    """Eq. (globalgrad) with n_c chosen by the rule above.  Each outer step
    runs MUFFIN and the derivative chains from the zero initialisation with
    theta fixed, ``check`` iterations at a time (derivatives carried, so each
    window end gives grad R_{0:k}), stops at n_c and takes the descent step.
    Returns (x of the last run, theta, records), records holding the theta
    used, SUGAR, PSURE, tau and k = n_c of every step."""
    theta = np.array(theta0, np.float64)
    eta = np.asarray(eta, np.float64)
    records, x = [], None
    for _ in range(outer):
        states, prev, k, last = None, None, 0, None
        while True:
            r = ada_pt(prob, delta, eps, noise_var, theta, check, Delta=check, eta=(0.0, 0.0),
                       theta_min=theta_min, reset=False, step_rule=step_rule, safety=safety,
                       states=states)
            states, k, last = r.states, k + check, r.trace[-1]
            nrm = float(np.linalg.norm(last["sugar"]))
            settled = prev is not None and k >= 2 * check and abs(nrm - prev) <= tol * nrm
            prev = nrm
            if settled or k >= n_cap:
                break
        rec = dict(last)
        rec["k"] = k
        records.append(rec)
        theta = np.maximum(theta - eta * rec["sugar"], theta_min)
        x = states[0].x
    return x, theta, records
