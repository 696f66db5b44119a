"""Band-parallel form of the FP64 oracle -- TEST INFRASTRUCTURE.

Sec. 2.3 splits one MUFFIN iteration (Algorithm 2) into per-band work (the
gradient, the spatial synthesis, the primal prox, the spatial analysis and
the dual update of U: eqs. grad2 .. stpu) done by slave nodes, and per-pixel
work over all bands (the spectral dual update and back-projection: eqs. vt,
v, upt) done by the master.  This module runs the oracle in that split on
the host's cores: worker processes own contiguous band blocks and run the
per-band steps in place on shared-memory arrays, the parent runs the
per-pixel steps; the same split carries the derivative iterates of
Algorithms 3 and 4 and ADA-PT (Algorithm 5).

Every step calls the same oracle functions as ``muffin.iteration`` and
``sure.ada_pt`` on band slices, in the same order, so the result equals the
serial oracle up to the rounding of batched FFTs (pinned in
``tests/test_oracle_parallel.py``).  It exists to time the oracle on all
cores and to compute stored expected values of long runs; it is not a
different method.  Workers are started with the ``spawn`` method.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import convolution, spectral
from .muffin import Problem, State, pos, sat, step_tau, weights
from .sure import Pi_mask, U_mask, psure, sugar

# ---------------------------------------------------------------- shared arrays
_W = {}          # worker side: name -> ndarray view
_SHM = []        # worker side: attached segments (kept alive)


def _attach(specs, prob_parts):
    """Pool initializer: map the parent's shared arrays into this worker."""
    for name, (shm_name, shape) in specs.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        _SHM.append(shm)
        _W[name] = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
    _W["prob"] = Problem(**prob_parts)


class _Arena:
    """Parent side: float64 arrays in shared memory, by name."""

    def __init__(self):
        self.specs, self.arr, self._shm = {}, {}, []

    def add(self, name, shape, init=None):
        nbytes = int(np.prod(shape)) * 8
        shm = shared_memory.SharedMemory(create=True, size=max(nbytes, 8))
        self._shm.append(shm)
        a = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
        a[...] = 0.0 if init is None else init
        self.specs[name] = (shm.name, tuple(shape))
        self.arr[name] = a
        return a

    def close(self):
        self.arr.clear()
        for shm in self._shm:
            shm.close()
            shm.unlink()
        self._shm = []


def _prob_parts(prob: Problem) -> dict:
    return dict(y=prob.y, hhat=prob.hhat, bank=prob.bank, J=prob.J, C=prob.C,
                sigma=prob.sigma, alpha_w=prob.alpha_w, beta_w=prob.beta_w,
                positivity=prob.positivity, dictionary=prob.dictionary)


# ---------------------------------------------------------------- slave steps
def _primal_bands(pre, s, yname, mu_l, tau, prob):
    """Eqs. grad2, adjointspat2, stpm, stpx, stpp, stpu for bands s of the
    chain whose arrays are prefixed ``pre``; returns the intermediates the
    derivative steps need (Algorithms 3/4 use the primal's m, p, x, x-tilde
    and pre-update u)."""
    X, U, T = _W[pre + "x"], _W[pre + "u"], _W[pre + "t"]
    x = X[s]
    hh = prob.hhat[s]
    grad = convolution.HT(convolution.H(x, hh) - _W[yname][s], hh)
    sp = mu_l[s][:, None, None] * prob.WsT(U[s])
    m = x - tau * (grad + sp + T[s])
    xt = pos(m) if prob.positivity else m
    z = 2.0 * xt - x
    p = U[s] + prob.sigma * mu_l[s][:, None, None, None] * prob.Ws(z)
    rec = dict(x=x.copy(), xt=xt, m=m, p=p, u_old=U[s].copy())
    U[s] = sat(p)
    _W[pre + "xt"][s] = xt
    _W[pre + "z"][s] = z
    return rec


def _dmu_bands(pre, s, rec, mu, tau, prob):
    """Per-band part of Algorithm 3 (eqs. updatenode_mu .. pi_mu)."""
    b = prob.beta_w[s][:, None, None]
    Xd, Ud, Td = _W[pre + "x"], _W[pre + "u"], _W[pre + "t"]
    x_d = Xd[s]
    hh = prob.hhat[s]
    grad_d = convolution.HT(convolution.H(x_d, hh), hh)
    s_d = mu * b * prob.WsT(Ud[s]) + b * prob.WsT(rec["u_old"])
    m_d = x_d - tau * (grad_d + s_d + Td[s])
    xt_d = (U_mask(rec["m"]) if prob.positivity else 1.0) * m_d
    w = 2.0 * rec["xt"] - rec["x"] + mu * (2.0 * xt_d - x_d)
    p_d = Ud[s] + prob.sigma * b[:, None] * prob.Ws(w)
    Ud[s] = Pi_mask(rec["p"]) * p_d
    _W[pre + "z"][s] = 2.0 * xt_d - x_d
    _W[pre + "xt"][s] = xt_d


def _dgamma_bands(pre, s, rec, mu, tau, prob):
    """Per-band part of Algorithm 4 (eqs. updatenode .. updateu)."""
    b = prob.beta_w[s][:, None, None]
    Xd, Ud, Td = _W[pre + "x"], _W[pre + "u"], _W[pre + "t"]
    x_d = Xd[s]
    hh = prob.hhat[s]
    grad_d = convolution.HT(convolution.H(x_d, hh), hh)
    s_d = mu * b * prob.WsT(Ud[s])
    m_d = x_d - tau * (grad_d + s_d + Td[s])
    xt_d = (U_mask(rec["m"]) if prob.positivity else 1.0) * m_d
    p_d = Ud[s] + prob.sigma * mu * b[:, None] * prob.Ws(2.0 * xt_d - x_d)
    Ud[s] = Pi_mask(rec["p"]) * p_d
    _W[pre + "z"][s] = 2.0 * xt_d - x_d
    _W[pre + "xt"][s] = xt_d


def _slave_plain(task):
    l0, l1, mu_l, tau = task
    _primal_bands("s_", slice(l0, l1), "y", mu_l, tau, _W["prob"])
    return 0


def _slave_adapt(task):
    l0, l1, mu, mu_l, tau = task
    prob, s = _W["prob"], slice(l0, l1)
    rec = _primal_bands("s_", s, "y", mu_l, tau, prob)
    recb = _primal_bands("b_", s, "ybar", mu_l, tau, prob)
    _dmu_bands("dm_", s, rec, mu, tau, prob)
    _dgamma_bands("dg_", s, rec, mu, tau, prob)
    _dmu_bands("dmb_", s, recb, mu, tau, prob)
    _dgamma_bands("dgb_", s, recb, mu, tau, prob)
    return 0


# ---------------------------------------------------------------- master steps
def _master_primal(A, pre, prob, gamma_n):
    """Eqs. vt, v, upt over every pixel spectrum; eq. updatenode2."""
    vt = A[pre + "v"] + prob.sigma * gamma_n[None] * spectral.apply_spectra(prob.C, A[pre + "z"])
    v_new = sat(vt)
    A[pre + "v"][...] = v_new
    A[pre + "t"][...] = gamma_n[None] * spectral.apply_spectra(prob.C.T, v_new)
    A[pre + "x"][...] = A[pre + "xt"]
    return vt, v_new


def _master_dmu(A, pre, vt, prob, gamma):
    a = prob.alpha_w[None]
    vt_d = A[pre + "v"] + prob.sigma * gamma * a * spectral.apply_spectra(prob.C, A[pre + "z"])
    v_d = Pi_mask(vt) * vt_d
    A[pre + "v"][...] = v_d
    A[pre + "t"][...] = gamma * a * spectral.apply_spectra(prob.C.T, v_d)
    A[pre + "x"][...] = A[pre + "xt"]


def _master_dgamma(A, pre, zp, vt, v_new, prob, gamma):
    a = prob.alpha_w[None]
    w = zp + gamma * A[pre + "z"]
    vt_d = A[pre + "v"] + prob.sigma * a * spectral.apply_spectra(prob.C, w)
    v_d = Pi_mask(vt) * vt_d
    A[pre + "v"][...] = v_d
    A[pre + "t"][...] = gamma * a * spectral.apply_spectra(prob.C.T, v_d) + \
        a * spectral.apply_spectra(prob.C.T, v_new)
    A[pre + "x"][...] = A[pre + "xt"]


def _chain(A, pre, prob):
    L, n, K = prob.L, prob.n, prob.planes
    for k in ("x", "xt", "z", "v", "t"):
        A.add(pre + k, (L, n, n))
    A.add(pre + "u", (L, K, n, n))


def _blocks(L, workers):
    edges = np.linspace(0, L, min(workers, L) + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def default_workers() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def _pool(A, prob, workers):
    # one BLAS thread per worker: the workers are the parallelism
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    return ctx.Pool(workers, initializer=_attach, initargs=(A.specs, _prob_parts(prob)))


def solve(prob: Problem, mu: float, gamma: float, n_iter: int, workers: int = None,
          step_rule: int = 0, safety: float = 0.99):
    """``muffin.solve`` from X = U = V = T = 0 in the band-parallel split;
    returns (x, tau)."""
    if prob.dictionary != "daubechies":
        raise ValueError("the band-parallel oracle covers the Daubechies dictionary")
    workers = workers or default_workers()
    mu_l, gamma_n = weights(prob, mu, gamma)
    tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
    A = _Arena()
    try:
        A.add("y", prob.y.shape, prob.y)
        _chain(A, "s_", prob)
        blocks = _blocks(prob.L, workers)
        with _pool(A, prob, len(blocks)) as pool:
            for _ in range(n_iter):
                pool.map(_slave_plain, [(a, b, mu_l, tau) for a, b in blocks])
                _master_primal(A.arr, "s_", prob, gamma_n)
        return A.arr["s_x"].copy(), tau
    finally:
        A.close()


def ada_pt(prob: Problem, delta, eps: float, noise_var, theta0, n_iter: int,
           Delta: int = 10, eta=(1e-3, 1e-3), theta_min: float = 1e-8,
           reset: bool = True, step_rule: int = 0, safety: float = 0.99,
           workers: int = None):
    """``sure.ada_pt`` (Algorithm 5) in the band-parallel split; returns
    (x, theta, trace, states): the trace records of ``sure.ada_pt`` and the
    final iterates as ``sure.AdaptResult.states`` orders them (primal on y,
    primal on y + eps delta, then dX/dmu, dX/dgamma of the first and of the
    second), each a ``muffin.State``."""
    if prob.dictionary != "daubechies":
        raise ValueError("the band-parallel oracle covers the Daubechies dictionary")
    workers = workers or default_workers()
    y = prob.y
    delta = np.asarray(delta, np.float64)
    noise_var = np.asarray(noise_var, np.float64)
    theta = np.array(theta0, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    mu_l, gamma_n = weights(prob, theta[0], theta[1])
    tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
    chains = ("s_", "b_", "dm_", "dg_", "dmb_", "dgb_")
    A = _Arena()
    trace = []
    try:
        A.add("y", y.shape, y)
        A.add("ybar", y.shape, y + eps * delta)
        for pre in chains:
            _chain(A, pre, prob)
        R = A.arr
        blocks = _blocks(prob.L, workers)
        with _pool(A, prob, len(blocks)) as pool:
            for k in range(n_iter):
                mu, gamma = theta
                mu_l, gamma_n = weights(prob, mu, gamma)
                pool.map(_slave_adapt, [(a, b, mu, mu_l, tau) for a, b in blocks])
                zs, zb = R["s_z"].copy(), R["b_z"].copy()
                vt, v_new = _master_primal(R, "s_", prob, gamma_n)
                vtb, v_newb = _master_primal(R, "b_", prob, gamma_n)
                _master_dmu(R, "dm_", vt, prob, gamma)
                _master_dgamma(R, "dg_", zs, vt, v_new, prob, gamma)
                _master_dmu(R, "dmb_", vtb, prob, gamma)
                _master_dgamma(R, "dgb_", zb, vtb, v_newb, prob, gamma)
                if (k + 1) % Delta == 0:
                    g = np.array([
                        sugar(y, R["s_x"], R["dm_x"], R["dmb_x"], delta, eps, noise_var, prob.hhat),
                        sugar(y, R["s_x"], R["dg_x"], R["dgb_x"], delta, eps, noise_var, prob.hhat)])
                    r = psure(y, R["s_x"], R["b_x"], delta, eps, noise_var, prob.hhat)
                    trace.append(dict(k=k + 1, theta=theta.copy(), sugar=g, psure=r, tau=tau))
                    theta = np.maximum(theta - eta * g, theta_min)
                    mu_l, gamma_n = weights(prob, theta[0], theta[1])
                    tau = step_tau(prob, mu_l, gamma_n, step_rule, safety)
                    if reset:
                        for pre in chains[2:]:
                            for key in ("x", "u", "v", "t"):
                                R[pre + key][...] = 0.0
        states = tuple(State(R[p + "x"].copy(), R[p + "u"].copy(), R[p + "v"].copy(),
                             R[p + "t"].copy()) for p in ("s_", "b_", "dm_", "dg_", "dmb_", "dgb_"))
        return R["s_x"].copy(), theta, trace, states
    finally:
        A.close()
