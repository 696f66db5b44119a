"""Element-by-element parity of every ADA-PT iterate against the FP64 oracle
(Algorithm 5 with the derivative iterates of Algorithms 3 and 4).

After a run that stops inside a window (so the derivative iterates are not
freshly reset), the plan's state blob holds X, U, V, T of all six chains:
the primal on y, the primal on y_bar = y + eps delta, and dX/dmu, dX/dgamma
of both.  Each is compared with the oracle's, element by element, as a
relative L2 error over the whole array:

* primal iterates X, X_bar and their U, V, T: <= 1e-5 (the cube tolerance);
* derivative iterates: <= DERIV_TOL = 1e-4.  They are linear recursions
  driven by the primal's masks U(m), Pi(p), Pi(v~) (Sec. 3.2); FP32 and
  FP64 decide a mask differently at a near-tie, which moves the coefficients
  it gates by their whole value.  Measured on a GB300: within 2e-6 of the
  oracle's at 32^2 x 8 and 64^2 x 64; at 1024^2 x 2 (2 M pixels, 16 M
  coefficients per chain) three derivative arrays show such flips at
  6e-5.  Where an error exceeds the cube tolerance, the differing entries
  must be few (isolated mask flips, not a wrong term).

The runs are chosen so that theta stays well above theta_min in both
components (the clamp would make the theta comparison vacuous), and the
change of theta over the run is compared as well as its final value.
"""
import numpy as np
import pytest

from oracle import muffin as om, parallel as opar, sure as osure
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, rel_l2

pytestmark = pytest.mark.gpu

PRIMAL_TOL = 1e-5
DERIV_TOL = 1e-4
THETA_TOL = 1e-3
THETA_MIN = 1e-8

# oracle order of AdaptResult.states -> (group, chain) of the state blob
STATE_MAP = {0: (0, 0), 1: (1, 0), 2: (0, 1), 3: (0, 2), 4: (1, 1), 5: (1, 2)}
NAMES = {0: "X", 1: "X_bar", 2: "dX/dmu", 3: "dX/dgamma", 4: "dX_bar/dmu", 5: "dX_bar/dgamma"}


def gpu_run(c, theta0, iters, window, eta, eps, reset, **kw):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, sure=True, **kw) as plan:
        th, trace, _ = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var,
                                      x, theta0, iters, window=window, eta=eta, eps=eps,
                                      reset=reset)
        st = plan.state_arrays()
    return np.array(th), trace, st


def compare_states(states, st, label):
    errs = {}
    for i, s in enumerate(states):
        g, ch = STATE_MAP[i]
        for k in ("x", "u", "v", "t"):
            ref = getattr(s, k)
            got = st[k][g, ch]
            e = rel_l2(got, ref) if np.linalg.norm(ref) > 0 else float(np.linalg.norm(got))
            errs[f"{NAMES[i]}.{k}"] = e
    print(label, {k: f"{v:.1e}" for k, v in errs.items()})
    for name, e in errs.items():
        tol = PRIMAL_TOL if name.split(".")[0] in ("X", "X_bar") else DERIV_TOL
        assert e <= tol, (name, e)
        if e > PRIMAL_TOL:
            i = [k for k, v in NAMES.items() if v == name.split(".")[0]][0]
            g, ch = STATE_MAP[i]
            ref = getattr(states[i], name.split(".")[1])
            d = np.abs(st[name.split(".")[1]][g, ch] - ref)
            big = int(np.sum(d > 1e-3 * np.max(np.abs(ref))))
            print(f"  {name}: {big} of {d.size} entries differ by > 1e-3 max|ref|")
            assert big <= max(8, d.size // 100000), (name, big)
    # the derivative iterates are live (not just reset) at the end of the run
    for i in (2, 3, 4, 5):
        assert np.linalg.norm(states[i].x) > 0, NAMES[i]
    return errs


def check_theta(th, ref_theta, theta0):
    th, ref_theta, theta0 = (np.asarray(v, np.float64) for v in (th, ref_theta, theta0))
    for j, name in enumerate(("mu", "gamma")):
        assert ref_theta[j] > 100 * THETA_MIN, f"{name} reached the clamp: the check is vacuous"
        assert abs(ref_theta[j] - theta0[j]) > 1e-3 * theta0[j], f"{name} did not move"
        assert abs(th[j] - ref_theta[j]) <= THETA_TOL * ref_theta[j], (name, th[j], ref_theta[j])
        # the change over the run, not only the end point
        d_gpu, d_ref = th[j] - theta0[j], ref_theta[j] - theta0[j]
        assert abs(d_gpu - d_ref) <= 2e-2 * abs(d_ref), (name, d_gpu, d_ref)


def check_trace(trace, ref_trace):
    assert len(trace) == len(ref_trace)
    for tg, to in zip(trace, ref_trace):
        assert tg["k"] == to["k"]
        assert tg["sugar_mu"] == pytest.approx(to["sugar"][0], rel=1e-3)
        assert tg["sugar_gamma"] == pytest.approx(to["sugar"][1], rel=1e-3)
        assert tg["psure"] == pytest.approx(to["psure"], rel=1e-3)


def run_case(c, theta0, iters, window, eta, reset=True, n_wavelets=8, levels=3, workers=None,
             **plan_kw):
    eps = fdmc_eps(c.noise_var)
    th, trace, st = gpu_run(c, theta0, iters, window, eta, eps, reset,
                            n_wavelets=n_wavelets, levels=levels, **plan_kw)
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=n_wavelets, J=levels)
    if workers:
        _, ref_theta, ref_trace, states = opar.ada_pt(prob, c.delta, eps, c.noise_var, theta0,
                                                      iters, Delta=window, eta=eta, reset=reset,
                                                      workers=workers)
    else:
        ref = osure.ada_pt(prob, c.delta, eps, c.noise_var, theta0, iters, Delta=window,
                           eta=eta, reset=reset)
        ref_theta, ref_trace, states = ref.theta, ref.trace, ref.states
    check_trace(trace, ref_trace)
    check_theta(th, ref_theta, theta0)
    return compare_states(states, st, f"{c.n}^2 x {c.L}")


def test_states_32x32x8_reset():
    """Two windows and three more iterations, derivative restart (default)."""
    c = make_cube(32, 8, 10, 2, 800, seed=12)
    run_case(c, (0.05, 0.05), 13, 5, (2e-5, 2e-4))


def test_states_32x32x8_carry_over():
    """Derivatives carried across windows (reset_each_window = 0)."""
    c = make_cube(32, 8, 10, 2, 800, seed=12)
    run_case(c, (0.05, 0.05), 14, 4, (2e-5, 2e-4), reset=False)


def test_states_64_bands_tcgen05_gamma_chain():
    """64 bands: the spectral step on tcgen05, where the d/dgamma chain's
    products accumulate onto the primal's in tensor memory; its V', T' and
    X' are compared element by element."""
    c = make_cube(64, 64, 20, 3, 2000, seed=21)
    run_case(c, (1e-2, 1e-2), 8, 3, (1e-5, 1e-5))


def test_states_1024_px_size_specialised_analysis():
    """1024^2 x 2: the analysis kernels specialised for a 1024 px side
    (levels 1 and 2) with derivative chains, against the oracle (band-
    parallel form, one worker per band); two iterations carried over one
    window end."""
    c = make_cube(1024, 2, 60, 4, 6000, seed=33)
    run_case(c, (1e-2, 1e-2), 3, 2, (2e-3, 2e-2), reset=False, workers=2)
