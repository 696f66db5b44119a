"""Pin of the band-parallel oracle: the split of Sec. 2.3 (per-band steps on
workers, per-pixel spectral steps in the parent) reproduces the serial
oracle's Algorithm 2 and Algorithm 5 runs, for uneven band blocks and with
more workers than bands."""
import numpy as np
import pytest

from oracle import muffin, parallel, sure
from synth import fdmc_eps, make_cube


def test_parallel_plain_equals_serial():
    c = make_cube(16, 5, 6, 1, 300, seed=41)
    prob = muffin.make_problem(c.dirty, c.psf, n_wavelets=3, J=2)
    st, tau = muffin.solve(prob, 0.03, 0.02, 12)
    x, tau_p = parallel.solve(prob, 0.03, 0.02, 12, workers=2)
    assert tau_p == tau
    assert np.max(np.abs(x - st.x)) <= 1e-13 * np.max(np.abs(st.x))


@pytest.mark.parametrize("reset,workers", [(True, 3), (False, 7)])
def test_parallel_ada_pt_equals_serial(reset, workers):
    c = make_cube(16, 4, 6, 1, 300, seed=42)
    prob = muffin.make_problem(c.dirty, c.psf, n_wavelets=2, J=2)
    eps = fdmc_eps(c.noise_var)
    ref = sure.ada_pt(prob, c.delta, eps, c.noise_var, (0.05, 0.03), 9, Delta=4,
                      eta=(1e-4, 1e-4), reset=reset)
    x, theta, trace, states = parallel.ada_pt(prob, c.delta, eps, c.noise_var, (0.05, 0.03), 9,
                                      Delta=4, eta=(1e-4, 1e-4), reset=reset,
                                      workers=workers)
    assert np.max(np.abs(x - ref.x)) <= 1e-12 * np.max(np.abs(ref.x))
    for a, b in zip(states, ref.states):
        for k in ("x", "u", "v", "t"):
            ra, rb = getattr(a, k), getattr(b, k)
            assert np.max(np.abs(ra - rb)) <= 1e-12 * max(np.max(np.abs(rb)), 1e-300)
    assert np.allclose(theta, ref.theta, rtol=1e-12, atol=0)
    assert not np.allclose(theta, (0.05, 0.03))
    assert len(trace) == len(ref.trace) == 2
    for a, b in zip(trace, ref.trace):
        assert a["k"] == b["k"]
        assert np.allclose(a["sugar"], b["sugar"], rtol=1e-10, atol=0)
        assert a["psure"] == pytest.approx(b["psure"], rel=1e-12)
