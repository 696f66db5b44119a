"""The MAD noise estimate (Sec. 3.1) on the GPU against the FP64 oracle:
per-band sigma_l^2 within 1e-5 relative (FP32 against FP64 Haar
coefficients; the medians are exact order statistics on both sides), for
even and odd coefficient counts, batched plans and the 1024 px side."""
import numpy as np
import pytest

from oracle import noise
from synth import make_cube
from tests.gpu_util import cuda, dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,B", [(2, 3, 1), (4, 2, 1), (64, 8, 1), (32, 4, 3), (1024, 2, 1)])
def test_mad_matches_oracle(n, L, B):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    rng = np.random.default_rng(n + L + B)
    y = (rng.standard_normal((B, L, n, n)) * rng.uniform(0.1, 2.0, (B, L, 1, 1))).astype(np.float32)
    y += np.linspace(0, 1, n, dtype=np.float32)[None, None, None, :]
    psf = np.zeros((B, L, n, n), np.float32)
    psf[..., 0, 0] = 1.0
    with pkg.Plan(n, L, psf if B > 1 else psf[0], batch=B, levels=1) as plan:
        got = np.asarray(plan.noise_mad(dev(y if B > 1 else y[0], torch))).reshape(B, L)
    for b in range(B):
        ref = noise.noise_var_mad(y[b].astype(np.float64))
        assert np.allclose(got[b], ref, rtol=1e-5, atol=0), (got[b], ref)


def test_mad_on_a_workload_cube():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(256, 8, 80, 4, 8000, seed=51)
    with pkg.Plan(256, 8, c.psf) as plan:
        got = plan.noise_mad(c.dirty)
    assert np.allclose(got, noise.noise_var_mad(c.dirty.astype(np.float64)), rtol=1e-5)
