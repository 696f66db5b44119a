"""The band-sharded halves of Algorithm 2 on the GPU (muffin_shard_spatial /
muffin_shard_spectral through paper_1905_08468_gb300.sharded) with every
band on one rank: the split iteration, with its exchanges, must reproduce
muffin_solve's fused iteration (the spectral half reads z = 2 x~ - x, and the
kernel's 2 z - z is exactly z).  One rank on one GPU: the exchanges are
identities on a gloo group of one process; several ranks are covered on the
CPU (tests/test_sharded_gloo.py), and several GPUs are unmeasured."""
import numpy as np
import pytest

from synth import make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,port", [(64, 8, 29661), (64, 64, 29662)])
def test_sharded_single_rank_equals_fused(n, L, port):
    torch = cuda()
    import torch.distributed as dist
    import paper_1905_08468_gb300 as pkg
    from paper_1905_08468_gb300 import sharded
    c = make_cube(n, L, 16, 2, 1500, seed=90 + L)
    mu, gamma, iters = 1e-2, 2e-2, 12
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(n, L, c.psf) as plan:
        info = plan.solve(dev(c.dirty, torch), x, iters, mu, gamma)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        be = sharded.GpuBackend(pkg, torch, n, L, 0, L, 0, n * n, c.psf, c.dirty)
        sol = sharded.BandShardedSolver(dist, be, n, L, 8, host_exchange=True)
        assert sol.tau(mu, gamma) == pytest.approx(info.tau, rel=1e-14)
        xs = sol.solve(iters, mu, gamma)
    finally:
        dist.destroy_process_group()
    e = rel_l2(xs, host(x))
    print(f"sharded vs fused {n}^2 x {L}: {e:.2e}, identical: {np.array_equal(xs, host(x).astype(np.float32))}")
    assert e <= 1e-6
