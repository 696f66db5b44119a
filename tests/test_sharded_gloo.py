"""Data plane of the band-sharded solve (Sec. 2.3 split, paper_1905_08468_gb300.
sharded) on world-size-2 gloo ranks on the CPU: every rank computes its
halves of Algorithm 2 with the FP64 oracle's operators (a stand-in backend;
the GPU backend binds the same calls to the library), the exchanges
transpose z = 2 x~ - x and t between band and pixel blocks, tau comes from
the all-reduced Lipschitz constant, and the assembled cube must equal the
serial oracle's Algorithm 2 to FP64 rounding.  Uneven band blocks (5 bands
on 2 ranks, 7 on 3) are covered."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import convolution, muffin as om, spectral  # noqa: E402
from synth import make_cube  # noqa: E402


class OracleBackend:
    def __init__(self, c, l0, l1, p0, p1, K, J, sigma=10.0):
        self.prob = om.make_problem(c.dirty[l0:l1], c.psf[l0:l1], n_wavelets=K, J=J, sigma=sigma)
        self.L, self.n = c.L, c.n
        self.C = spectral.dct_matrix(c.L)
        self.sigma = sigma
        self.st = om.zero_state(self.prob)
        self.v = np.zeros((c.L, p1 - p0))

    def lipschitz(self):
        return convolution.lipschitz(self.prob.hhat)

    def zeros_band(self):
        return torch.zeros((self.prob.L, self.n, self.n), dtype=torch.float64)

    def spatial(self, t_band, mu, gamma, tau):
        p, st = self.prob, self.st
        x = st.x
        grad = convolution.HT(convolution.H(x, p.hhat) - p.y, p.hhat)
        s = mu * p.WsT(st.u)
        m = x - tau * (grad + s + t_band.numpy())
        xt = om.pos(m)
        z = 2.0 * xt - x
        st.u = om.sat(st.u + p.sigma * mu * p.Ws(z))
        st.x = xt
        return torch.from_numpy(z)

    def spectral(self, z_pix, p0, gamma):
        vt = self.v + self.sigma * gamma * (self.C @ z_pix.numpy())
        self.v = om.sat(vt)
        return torch.from_numpy(gamma * (self.C.T @ self.v))

    def x(self):
        return self.st.x


CASE = dict(n=16, K=3, J=2, mu=0.03, gamma=0.02, iters=9)


def _rank(rank, world, port, L, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1905_08468_gb300 import sharded
        n = CASE["n"]
        c = make_cube(n, L, 6, 1, 300, seed=77)
        bands = sharded.band_ranges(L, world)
        pix = sharded.pixel_ranges(n * n, world)
        be = OracleBackend(c, *bands[rank], *pix[rank], CASE["K"], CASE["J"])
        sol = sharded.BandShardedSolver(dist, be, n, L, CASE["K"], host_exchange=True)
        x = sol.solve(CASE["iters"], CASE["mu"], CASE["gamma"])
        np.save(os.path.join(outdir, f"x{rank}.npy"), x)
        np.save(os.path.join(outdir, f"tau{rank}.npy"), np.array([sol.tau(CASE["mu"], CASE["gamma"])]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("L,world,port", [(5, 2, 29631), (7, 3, 29632)])
def test_band_sharded_equals_serial(L, world, port):
    from paper_1905_08468_gb300 import sharded
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank, args=(world, port, L, d), nprocs=world, join=True)
        xs = [np.load(os.path.join(d, f"x{r}.npy")) for r in range(world)]
        taus = [float(np.load(os.path.join(d, f"tau{r}.npy"))[0]) for r in range(world)]
    x = np.concatenate(xs)
    c = make_cube(CASE["n"], L, 6, 1, 300, seed=77)
    prob = om.make_problem(c.dirty, c.psf, n_wavelets=CASE["K"], J=CASE["J"])
    st, tau = om.solve(prob, CASE["mu"], CASE["gamma"], CASE["iters"])
    assert all(t == pytest.approx(tau, rel=1e-14) for t in taus)
    assert np.max(np.abs(x - st.x)) <= 1e-12 * np.max(np.abs(st.x))
    assert sum(b - a for a, b in sharded.band_ranges(L, world)) == L


def test_partitions():
    from paper_1905_08468_gb300 import sharded
    assert sharded.band_ranges(7, 3) == [(0, 2), (2, 4), (4, 7)]
    pr = sharded.pixel_ranges(1024 * 1024, 6)
    assert pr[0][0] == 0 and pr[-1][1] == 1024 * 1024
    assert all((b - a) % 4 == 0 and b > a for a, b in pr)
    with pytest.raises(ValueError):
        sharded.pixel_ranges(18, 2)
