"""Spectral step on the tcgen05 tensor cores (64-band plans) against the
mma.sync kernel and the FP64 oracle: plain MUFFIN, ADA-PT, a ragged pixel
tile, batches."""
import numpy as np
import pytest

from oracle import muffin as om
from oracle import sure as osu
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _solve(pkg, torch, c, tc, iters, **kw):
    x = torch.zeros((c.L, c.n, c.n), device="cuda")
    with pkg.Plan(c.n, c.L, c.psf, **kw) as p:
        p.set_spectral_kernel(tc)
        p.solve(dev(c.dirty, torch), x, iters, 1e-2, 2e-2)
    return x


@pytest.mark.parametrize("n,iters", [(32, 60), (8, 40), (16, 30)])
def test_plain_tcgen05_matches_mma_sync_and_oracle(n, iters):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, 64, max(2, n // 4), 1, 30 * n, seed=1500 + n)
    xt = _solve(pkg, torch, c, True, iters)
    xm = _solve(pkg, torch, c, False, iters)
    assert rel_l2(host(xt), host(xm)) <= 1e-6
    prob = om.make_problem(c.dirty, c.psf)
    st, _ = om.solve(prob, 1e-2, 2e-2, iters)
    assert rel_l2(host(xt), st.x) <= 1e-5


def test_adapt_tcgen05_matches_oracle_and_batch():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 16, 64
    cs = [make_cube(n, L, 4, 1, 480, seed=1600 + i) for i in range(3)]
    nv = np.concatenate([c.noise_var for c in cs])
    eps = fdmc_eps(nv)
    args = dict(window=5, eta=(2e-4, 2e-4), eps=eps)
    singles = []
    for i, c in enumerate(cs):
        x = torch.zeros((L, n, n), device="cuda")
        with pkg.Plan(n, L, c.psf, sure=True) as p:
            th, tr, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                    (0.03, 0.02), 15, **args)
        singles.append((x, th, tr))
        if i == 0:
            prob = om.make_problem(c.dirty, c.psf)
            r = osu.ada_pt(prob, c.delta, eps, c.noise_var, (0.03, 0.02), 15, Delta=5,
                           eta=(2e-4, 2e-4))
            assert rel_l2(host(x), r.x) <= 1e-5
            assert np.max(np.abs(np.array(th) / r.theta - 1)) <= 1e-3
            xm = torch.zeros_like(x)
            with pkg.Plan(n, L, c.psf, sure=True) as p:
                p.set_spectral_kernel(False)
                thm, _, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var,
                                        xm, (0.03, 0.02), 15, **args)
            assert rel_l2(host(x), host(xm)) <= 1e-6
            assert np.max(np.abs(np.array(th) / np.array(thm) - 1)) <= 1e-6
    xb = torch.zeros((3, L, n, n), device="cuda")
    with pkg.Plan(n, L, np.stack([c.psf for c in cs]), sure=True, batch=3) as p:
        thb, trb, _ = p.sure_tune(dev(np.stack([c.dirty for c in cs]), torch),
                                  dev(np.stack([c.delta for c in cs]), torch), nv, xb,
                                  [(0.03, 0.02)] * 3, 15, **args)
    for i in range(3):
        assert torch.equal(xb[i], singles[i][0])
        assert thb[i] == singles[i][1] and trb[i] == singles[i][2]


def test_tcgen05_needs_64_bands():
    cuda()
    import paper_1905_08468_gb300 as pkg
    psf = np.zeros((32, 16, 16), np.float32)
    psf[:, 0, 0] = 1
    with pkg.Plan(16, 32, psf) as p:
        with pytest.raises(pkg.MuffinError) as e:
            p.set_spectral_kernel(True)
        assert e.value.status == 1
        p.set_spectral_kernel(False)


def test_bounded_wait_times_out_without_fault_and_plan_recovers():
    """The products are skipped on purpose (host-side hook), so the kernel's
    bounded waits run out: the call reports MUFFIN_ETIMEOUT, the context and
    the plan stay usable, and a normal call afterwards matches a fresh plan."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(16, 64, 4, 1, 480, seed=1700)
    ref = _solve(pkg, torch, c, True, 12)
    x = torch.zeros_like(ref)
    with pkg.Plan(16, 64, c.psf) as p:
        p.inject_timeout(True)
        with pytest.raises(pkg.MuffinError) as e:
            p.solve(dev(c.dirty, torch), x, 3, 1e-2, 2e-2)
        assert e.value.status == 4
        p.inject_timeout(False)
        x.zero_()
        p.solve(dev(c.dirty, torch), x, 12, 1e-2, 2e-2)
    torch.cuda.synchronize()
    assert torch.equal(x, ref)
