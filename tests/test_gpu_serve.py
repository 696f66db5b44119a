"""Request server: continuous batching of uneven cubes with admission by HBM
footprint.  Every result in the mix must equal the same request solved
alone (a plan of its own), and the pools must stay within the budget."""
import numpy as np
import pytest

from synth import make_cube
from tests.gpu_util import cuda, dev

pytestmark = pytest.mark.gpu


def alone(pkg, torch, c, mu, gamma, iters):
    x = torch.zeros((c.L, c.n, c.n), device="cuda")
    with pkg.Plan(c.n, c.L, c.psf) as p:
        p.solve(dev(c.dirty, torch), x, iters, mu, gamma)
    return x.cpu().numpy()


def drain(srv, tickets, outs, max_steps=10000):
    done = {}
    for _ in range(max_steps):
        srv.step()
        for t in tickets:
            if t not in done and srv.poll(t, outs[t]):
                done[t] = True
        if len(done) == len(tickets):
            return
    raise AssertionError("server did not finish")


def test_mix_equals_alone_uneven_shapes_and_iterations():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    specs = [(32, 4, 23, 1e-2, 1e-2), (64, 8, 40, 2e-2, 5e-3), (32, 4, 17, 5e-3, 2e-2),
             (32, 4, 30, 1e-2, 3e-2), (64, 8, 11, 1e-2, 1e-2), (32, 8, 25, 1e-2, 1e-2),
             (32, 4, 9, 3e-2, 1e-2)]
    cubes = [make_cube(n, L, n // 4, 1, 30 * n, seed=200 + i) for i, (n, L, *_) in enumerate(specs)]
    with pkg.Server(max_batch=3, chunk=7) as srv:
        tickets, outs = [], {}
        for c, (n, L, it, mu, ga) in zip(cubes, specs):
            t = srv.submit(c.psf, c.dirty, mu, ga, it)
            tickets.append(t)
            outs[t] = np.zeros((L, n, n), np.float32)
        drain(srv, tickets, outs)
        used, pools = srv.stats()
        assert pools >= 2
    for t, c, (n, L, it, mu, ga) in zip(tickets, cubes, specs):
        assert np.array_equal(outs[t], alone(pkg, torch, c, mu, ga, it)), (n, L, it)


def test_admission_by_footprint_queues_then_releases():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    # budget for exactly one pool of the larger shape: the two shapes must
    # take turns (an idle pool is released for the other shape)
    big = pkg.estimate_bytes(64, 8, batch=2)
    small = pkg.estimate_bytes(32, 4, batch=2)
    assert small < big
    budget = big + small // 2
    specs = [(64, 8, 12), (32, 4, 12), (64, 8, 8), (32, 4, 5)]
    cubes = [make_cube(n, L, n // 4, 1, 30 * n, seed=300 + i) for i, (n, L, _) in enumerate(specs)]
    with pkg.Server(max_batch=2, chunk=4, hbm_budget_bytes=budget) as srv:
        tickets, outs = [], {}
        for c, (n, L, it) in zip(cubes, specs):
            t = srv.submit(c.psf, c.dirty, 1e-2, 1e-2, it)
            tickets.append(t)
            outs[t] = np.zeros((L, n, n), np.float32)
        active, queued = srv.step()
        # the 32^2 request does not fit beside the 64^2 pool and nobody
        # overtakes it: arrival order is kept
        assert active == 1 and queued == 3
        assert srv.stats()[0] <= budget
        drain(srv, tickets, outs)
        assert srv.stats()[0] <= budget
        # a request whose pool can never fit is refused at submit
        huge = make_cube(256, 16, 8, 1, 2000, seed=9)
        with pytest.raises(pkg.MuffinError) as e:
            srv.submit(huge.psf, huge.dirty, 1e-2, 1e-2, 5)
        assert e.value.status == 2
    for t, c, (n, L, it) in zip(tickets, cubes, specs):
        assert np.array_equal(outs[t], alone(pkg, torch, c, 1e-2, 1e-2, it))


def test_active_work_cap_keeps_arrival_order():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    cs = [make_cube(32, 4, 8, 1, 900, seed=500 + i) for i in range(3)]
    with pkg.Server(max_batch=4, chunk=5, max_active_voxels=32 * 32 * 4) as srv:
        tickets = [srv.submit(c.psf, c.dirty, 1e-2, 1e-2, 10) for c in cs]
        assert srv.step() == (1, 2)               # one request's worth of voxels
        outs = {t: np.zeros((4, 32, 32), np.float32) for t in tickets}
        order = []
        for _ in range(50):
            srv.step()
            for t in tickets:
                if t not in order and srv.poll(t, outs[t]):
                    order.append(t)
            if len(order) == 3:
                break
        assert order == tickets
    for t, c in zip(tickets, cs):
        assert np.array_equal(outs[t], alone(pkg, torch, c, 1e-2, 1e-2, 10))


def test_device_buffers_and_poll_before_done():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(32, 4, 8, 1, 900, seed=401)
    with pkg.Server(max_batch=2, chunk=5) as srv:
        t = srv.submit(dev(c.psf, torch), dev(c.dirty, torch), 1e-2, 1e-2, 12)
        out = torch.zeros((4, 32, 32), device="cuda")
        assert not srv.poll(t, out)
        srv.step()
        assert not srv.poll(t, out)
        for _ in range(5):
            srv.step()
        assert srv.poll(t, out)
        with pytest.raises(pkg.MuffinError):
            srv.poll(t, out)                     # delivered tickets are released
    assert np.array_equal(out.cpu().numpy(), alone(pkg, torch, c, 1e-2, 1e-2, 12))


@pytest.mark.parametrize("n,L,B,sure,J", [(32, 4, 1, False, 3), (64, 8, 3, False, 3),
                                           (16, 5, 2, True, 2), (128, 16, 1, True, 3)])
def test_footprint_estimate_matches_allocation(n, L, B, sure, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    psf = np.zeros((B, L, n, n), np.float32)
    psf[:, :, 0, 0] = 1.0
    with pkg.Plan(n, L, psf, batch=B, sure=sure, levels=J) as p:
        assert pkg.estimate_bytes(n, L, batch=B, sure=sure, levels=J) == p.device_bytes


def test_nonfinite_request_is_rejected_without_stopping_the_server():
    """A request with a NaN in its dirty cube is rejected at admission (its
    poll reports MUFFIN_ENUMERIC and releases the ticket); the requests
    around it are served as usual."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    cs = [make_cube(32, 4, 8, 1, 900, seed=600 + i) for i in range(3)]
    bad = cs[1].dirty.copy()
    bad[1, 2, 3] = np.nan
    with pkg.Server(max_batch=2, chunk=5) as srv:
        t0 = srv.submit(cs[0].psf, cs[0].dirty, 1e-2, 1e-2, 10)
        t1 = srv.submit(cs[1].psf, bad, 1e-2, 1e-2, 10)
        t2 = srv.submit(cs[2].psf, cs[2].dirty, 1e-2, 1e-2, 10)
        outs = {t: np.zeros((4, 32, 32), np.float32) for t in (t0, t2)}
        rejected, done = False, set()
        for _ in range(100):
            srv.step()
            if not rejected:
                try:
                    srv.poll(t1, None)
                except pkg.MuffinError as e:
                    assert e.status == 5
                    rejected = True
            for t in outs:
                if t not in done and srv.poll(t, outs[t]):
                    done.add(t)
            if rejected and len(done) == 2:
                break
        assert rejected and len(done) == 2
        with pytest.raises(pkg.MuffinError):
            srv.poll(t1, None)                   # the ticket is released
    for t, c in ((t0, cs[0]), (t2, cs[2])):
        assert np.array_equal(outs[t], alone(pkg, torch, c, 1e-2, 1e-2, 10))
