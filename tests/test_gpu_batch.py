"""Batched plans (several cubes advanced by the same launches) and CUDA-graph
replay: a batch must reproduce independent single-cube plans exactly, and
graph replay must reproduce direct launches exactly."""
import numpy as np
import pytest

from oracle import muffin as om
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def cubes(n, L, B, seed0):
    return [make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=seed0 + i) for i in range(B)]


@pytest.mark.parametrize("n,L,B", [(32, 4, 3), (64, 8, 2), (16, 20, 3)])
def test_batched_solve_equals_single_plans(n, L, B):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    cs = cubes(n, L, B, 50)
    mus = [1e-2, 2e-2, 5e-3][:B]
    gammas = [1e-2, 3e-3, 2e-2][:B]
    psf = np.stack([c.psf for c in cs])
    dirty = dev(np.stack([c.dirty for c in cs]), torch)
    xb = torch.zeros((B, L, n, n), device="cuda")
    with pkg.Plan(n, L, psf, batch=B) as plan:
        plan.solve(dirty, xb, 25, mus, gammas)
        lips = plan.lipschitz
    for i, c in enumerate(cs):
        xs = torch.zeros((L, n, n), device="cuda")
        with pkg.Plan(n, L, c.psf) as p1:
            p1.solve(dev(c.dirty, torch), xs, 25, mus[i], gammas[i])
            assert p1.lipschitz == lips[i]
        assert torch.equal(xs, xb[i]), i
    # and one cube against the FP64 oracle
    prob = om.make_problem(cs[1].dirty, cs[1].psf)
    st, _ = om.solve(prob, mus[1], gammas[1], 25)
    assert rel_l2(host(xb[1]), st.x) <= 1e-5


def test_graph_replay_equals_direct_launches():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(64, 8, 10, 2, 1500, seed=61)
    d = dev(c.dirty, torch)
    out = []
    for graphs in (True, False):
        x = torch.zeros_like(d)
        with pkg.Plan(64, 8, c.psf) as p:
            p.graphs(graphs)
            p.solve(d, x, 17, 1e-2, 1e-2)           # odd count: graph + tail
            p.solve(None, x, 8, 1e-2, 1e-2, warm=True)
        out.append(x)
    assert torch.equal(out[0], out[1])


def test_batched_sure_equals_single_plans_and_graphs():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, B = 32, 4, 2
    cs = cubes(n, L, B, 70)
    eps = fdmc_eps(np.concatenate([c.noise_var for c in cs]))
    args = dict(window=5, eta=(2e-4, 2e-4), eps=eps)
    theta0 = [(0.05, 0.05), (0.02, 0.08)]
    psf = np.stack([c.psf for c in cs])
    d = dev(np.stack([c.dirty for c in cs]), torch)
    de = dev(np.stack([c.delta for c in cs]), torch)
    nv = np.concatenate([c.noise_var for c in cs])
    res = {}
    for graphs in (True, False):
        xb = torch.zeros((B, L, n, n), device="cuda")
        with pkg.Plan(n, L, psf, sure=True, batch=B) as plan:
            plan.graphs(graphs)
            th, tr, info = plan.sure_tune(d, de, nv, xb, theta0, 23, **args)
        res[graphs] = (xb, th, tr)
    assert torch.equal(res[True][0], res[False][0])
    assert res[True][1] == res[False][1] and res[True][2] == res[False][2]
    xb, th, tr = res[True]
    assert [t["k"] for t in tr[0]] == [5, 10, 15, 20]
    for i, c in enumerate(cs):
        xs = torch.zeros((L, n, n), device="cuda")
        with pkg.Plan(n, L, c.psf, sure=True) as p1:
            th1, tr1, _ = p1.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var,
                                       xs, theta0[i], 23, **args)
        assert torch.equal(xs, xb[i])
        assert th1 == th[i] and tr1 == tr[i]
