"""IUWT (starlet) dictionary on the GPU against the FP64 oracle: single
operators, plain MUFFIN, ADA-PT, weights, batching and checkpoints."""
import numpy as np
import pytest

from oracle import iuwt, muffin as om, sure as osu
from oracle import weights as ow
from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _plan(pkg, c, J, **kw):
    return pkg.Plan(c.n, c.L, c.psf, levels=J, dictionary="iuwt", **kw)


@pytest.mark.parametrize("n,L,J", [(64, 4, 3), (32, 3, 4), (16, 2, 1), (8, 3, 2), (128, 2, 4)])
def test_operators_match_oracle(n, L, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=1000 + n + J)
    rng = np.random.default_rng(n + J)
    x = rng.normal(size=(L, n, n)).astype(np.float32)
    u = rng.normal(size=(L, J + 1, n, n)).astype(np.float32)
    with _plan(pkg, c, J) as p:
        uo = torch.zeros((L, J + 1, n, n), device="cuda")
        p.op_analysis(dev(x, torch), uo)
        xo = torch.zeros((L, n, n), device="cuda")
        p.op_synthesis(dev(u, torch), xo)
    assert rel_l2(host(uo), iuwt.analysis(x.astype(np.float64), J)) <= 1e-6
    assert rel_l2(host(xo), iuwt.adjoint(u.astype(np.float64), J)) <= 1e-6


@pytest.mark.parametrize("n,L,J,iters", [(64, 8, 3, 200), (32, 4, 2, 120), (16, 6, 4, 80)])
def test_plain_muffin_matches_oracle(n, L, J, iters):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=1100 + n)
    x = torch.zeros((L, n, n), device="cuda")
    with _plan(pkg, c, J) as p:
        p.solve(dev(c.dirty, torch), x, iters, 1e-2, 1e-2)
    prob = om.make_problem(c.dirty, c.psf, J=J, dictionary="iuwt")
    st, _ = om.solve(prob, 1e-2, 1e-2, iters)
    assert rel_l2(host(x), st.x) <= 1e-5


def test_adapt_matches_oracle_and_batch_equals_single():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, J = 32, 4, 3
    cs = [make_cube(n, L, 8, 1, 900, seed=1200 + i) for i in range(2)]
    nv = np.concatenate([c.noise_var for c in cs])
    eps = fdmc_eps(nv)
    args = dict(window=5, eta=(2e-4, 2e-4), eps=eps)
    xs = []
    for i, c in enumerate(cs):
        x = torch.zeros((L, n, n), device="cuda")
        with _plan(pkg, c, J, sure=True) as p:
            th, tr, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                    (0.03, 0.02), 20, **args)
        xs.append((x, th, tr))
        prob = om.make_problem(c.dirty, c.psf, J=J, dictionary="iuwt")
        r = osu.ada_pt(prob, c.delta, eps, c.noise_var, (0.03, 0.02), 20, Delta=5, eta=(2e-4, 2e-4))
        assert rel_l2(host(x), r.x) <= 1e-5
        assert np.max(np.abs(np.array(th) / r.theta - 1)) <= 1e-3
    xb = torch.zeros((2, L, n, n), device="cuda")
    with pkg.Plan(n, L, np.stack([c.psf for c in cs]), levels=J, dictionary="iuwt", sure=True,
                  batch=2) as p:
        thb, trb, _ = p.sure_tune(dev(np.stack([c.dirty for c in cs]), torch),
                                  dev(np.stack([c.delta for c in cs]), torch), nv, xb,
                                  [(0.03, 0.02), (0.03, 0.02)], 20, **args)
    for i in range(2):
        assert torch.equal(xb[i], xs[i][0]) and thb[i] == xs[i][1] and trb[i] == xs[i][2]


def test_weights_checkpoint_and_estimate():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, J = 32, 6, 3
    c = make_cube(n, L, 8, 1, 900, seed=1300)
    x0 = np.abs(c.dirty)
    with _plan(pkg, c, J) as p:
        assert p.device_bytes == pkg.estimate_bytes(n, L, levels=J, dictionary="iuwt")
        a, b = p.weights_from_x0(dev(x0, torch), 1e-2, 1e-3)   # allocates operator buffers
        d = dev(c.dirty, torch)
        x = torch.zeros_like(d)
        p.solve(d, x, 10, 1e-2, 1e-2)
        blob = p.state_export()
        p.solve(None, x, 10, 1e-2, 1e-2, warm=True)
        ref = x.clone()
        p.state_import(blob)
        p.solve(None, x, 10, 1e-2, 1e-2, warm=True)
        assert torch.equal(x, ref)
    # beta from the explicit transform: the starlet is not a tight frame
    ao, bo = ow.weights_from_x0(x0, J=J, eps_alpha=1e-2, eps_beta=1e-3, dictionary="iuwt")
    assert rel_l2(a, ao) <= 1e-6
    assert np.max(np.abs(b / bo - 1)) <= 1e-6
    # a Daubechies checkpoint does not load into a starlet plan
    with pkg.Plan(n, L, c.psf, levels=J, n_wavelets=J + 1) as q:
        with pytest.raises(pkg.MuffinError):
            q.state_import(blob)
    with pytest.raises(pkg.MuffinError) as e:
        pkg.Plan(n, L, c.psf, levels=5, dictionary="iuwt")
    assert e.value.status == 1
