"""FP32 spectral step (plans with precision "fp32"): the orthonormal DCT-II of
every pixel spectrum by Makhoul's fast algorithm on the CUDA cores, against
the FP64 oracle's dense DCT matrix, in the operator, in plain MUFFIN and in
ADA-PT (the d/dgamma chain's inhomogeneous terms of Algorithm 4), with
ragged pixel tiles; and the primal step override tau."""
import numpy as np
import pytest

from oracle import muffin as om, spectral
from synth import make_cube
from tests.gpu_util import cuda, dev, host, rel_l2
from tests.test_gpu_states import run_case

pytestmark = pytest.mark.gpu

# (n, L): pixels per tile are 512 / L pairs up to 128 pairs, so 8^2 px is a
# single ragged tile below 128 bands and 4^2 px spans two tiles at 1024
OP_SHAPES = [(4, 2), (8, 4), (8, 8), (16, 16), (8, 32), (32, 64), (8, 64), (8, 128),
             (16, 256), (4, 512), (4, 1024)]


@pytest.mark.parametrize("n,L", OP_SHAPES)
@pytest.mark.parametrize("inverse", [False, True])
def test_fp32_dct_operator_matches_oracle(n, L, inverse):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    rng = np.random.default_rng(7 * L + n)
    x = rng.standard_normal((L, n, n)).astype(np.float32)
    C = spectral.dct_matrix(L)
    ref = spectral.apply_spectra(C.T if inverse else C, x.astype(np.float64))
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1
    with pkg.Plan(n, L, psf, n_wavelets=1, levels=1, precision="fp32") as plan:
        v = torch.empty((L, n, n), device="cuda")
        plan.op_dct(dev(x, torch), v, inverse=inverse)
        e = rel_l2(host(v), ref)
        # C^T C = I through both FP32 transforms
        back = torch.empty_like(v)
        plan.op_dct(v, back, inverse=not inverse)
        eb = rel_l2(host(back), x)
    print(f"fp32 DCT n={n} L={L} inverse={inverse}: {e:.1e}, round trip {eb:.1e}")
    assert e <= 1e-6, e
    assert eb <= 2e-6, eb


@pytest.mark.parametrize("n,L,iters", [(16, 8, 40), (16, 64, 30), (8, 256, 20), (32, 32, 25)])
def test_plain_fp32_matches_oracle_and_tf32(n, L, iters):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=4100 + L + n)
    xs = {}
    for prec in ("fp32", "tf32"):
        x = torch.zeros((L, n, n), device="cuda")
        with pkg.Plan(n, L, c.psf, precision=prec) as p:
            p.solve(dev(c.dirty, torch), x, iters, 1e-2, 2e-2)
        xs[prec] = host(x)
    prob = om.make_problem(c.dirty, c.psf)
    st, _ = om.solve(prob, 1e-2, 2e-2, iters)
    e32, etf = rel_l2(xs["fp32"], st.x), rel_l2(xs["tf32"], st.x)
    print(f"plain {n}^2 x {L}: fp32 {e32:.1e}, tf32 {etf:.1e}")
    assert e32 <= 1e-5
    assert rel_l2(xs["fp32"], xs["tf32"]) <= 1e-5


@pytest.mark.parametrize("n,L,levels,sure", [(16, 2, 3, True), (4, 1024, 2, False),
                                             (8, 512, 3, True)])
def test_fp32_band_count_extremes(n, L, levels, sure):
    """The iteration at the smallest and largest band counts of the FP32
    step (one task per pixel pair at L = 2; 8-pixel tiles at L = 1024)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    from oracle import sure as osure
    from synth import fdmc_eps
    c = make_cube(n, L, 2, 1, 20 * n, seed=4500 + L)
    prob = om.make_problem(c.dirty, c.psf, J=levels)
    x = torch.zeros((L, n, n), device="cuda")
    with pkg.Plan(n, L, c.psf, levels=levels, sure=sure, precision="fp32") as p:
        if sure:
            eps = fdmc_eps(c.noise_var)
            th, _, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                   (0.05, 0.05), 10, window=5, eta=(2e-5, 2e-4), eps=eps)
            ref = osure.ada_pt(prob, c.delta, eps, c.noise_var, (0.05, 0.05), 10, Delta=5,
                               eta=(2e-5, 2e-4))
            refx = ref.x
            assert np.max(np.abs(np.array(th) / ref.theta - 1)) <= 1e-3
        else:
            p.solve(dev(c.dirty, torch), x, 15, 1e-2, 2e-2)
            refx = om.solve(prob, 1e-2, 2e-2, 15)[0].x
    e = rel_l2(host(x), refx)
    print(f"fp32 {n}^2 x {L} sure={sure}: {e:.1e}")
    assert e <= 1e-5


def test_adapt_fp32_states_match_oracle():
    """ADA-PT with the FP32 spectral step: every chain's X, U, V, T element by
    element against the oracle (64 bands, so the d/dgamma chain's spectral
    terms are the ones the tcgen05 kernel accumulates in tensor memory)."""
    c = make_cube(32, 64, 12, 2, 1500, seed=4200)
    run_case(c, (1e-2, 1e-2), 8, 3, (1e-5, 1e-5), precision="fp32")


def test_adapt_fp32_16_bands_moving_theta():
    c = make_cube(32, 16, 10, 2, 800, seed=4201)
    run_case(c, (0.05, 0.05), 13, 5, (2e-5, 2e-4), precision="fp32")


def test_fp32_batch_equals_singles():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 16, 32
    cs = [make_cube(n, L, 4, 1, 480, seed=4300 + i) for i in range(2)]
    singles = []
    for c in cs:
        x = torch.zeros((L, n, n), device="cuda")
        with pkg.Plan(n, L, c.psf, precision="fp32") as p:
            p.solve(dev(c.dirty, torch), x, 12, 1e-2, 2e-2)
        singles.append(x)
    xb = torch.zeros((2, L, n, n), device="cuda")
    with pkg.Plan(n, L, np.stack([c.psf for c in cs]), precision="fp32", batch=2) as p:
        p.solve(dev(np.stack([c.dirty for c in cs]), torch), xb, 12, [1e-2] * 2, [2e-2] * 2)
    for i in range(2):
        assert torch.equal(xb[i], singles[i])


def test_fp32_rejections():
    cuda()
    import paper_1905_08468_gb300 as pkg
    for L in (1, 100, 2048):
        psf = np.zeros((L, 8, 8), np.float32)
        psf[:, 0, 0] = 1
        with pytest.raises(pkg.MuffinError):
            pkg.Plan(8, L, psf, precision="fp32")
    psf = np.zeros((64, 8, 8), np.float32)
    psf[:, 0, 0] = 1
    with pkg.Plan(8, 64, psf, precision="fp32") as p:
        with pytest.raises(pkg.MuffinError):
            p.set_spectral_kernel(True)
    with pytest.raises(ValueError):
        pkg.Plan(8, 64, psf, precision="fp16")
    assert pkg.estimate_bytes(8, 64, precision="fp32") > pkg.estimate_bytes(8, 64)
    # the footprint estimate is exact for FP32-precision plans too
    for n, L, sure, batch in [(16, 64, True, 1), (32, 256, False, 2), (8, 2, False, 1)]:
        psf = np.zeros((batch, L, n, n), np.float32)
        psf[:, :, 0, 0] = 1
        with pkg.Plan(n, L, psf if batch > 1 else psf[0], sure=sure, batch=batch,
                      precision="fp32") as p:
            assert p.device_bytes == pkg.estimate_bytes(n, L, sure=sure, batch=batch,
                                                        precision="fp32")


def test_tau_override_plain_and_adapt():
    """A fixed tau replaces the step rule: the plain solve equals the oracle's
    Algorithm 2 run with that tau, and every ADA-PT window reports it."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L = 16, 8
    c = make_cube(n, L, 4, 1, 480, seed=4400)
    prob = om.make_problem(c.dirty, c.psf)
    tau_rule = om.step_tau(prob, 1e-2, 2e-2)
    tau = 0.6 * tau_rule
    x = torch.zeros((L, n, n), device="cuda")
    with pkg.Plan(n, L, c.psf, tau=tau) as p:
        info = p.solve(dev(c.dirty, torch), x, 30, 1e-2, 2e-2)
    assert info.tau == tau
    st, t_used = om.solve(prob, 1e-2, 2e-2, 30, tau=tau)
    assert t_used == tau
    assert rel_l2(host(x), st.x) <= 1e-5
    st_rule, _ = om.solve(prob, 1e-2, 2e-2, 30)
    assert rel_l2(host(x), st_rule.x) > 1e-4      # the override changed the iterates
    xs = torch.zeros((L, n, n), device="cuda")
    with pkg.Plan(n, L, c.psf, sure=True, tau=tau) as p:
        _, trace, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, xs,
                                  (0.05, 0.05), 10, window=5, eta=(2e-5, 2e-4), eps=1e-3)
    assert trace and all(r["tau"] == tau for r in trace)
    with pytest.raises(pkg.MuffinError):
        pkg.Plan(n, L, c.psf, tau=-1.0)
