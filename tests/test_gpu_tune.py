"""Per-shape launch tuning: every variant must give bit-identical results,
the tuner must pick a valid variant, invalidate the iterate state and cache
its choice (in process and in a text file)."""
import numpy as np
import pytest

from synth import fdmc_eps, make_cube
from tests.gpu_util import cuda, dev

pytestmark = pytest.mark.gpu


def _solve(pkg, torch, c, syn, ctas, iters=13, grad_chunk=0):
    x = torch.zeros((c.L, c.n, c.n), device="cuda")
    with pkg.Plan(c.n, c.L, c.psf) as p:
        p.set_tuning(syn, ctas)
        p.set_schedule(grad_chunk=grad_chunk)
        p.solve(dev(c.dirty, torch), x, iters, 1e-2, 2e-2)
    return x


@pytest.mark.parametrize("n,L", [(64, 8), (16, 20), (128, 64)])
def test_plain_variants_bit_identical(n, L):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=800 + n)
    ref = _solve(pkg, torch, c, 0, 0)
    for syn in range(4):
        for ctas in (0, 1, 2):
            if syn == 0 and ctas == 0:
                continue
            assert torch.equal(_solve(pkg, torch, c, syn, ctas), ref), (syn, ctas)
    # the gradient's FFT passes over image chunks (ragged last chunk included)
    for chunk in (1, 3, L - 1):
        assert torch.equal(_solve(pkg, torch, c, 0, 0, grad_chunk=chunk), ref), chunk


def test_fft_radix_plans_agree_and_match_oracle():
    """The radix-8 FFT plan (n >= 64) against the default radix-16 plan: same
    operator up to FP32 rounding, both within the gradient tolerance of the
    oracle, and a plain solve within the cube tolerance."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    from oracle import convolution
    from tests.gpu_util import host, rel_l2
    for n, L in ((64, 3), (256, 2), (1024, 1)):
        c = make_cube(n, L, max(2, n // 4), 1, 30 * n, seed=860 + n)
        x = np.random.default_rng(n).uniform(0, 1, (L, n, n)).astype(np.float32)
        hh = convolution.psf_spectrum(c.psf)
        ref = convolution.HT(convolution.H(x.astype(np.float64), hh) - c.dirty.astype(np.float64), hh)
        out = {}
        for radix in (16, 8):
            with pkg.Plan(n, L, c.psf) as p:
                p.set_schedule(fft_radix=radix)
                g = torch.empty((L, n, n), device="cuda")
                p.op_gradient(dev(x, torch), g, dirty=dev(c.dirty, torch))
                out[radix] = host(g)
            assert rel_l2(out[radix], ref) <= 1e-6, (n, radix)
    c = make_cube(64, 8, 16, 1, 1900, seed=870)
    xs = [_solve(pkg, torch, c, 0, 0, iters=30) for _ in range(1)]
    x8 = torch.zeros((c.L, c.n, c.n), device="cuda")
    with pkg.Plan(c.n, c.L, c.psf) as p:
        p.set_schedule(fft_radix=8)
        p.solve(dev(c.dirty, torch), x8, 30, 1e-2, 2e-2)
    assert rel_l2(host(x8), host(xs[0])) <= 1e-5


@pytest.mark.parametrize("sure", [False, True])
def test_analysis_ring_bit_identical(sure):
    """The U ring of the size-specialised analysis (512 px: levels 1 and 2)
    gives the same bits as the per-thread loads, plain and ADA-PT."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(512, 2, 30, 2, 3000, seed=890)
    eps = fdmc_eps(c.noise_var)
    res = []
    for ring in (0, 1):
        x = torch.zeros((c.L, c.n, c.n), device="cuda")
        with pkg.Plan(c.n, c.L, c.psf, sure=sure) as p:
            p.set_schedule(ana_ring=ring)
            if sure:
                th, tr, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                        (1e-2, 1e-2), 6, window=3, eta=(2e-3, 2e-2), eps=eps)
            else:
                p.solve(dev(c.dirty, torch), x, 6, 1e-2, 1e-2)
                th, tr = None, None
            st = p.state_arrays()
        res.append((x, th, tr, st))
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] and res[0][2] == res[1][2]
    for k in ("x", "u", "v", "t"):
        assert np.array_equal(res[0][3][k], res[1][3][k]), k


@pytest.mark.parametrize("n,L,sure,levels", [(512, 2, False, 3), (512, 2, True, 3),
                                             (1024, 2, True, 3), (2048, 1, False, 2),
                                             (64, 8, True, 3), (64, 8, False, 3),
                                             (32, 4, True, 1)])
def test_analysis_pipe_bit_identical(n, L, sure, levels):
    """The chain-major level-1 analysis with one barrier per step gives the
    same bits as the basis-major kernel: size-specialised (512, 1024, 2048 px)
    and run-time sizes, one and three chains; with one level the plan keeps
    the basis-major kernel (the setting has no effect)."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(n, L, max(4, n // 16), 2, 12 * n, seed=900 + n + L)
    eps = fdmc_eps(c.noise_var)
    res = []
    for pipe in (0, 1):
        x = torch.zeros((c.L, c.n, c.n), device="cuda")
        with pkg.Plan(c.n, c.L, c.psf, sure=sure, levels=levels) as p:
            p.set_schedule(ana_pipe=pipe)
            assert p.schedule()["ana_pipe"] == pipe
            if sure:
                th, tr, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                        (1e-2, 1e-2), 7, window=3, eta=(2e-3, 2e-2), eps=eps)
            else:
                p.solve(dev(c.dirty, torch), x, 5, 1e-2, 1e-2)
                th, tr = None, None
            st = p.state_arrays()
        res.append((x, th, tr, st))
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] and res[0][2] == res[1][2]
    for k in ("x", "u", "v", "t"):
        assert np.array_equal(res[0][3][k], res[1][3][k]), k


def test_group_order_bit_identical():
    """ADA-PT: the two chain groups' kernels phase by phase, or concurrently
    on two streams, give the same bits as group after group."""
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(64, 8, 16, 1, 1900, seed=880)
    eps = fdmc_eps(c.noise_var)
    res = []
    for order in (0, 1, 2):
        x = torch.zeros((c.L, c.n, c.n), device="cuda")
        with pkg.Plan(c.n, c.L, c.psf, sure=True) as p:
            p.set_schedule(group_order=order)
            th, tr, _ = p.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                    (0.03, 0.03), 23, window=5, eta=(1e-5, 1e-4), eps=eps)
        res.append((x, th, tr))
    for r in res[1:]:
        assert torch.equal(res[0][0], r[0]) and res[0][1] == r[1] and res[0][2] == r[2]


def test_sure_batch_variants_bit_identical():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    n, L, B = 32, 4, 2
    cs = [make_cube(n, L, 8, 1, 900, seed=820 + i) for i in range(B)]
    nv = np.concatenate([c.noise_var for c in cs])
    args = dict(window=5, eta=(2e-4, 2e-4), eps=fdmc_eps(nv))
    psf = np.stack([c.psf for c in cs])
    d = dev(np.stack([c.dirty for c in cs]), torch)
    de = dev(np.stack([c.delta for c in cs]), torch)
    out = []
    for syn, ctas, chunk in [(0, 0, 0), (3, 1, 5), (1, 2, 0), (2, 0, 7)]:
        x = torch.zeros((B, L, n, n), device="cuda")
        with pkg.Plan(n, L, psf, sure=True, batch=B) as p:
            p.set_tuning(syn, ctas)
            p.set_schedule(grad_chunk=chunk)
            th, tr, _ = p.sure_tune(d, de, nv, x, [(0.05, 0.05), (0.02, 0.08)], 15, **args)
        out.append((x, th, tr))
    for x, th, tr in out[1:]:
        assert torch.equal(x, out[0][0])
        assert th == out[0][1] and tr == out[0][2]


def test_autotune_choice_state_and_file_cache(tmp_path):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    c = make_cube(64, 8, 16, 1, 1900, seed=840)
    cache = tmp_path / "tune.txt"
    ref = _solve(pkg, torch, c, 0, 0)
    with pkg.Plan(64, 8, c.psf) as p:
        x = torch.zeros_like(ref)
        p.solve(dev(c.dirty, torch), x, 3, 1e-2, 2e-2)
        info = p.autotune(str(cache))
        # default, 3 more syn variants, 2 grids, radix 8, the other analysis kernel
        assert info.from_cache == 0 and info.candidates == 8
        assert 0 <= info.syn_packed <= 3 and info.dct_ctas_per_sm >= 0
        assert 0 < info.ms_best <= info.ms_default
        # the timing iterations replaced the iterate state: no warm start
        with pytest.raises(pkg.MuffinError) as e:
            p.solve(None, x, 2, 1e-2, 2e-2, warm=True)
        assert e.value.status == 6
        x = torch.zeros_like(ref)
        p.solve(dev(c.dirty, torch), x, 13, 1e-2, 2e-2)
        assert torch.equal(x, ref)
    lines = [ln.split() for ln in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0][0] == "muffin-tune-6" and "n=64,L=8" in lines[0][1]
    assert len(lines[0]) == 10
    # the same shape again: in-process cache
    with pkg.Plan(64, 8, c.psf) as p:
        again = p.autotune(str(cache))
        assert again.from_cache == 1 and again.candidates == 0
        assert (again.syn_packed, again.dct_ctas_per_sm) == (info.syn_packed, info.dct_ctas_per_sm)
    # a shape only the file knows (written by hand), beside lines to ignore
    key = lines[0][1].replace("n=64,L=8", "n=16,L=8")
    cache.write_text("garbage line\nmuffin-tune-6 %s 9 1 0 0 16 0 0 0\nmuffin-tune-5 %s 3 2 0 1 16 0 0\n"
                     "muffin-tune-6 %s 2 1 0 3 8 0 0 1\n" % (key, key, key))
    c16 = make_cube(16, 8, 4, 1, 480, seed=841)
    with pkg.Plan(16, 8, c16.psf) as p:
        got = p.autotune(str(cache))
        assert got.from_cache == 1
        assert (got.syn_packed, got.dct_ctas_per_sm, got.grad_chunk) == (2, 1, 3)
        assert got.ana_pipe == 1 and p.schedule()["ana_pipe"] == 1
        # a 16 px side has no radix-8 plan: the cached radix falls back to 16
        assert p.schedule()["grad_chunk"] == 3 and p.schedule()["fft_radix"] == 16


def test_set_tuning_rejects_bad_values():
    cuda()
    import paper_1905_08468_gb300 as pkg
    psf = np.zeros((4, 16, 16), np.float32)
    psf[:, 0, 0] = 1
    with pkg.Plan(16, 4, psf) as p:
        for bad in [(4, 0), (-1, 0), (0, -1)]:
            with pytest.raises(pkg.MuffinError) as e:
                p.set_tuning(*bad)
            assert e.value.status == 1


def test_convergence_mode_reports_trajectories(tmp_path):
    """bench.py --convergence on a small cube: one record per window, SNR and
    WMSE per chunk, finite values (the experiment itself is run at 256^2 x 32);
    the final SNR and WMSE of every start equal the oracle's metrics (Sec.
    4.1) of the saved cube against the true sky."""
    import json
    import os
    import subprocess
    import sys
    from oracle import convolution, metrics
    from synth import make_workload
    cuda()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    save = str(tmp_path / "final.npz")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--convergence",
                        "--workload", "c1_64x64x8", "--conv-iters", "120", "--conv-chunk", "60",
                        "--conv-inits", "3e-2,1e-1;3e-4,1e-3", "--conv-save", save],
                       capture_output=True, text=True, cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(out["runs"]) == 2
    for run in out["runs"]:
        assert [p["k"] for p in run["curve"]] == [60, 120]
        assert all(np.isfinite(p["snr_db"]) and p["wmse"] > 0 for p in run["curve"])
        assert run["theta_every"][0][0] == 10
        assert all(t >= 1e-8 for t in run["theta"])
    c = make_workload("c1_64x64x8")
    hh = convolution.psf_spectrum(c.psf)
    finals = np.load(save)
    for i, run in enumerate(out["runs"]):
        x = finals[f"x{i}"].astype(np.float64)
        assert run["snr_db"] == pytest.approx(metrics.snr_db(c.sky, x), abs=1e-5)
        assert run["wmse"] == pytest.approx(metrics.wmse(c.sky, x, hh), rel=1e-5)
