"""Long runs of the workload configurations against stored FP64 oracle runs.

The oracle needs about an hour of CPU for these, so ``tests/golden/
make_long_runs.py`` (which calls only ``oracle/``) stored, per run, the cube
at 2048 fixed voxels, its per-band norms and 32 Rademacher projections
(``tests/golden/summary.py``).  The GPU run is compared through them:

* 256^2 x 32, mu = gamma = 1e-2, 500 iterations (Algorithm 2);
* 256^2 x 16 with the 2048^2 x 256 workload's densities, 200 iterations;
* 256^2 x 16 with the 1024^2 x 64 workload's densities, ADA-PT (Algorithm
  5), 300 iterations, Delta = 10 (30 theta updates): the cube, the final
  theta and every window's SUGAR and PSURE.

Tolerances: cube relative L2 1e-5 (on the sampled voxels, and as estimated
from the projections), theta 1e-3, SUGAR/PSURE 1e-3.  The plain runs are
repeated with the FP32 spectral step (precision "fp32") against the same
stored oracle runs.
"""
import json
import os
import sys

import numpy as np
import pytest

from synth import make_cube, make_workload
from tests.gpu_util import cuda, dev, host

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
from summary import errors  # noqa: E402

pytestmark = pytest.mark.gpu

GOLD = os.path.join(HERE, "golden", "long_runs.json")


def golden(key):
    if not os.path.exists(GOLD):
        pytest.fail("tests/golden/long_runs.json is missing (run tests/golden/make_long_runs.py)")
    with open(GOLD) as f:
        return json.load(f)[key]


def check_cube(x, s, tol=1e-5):
    e = errors(x, s)
    print({k: f"{v:.2e}" for k, v in e.items()})
    assert e["sampled"] <= tol, e
    assert e["projected"] <= tol, e
    assert e["band_norm"] <= tol, e


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
@pytest.mark.parametrize("key", ["c2", "c5crop"])
def test_plain_long_run(key, precision):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    g = golden(key)
    c = make_workload(g["workload"])
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, precision=precision) as plan:
        info = plan.solve(dev(c.dirty, torch), x, g["iters"], g["mu"], g["gamma"])
    assert info.tau == pytest.approx(g["tau"], rel=1e-12)
    check_cube(host(x), g["x"])


def test_adapt_300_iterations_of_the_tuning_crop():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    g = golden("c3crop_adapt")
    cb = g["cube"]
    c = make_cube(cb["n"], cb["L"], cb["sources"], cb["blobs"], cb["uv"], seed=cb["seed"])
    x = dev(np.zeros_like(c.dirty), torch)
    with pkg.Plan(c.n, c.L, c.psf, sure=True) as plan:
        th, trace, _ = plan.sure_tune(dev(c.dirty, torch), dev(c.delta, torch), c.noise_var, x,
                                      tuple(g["theta0"]), g["iters"], window=g["window"],
                                      eta=tuple(g["eta"]), eps=g["eps"])
    check_cube(host(x), g["x"])
    assert len(trace) == len(g["trace"]) == g["iters"] // g["window"]
    for tg, to in zip(trace, g["trace"]):
        assert tg["k"] == to["k"]
        assert tg["sugar_mu"] == pytest.approx(to["sugar_mu"], rel=1e-3)
        assert tg["sugar_gamma"] == pytest.approx(to["sugar_gamma"], rel=1e-3)
        assert tg["psure"] == pytest.approx(to["psure"], rel=1e-3)
    for j in range(2):
        assert g["theta"][j] > 1e-6, "theta reached the clamp: the comparison would be vacuous"
        assert abs(g["theta"][j] - g["theta0"][j]) > 1e-2 * g["theta0"][j]
        assert th[j] == pytest.approx(g["theta"][j], rel=1e-3)
