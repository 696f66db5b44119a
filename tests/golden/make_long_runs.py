"""Writes ``long_runs.json``: summaries of long FP64 oracle runs that a GPU
test cannot wait for.  Calls only ``oracle/`` (its band-parallel form, which
is pinned to the serial oracle) and the shared input generator.

Runs (the plain ones are Algorithm 2 with mu = gamma = 1e-2 from X = 0; the
tuning run is Algorithm 5):

* ``c2``: the 256^2 x 32 workload (seed 2), 500 iterations;
* ``c5crop``: the 256^2 x 16 cube with the 2048^2 x 256 workload's
  densities (seed 5), 200 iterations;
* ``c3crop_adapt``: a 256^2 x 16 cube with the 1024^2 x 64 workload's
  densities (seed 3), ADA-PT from theta = (1e-2, 1e-2), 300 iterations,
  Delta = 10 (30 theta updates), eta = (3e-7, 3e-6), eps from the noise
  variances; the per-window SUGAR and PSURE and the final theta are stored.

Usage: python tests/golden/make_long_runs.py [workers]   (about an hour on 8
cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

from oracle import muffin, parallel  # noqa: E402
from synth import fdmc_eps, make_cube, make_workload  # noqa: E402
from summary import summarise  # noqa: E402

ADAPT = dict(theta0=(1e-2, 1e-2), iters=300, window=10, eta=(3e-7, 3e-6))


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else parallel.default_workers()
    out = {"source": "oracle.parallel (FP64), written by tests/golden/make_long_runs.py"}
    for key, wl, iters in (("c2", "c2_256x256x32", 500), ("c5crop", "c5crop_256x256x16", 200)):
        t = time.time()
        c = make_workload(wl)
        prob = muffin.make_problem(c.dirty, c.psf)
        x, tau = parallel.solve(prob, 1e-2, 1e-2, iters, workers=workers)
        out[key] = dict(workload=wl, iters=iters, mu=1e-2, gamma=1e-2, tau=tau,
                        x=summarise(x, seed=len(key)))
        print(f"{key}: {time.time() - t:.0f} s", flush=True)
    t = time.time()
    c = make_cube(256, 16, 125, 6, 12500, seed=3)
    prob = muffin.make_problem(c.dirty, c.psf)
    eps = fdmc_eps(c.noise_var)
    x, theta, trace, _ = parallel.ada_pt(prob, c.delta, eps, c.noise_var, ADAPT["theta0"],
                                      ADAPT["iters"], Delta=ADAPT["window"], eta=ADAPT["eta"],
                                      workers=workers)
    out["c3crop_adapt"] = dict(
        cube=dict(n=256, L=16, sources=125, blobs=6, uv=12500, seed=3), eps=eps,
        theta0=list(ADAPT["theta0"]), iters=ADAPT["iters"], window=ADAPT["window"],
        eta=list(ADAPT["eta"]), theta=[float(v) for v in theta],
        trace=[dict(k=r["k"], mu=float(r["theta"][0]), gamma=float(r["theta"][1]),
                    sugar_mu=float(r["sugar"][0]), sugar_gamma=float(r["sugar"][1]),
                    psure=float(r["psure"]), tau=float(r["tau"])) for r in trace],
        x=summarise(x, seed=7))
    print(f"c3crop_adapt: {time.time() - t:.0f} s, theta {theta}", flush=True)
    with open(os.path.join(HERE, "long_runs.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
