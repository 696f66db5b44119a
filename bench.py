#!/usr/bin/env python
"""Throughput of ADA-PT'ed MUFFIN on GB300: voxel-iterations per second.

Workload (default): the 1024 x 1024 x 64 cube of the synthetic recipe
(2000 point sources, 100 blobs, 200000 uv points, 20 dB per band), MUFFIN
with SURE/SUGAR auto-tuning of (mu, gamma).  One step = one
``muffin_sure_tune`` call of 300 ADA-PT iterations (window 10, so 30 theta
updates) from X0 = 0; a voxel-iteration advances one pixel of one band by one
iteration in all six chains (primal and FDMC primal, four derivative chains).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead, on a bounded crop of the same workload.
Multi-GPU (torchrun): every rank solves its own cube (replicas, weak scaling,
no collective on the data path); the timed region is bracketed by barriers
and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-iters/s (px x bands x iters) at 1024^2 x 64, ADA-PT'ed MUFFIN"
UNIT = "voxel-iters/s"
THETA0 = (1e-2, 1e-2)
# gradient steps that move theta by about 1 % (mu) and 2 % (gamma) per window
# at 1024^2 x 64 (SUGAR there is ~2e4 for mu and ~3e3 for gamma at the start)
ETA = (5e-9, 5e-8)
# oracle sample: the top-left 128^2 pixels of all 64 bands (the per-pixel DCT
# step keeps its share of the work), two ADA-PT iterations
CROP = dict(n=128, L=64, iters=2)

# DRAM bytes (read + write) per chain-voxel of a kernel, from a committed
# ncu capture (profiles/), valid only while the kernel's source file is the
# one the counters were taken on (sha256 prefix).
CAPTURED_TRAFFIC = {
    "ana_level1_dual": ("paper_1905_08468_gb300/csrc/wavelet.cu", "d2db0c7118e4171c", 61.63),
}


# ------------------------------------------------------------------ ranks
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, _, world = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29512")
        dist.init_process_group(backend, rank=rank, world_size=world)
    return dist


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(v: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        return parse_clocks(self.f.read())


def parse_clocks(text: str) -> dict:
    sm, mx, reasons = [], [], set()
    for line in text.strip().splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for name, val in zip(REASONS, parts[5:9]):
            if val.lower() == "active":
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle leg
# The oracle runs in a subprocess of its own (no CUDA, its own BLAS settings)
# on a crop saved once by the parent; `parallel` selects the band-parallel
# form (Sec. 2.3 split) on all cores.
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from synth import fdmc_eps
from oracle import muffin as om, sure as osure, parallel as opar
if __name__ == "__main__":
    z = np.load({crop!r})
    iters = {iters}
    prob = om.make_problem(z["dirty"], z["psf"])
    nv = z["noise_var"]
    eps = fdmc_eps(nv)
    workers = opar.default_workers() if {parallel!r} else 1
    t0 = time.perf_counter()
    if {parallel!r}:
        opar.ada_pt(prob, z["delta"], eps, nv, {theta0!r}, iters, Delta=10, eta=(0.0, 0.0),
                    workers=workers)
    else:
        osure.ada_pt(prob, z["delta"], eps, nv, {theta0!r}, iters, Delta=10, eta=(0.0, 0.0))
    dt = time.perf_counter() - t0
    print(json.dumps(dict(seconds=dt, voxels=int(z["dirty"].size), iters=iters, cores=workers)))
"""

_CROP_FILE = None


def crop_file(name: str, cube=None) -> str:
    """The oracle's sample: the top-left CROP['n']^2 pixels of the first
    CROP['L'] bands of the workload, saved once per process."""
    global _CROP_FILE
    if _CROP_FILE is None:
        import numpy as np
        if cube is None:
            from synth import make_workload
            cube = make_workload(name)
        n, L = CROP["n"], CROP["L"]
        sl = (slice(0, L), slice(0, n), slice(0, n))
        fd, path = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        np.savez(path, dirty=cube.dirty[sl], psf=cube.psf[sl], delta=cube.delta[sl],
                 noise_var=cube.noise_var[:L])
        _CROP_FILE = path
    return _CROP_FILE


def oracle_sample(name: str, parallel: bool, cube=None) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SAMPLE.format(root=ROOT, crop=crop_file(name, cube), theta0=THETA0,
                                parallel=parallel, iters=CROP["iters"])
    with tempfile.NamedTemporaryFile("w", suffix=".py", delete=False) as f:
        f.write(code)       # a file, so that spawned workers can re-import it
    try:
        r = subprocess.run([sys.executable, f.name], capture_output=True, text=True,
                           env=env, timeout=900)
    finally:
        os.unlink(f.name)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-2000:]}")
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["value"] = d["voxels"] * d["iters"] / d["seconds"]
    return d


def cpu_baseline_obj(d: dict) -> dict:
    form = (f"band-parallel (Sec. 2.3 split), {d['cores']} worker processes"
            if d["cores"] > 1 else "1 thread")
    return {"value": d["value"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, {d['iters']} ADA-PT iterations (6 chains) "
                       f"on the top-left {CROP['n']}x{CROP['n']} px of all {CROP['L']} bands "
                       f"of the 1024^2 x 64 cube, {form}, {d['seconds']:.1f} s")}


def run_reference(args) -> None:
    rank, _, world = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(args.workload, parallel=True)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        d = oracle_sample(args.workload, parallel=True)
        vals.append(d["value"])
        secs += d["seconds"]
    v = statistics.mean(vals)
    last = dict(d, value=v)
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args, oracle=True),
           "cpu_baseline": cpu_baseline_obj(last),
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU leg
def workload_config(args, oracle=False) -> dict:
    from synth import WORKLOADS
    n, L, n_src, n_blob, n_uv, seed = WORKLOADS[args.workload]
    plain = getattr(args, "plain", False)
    cfg = {"workload": (f"plain MUFFIN {n}x{n} px x {L} bands, mu = gamma = {args.mu:g}" if plain
                        else f"ADA-PT'ed MUFFIN {n}x{n} px x {L} bands"),
           "n": n, "bands": L, "sources": n_src, "blobs": n_blob, "uv_points": n_uv,
           "snr_db": 20, "seed": seed, "iters_per_step": args.iters,
           "window": args.window,
           "wavelets": ("IUWT (starlet), 3 scales" if getattr(args, "dictionary", "daubechies") == "iuwt"
                        else "db1..db8, 3 levels"),
           "spectral": ("DCT-II in FP32 on the CUDA cores (fast DCT, one complex DFT per pixel pair)"
                        if getattr(args, "precision", "tf32") == "fp32" else
                        "DCT-II, 3xTF32 products on the tensor cores (tcgen05 for 64 bands, else mma.sync)"),
           "chains": 1 if plain else 6,
           "theta0": None if plain else list(THETA0), "eta": None if plain else list(ETA),
           "l2": "inputs larger than L2 (state ~26 GB per cube at 1024^2 x 64 ADA-PT)"}
    if oracle:
        cfg["oracle_sample"] = dict(CROP)
    return cfg


def captured_traffic(kernel: str, chain_voxels: float):
    import hashlib
    ent = CAPTURED_TRAFFIC.get(kernel)
    if not ent:
        return None
    path, sha, per_voxel = ent
    with open(os.path.join(ROOT, path), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != sha:
            return None
    return per_voxel * chain_voxels


# ------------------------------------------------------------------ serving
def nearest_rank(vals, q):
    v = sorted(vals)
    return v[max(0, math.ceil(q * len(v)) - 1)]


def serve_cube(n, L, seed):
    from synth import make_cube
    r = (n / 256.0) ** 2      # densities per pixel of the 256^2 x 32 workload
    return make_cube(n, L, max(1, round(200 * r)), max(1, round(20 * r)),
                     max(100, round(20000 * r)), seed, with_delta=False)


def run_serve(args) -> None:
    """Served Poisson stream: continuous batching (muffin_server) against the
    same stream served one cube per launch, first come first served, no
    graphs.  Latency = result ready - arrival."""
    import numpy as np
    import torch
    from synth import serve_stream
    import paper_1905_08468_gb300 as pkg

    torch.cuda.set_device(0)
    stream = serve_stream(seed=args.serve_seed)[: args.serve_requests]
    if args.serve_rate != 4.0:          # same draws, arrivals rescaled (0: one burst)
        k = 0.0 if args.serve_rate <= 0 else 4.0 / args.serve_rate
        stream = [(t * k, n, L, sd) for t, n, L, sd in stream]
    cubes = [serve_cube(n, L, seed) for _, n, L, seed in stream]
    iters, mu = args.serve_iters, 1e-2

    def replay(run_one):
        lat, t0 = [], time.perf_counter()
        run_one(t0, lat)
        make = time.perf_counter() - t0
        vox = sum(c.voxels for c in cubes) * iters
        return lat, make, vox / make

    outs_b = {}

    def batched(t0, lat):
        with pkg.Server(max_batch=args.serve_batch, chunk=args.serve_chunk) as srv:
            nxt, tick, arr = 0, {}, {}
            while len(lat) < len(stream):
                now = time.perf_counter() - t0
                while nxt < len(stream) and stream[nxt][0] <= now:
                    c = cubes[nxt]
                    t = srv.submit(c.psf, c.dirty, mu, mu, iters)
                    tick[t], arr[t] = nxt, stream[nxt][0]
                    nxt += 1
                active, queued = srv.step()
                for t in list(tick):
                    c = cubes[tick[t]]
                    out = np.empty((c.L, c.n, c.n), np.float32)
                    if srv.poll(t, out):
                        lat.append(time.perf_counter() - t0 - arr[t])
                        outs_b[tick[t]] = out
                        del tick[t]
                if active == 0 and queued == 0 and nxt < len(stream):
                    time.sleep(max(0.0, stream[nxt][0] - (time.perf_counter() - t0)))

    outs_1 = {}

    def one_by_one(t0, lat):
        plans = {}
        for i, (arr, n, L, _) in enumerate(stream):
            wait = arr - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            c = cubes[i]
            if (n, L) not in plans:
                plans[(n, L)] = pkg.Plan(n, L, c.psf)
                plans[(n, L)].graphs(False)
            p = plans[(n, L)]
            p.load_psf(c.psf)
            x = np.zeros((L, n, n), np.float32)
            p.solve(c.dirty, x, iters, mu, mu)
            lat.append(time.perf_counter() - t0 - arr)
            outs_1[i] = x
        for p in plans.values():
            p.close()

    lb, mb, tb = replay(batched)
    l1, m1, t1 = replay(one_by_one)
    same = all(np.array_equal(outs_b[i], outs_1[i]) for i in range(len(stream)))
    rate = "burst" if args.serve_rate <= 0 else f"{args.serve_rate:g}/s"
    out = {"metric": f"served stream: p50/p99 latency and throughput ({len(stream)} Poisson requests, {rate})",
           "value": tb, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
           "higher_is_better": True, "data": "synthetic", "dtype": "f32",
           "config": {"workload": "served Poisson stream, n in {128,256,512}, "
                                  "L in {16,32,64}", "requests": len(stream),
                      "arrival_seed": args.serve_seed,
                      "iters": iters, "mu": mu, "gamma": mu, "max_batch": args.serve_batch,
                      "chunk": args.serve_chunk},
           "batched": {"p50_s": nearest_rank(lb, 0.5), "p99_s": nearest_rank(lb, 0.99),
                       "makespan_s": mb, "voxel_iters_per_s": tb},
           "one_cube_per_launch": {"p50_s": nearest_rank(l1, 0.5),
                                   "p99_s": nearest_rank(l1, 0.99),
                                   "makespan_s": m1, "voxel_iters_per_s": t1},
           "results_identical": same}
    print(json.dumps(out), flush=True)


def run_convergence(args) -> None:
    """ADA-PT'ed MUFFIN from several initial (mu, gamma) on a synthetic cube
    (the convergence experiment of Sec. 4.2.2, on a stand-in for its data):
    theta and SUGAR at every window, SNR and WMSE (Sec. 4.1) of the
    reconstruction every chunk.  WMSE uses the library's own H^T H operator:
    ||H d||^2 = <d, H^T H d>."""
    import math
    import numpy as np
    import torch
    from synth import fdmc_eps, make_workload
    import paper_1905_08468_gb300 as pkg

    torch.cuda.set_device(0)
    c = make_workload(args.workload)
    eps = fdmc_eps(c.noise_var)
    dev = torch.device("cuda")
    dirty = torch.from_numpy(c.dirty).to(dev)
    delta = torch.from_numpy(c.delta).to(dev)
    sky = torch.from_numpy(c.sky).to(dev)
    plan = pkg.Plan(c.n, c.L, c.psf, sure=True)
    g = torch.empty_like(dirty)
    nl = sky.numel()
    sky_e = float((sky.double() ** 2).sum())

    def metrics(x):
        d = (sky - x).contiguous()
        plan.op_gradient(d, g)
        err = float((d.double() ** 2).sum())
        return 10.0 * math.log10(sky_e / err), float((d.double() * g.double()).sum()) / nl

    inits = [tuple(float(v) for v in t.split(",")) for t in args.conv_inits.split(";")]
    finals = {}
    eta = tuple(float(v) for v in args.conv_eta.split(","))
    runs = []
    t0 = time.perf_counter()
    for th0 in inits:
        x = torch.zeros_like(dirty)
        th, windows, curve, k, warm = th0, [], [], 0, False
        while k < args.conv_iters:
            it = min(args.conv_chunk, args.conv_iters - k)
            th, tr, _ = plan.sure_tune(dirty, delta, c.noise_var, x, th, it, window=args.window,
                                       eta=eta, eps=eps, warm=warm)
            warm = True
            k += it
            windows += tr
            snr, wm = metrics(x)
            curve.append({"k": k, "snr_db": snr, "wmse": wm})
        last = windows[-10:]
        finals[f"x{len(runs)}"] = x.cpu().numpy()
        runs.append({"theta0": list(th0), "theta": list(th),
                     "sugar_last": [float(np.mean([w["sugar_mu"] for w in last])),
                                    float(np.mean([w["sugar_gamma"] for w in last]))],
                     "sugar_first": [windows[0]["sugar_mu"], windows[0]["sugar_gamma"]],
                     "snr_db": curve[-1]["snr_db"], "wmse": curve[-1]["wmse"],
                     "curve": curve,
                     "theta_every": [[w["k"], w["mu"], w["gamma"], w["sugar_mu"], w["sugar_gamma"]]
                                     for w in windows[:: max(1, len(windows) // 50)]]})
    secs = time.perf_counter() - t0
    mus = [r["theta"][0] for r in runs]
    gammas = [r["theta"][1] for r in runs]
    out = {"metric": "ADA-PT convergence from %d initialisations" % len(runs),
           "value": max(mus) / min(mus), "unit": "final mu spread (max/min)",
           "gamma_spread": max(gammas) / min(gammas), "n_gpus": 1, "steps": 1, "warmup": 0,
           "higher_is_better": False, "data": "synthetic", "dtype": "f32",
           "config": {"workload": args.workload, "iters": args.conv_iters,
                      "window": args.window, "eta": list(eta), "eps": eps},
           "seconds": secs, "runs": runs}
    if args.conv_save:
        np.savez(args.conv_save, **finals)
    print(json.dumps(out), flush=True)
    plan.close()


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="muffin", choices=["muffin", "reference"])
    ap.add_argument("--workload", default="c3_1024x1024x64")
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--window", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dictionary", default="daubechies", choices=["daubechies", "iuwt"],
                    help="spatial dictionary W_s (union of 8 Daubechies bases, or the starlet)")
    ap.add_argument("--tuning", default="",
                    help="fixed launch variants 'syn_packed,dct_ctas_per_sm' instead of tuning")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch variants instead of tuning them for the shape")
    ap.add_argument("--serve", action="store_true",
                    help="served Poisson stream (continuous batching vs one cube per launch)")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-iters", type=int, default=300)
    ap.add_argument("--serve-batch", type=int, default=8)
    ap.add_argument("--serve-chunk", type=int, default=10,
                    help="iterations per pool chunk of the server")
    ap.add_argument("--convergence", action="store_true",
                    help="ADA-PT from several initial (mu, gamma): theta, SUGAR, SNR, WMSE curves")
    ap.add_argument("--conv-inits", default="3e-2,1e-1;3e-2,1e-3;3e-4,1e-3;3e-4,1e-1")
    ap.add_argument("--conv-eta", default="1e-6,1e-5")
    ap.add_argument("--conv-iters", type=int, default=5000)
    ap.add_argument("--conv-chunk", type=int, default=250)
    ap.add_argument("--conv-save", default="",
                    help="save the final cube of every start to this .npz (for checks)")
    ap.add_argument("--serve-seed", type=int, default=4,
                    help="arrival-stream seed (request i draws its cube from seed 4000 + i)")
    ap.add_argument("--serve-rate", type=float, default=4.0,
                    help="mean arrivals per second (0: all requests at once)")
    ap.add_argument("--plain", action="store_true",
                    help="plain MUFFIN (Algorithm 2, fixed mu = gamma = --mu) instead of ADA-PT")
    ap.add_argument("--mu", type=float, default=1e-2)
    ap.add_argument("--schedule", default="",
                    help="schedule overrides after tuning, e.g. ana_pipe=0,group_order=1")
    ap.add_argument("--precision", default="tf32", choices=["tf32", "fp32"],
                    help="spectral DCT: 3xTF32 tensor-core products (default) or the FP32 "
                         "fast DCT on the CUDA cores")
    ap.add_argument("--grad-chunk", type=int, default=-1,
                    help="images per pass of the gradient FFTs (-1: the tuner's choice)")
    ap.add_argument("--no-cufft", action="store_true",
                    help="skip the cuFFT timing reference of the gradient")
    ap.add_argument("--cufft-reference", action="store_true",
                    help="cuFFT timing reference of the gradient at 256^2 x 32 and 1024^2 x 64")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.cufft_reference:
        run_cufft_reference(args)
        return
    if args.convergence:
        if args.workload == "c3_1024x1024x64":
            args.workload = "c2_256x256x32"
        run_convergence(args)
        return

    run_gpu(args)


# Algorithmic bytes per chain-voxel that the path must move (the 86 B / 490 B
# floor of one plain chain / the six ADA-PT chains, split by kernel) against
# each kernel's own design bytes (which add the scratch round trips of this
# multi-pass schedule: LL approximations between levels, FFT spectra, the
# gradient image).  achieved = floor-attributable bytes / duration.
ATTRIBUTABLE = {
    # x~, x read; level-1 U details read and written (the LL_1 write is scratch)
    "ana_level1_dual": (56.0, 64.0),
    # level-1 U details, x, t read; x~ written (LL_1 read and the gradient are scratch)
    "syn_level1_prox": (36.0, 48.0),
    # x~, x, v read; v, t written
    "spectral_dual": (20.0, 20.0),
}
FLOOR_BYTES = {"adapt": 490.0, "plain": 86.0}


def attributable_bytes(name: str, design_bytes: float) -> float:
    a = ATTRIBUTABLE.get(name)
    return design_bytes * a[0] / a[1] if a else design_bytes


def cufft_gradient_ms(torch, psf, x, b, reps=10):
    """The gradient H^T H x - b of every image of x ([nimg, n, n], images
    cycling over the PSFs' bands) with cuFFT (torch.fft) and elementwise
    torch kernels: a timing reference for the library's own FFT kernels."""
    nimg, n = x.shape[0], x.shape[-1]
    L = psf.shape[0]
    k = (torch.fft.rfft2(psf.double()).abs() ** 2).float()
    k = k.repeat((nimg + L - 1) // L, 1, 1)[:nimg].contiguous()
    bb = b.repeat((nimg + L - 1) // L, 1, 1)[:nimg].contiguous()

    def once():
        return torch.fft.irfft2(torch.fft.rfft2(x) * k, s=(n, n)) - bb

    for _ in range(3):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def muffin_gradient_ms(stats, nimg_bytes):
    """Average duration of one gradient launch (the three FFT passes) from a
    profiled step: the entries of the per-iteration launches (the most
    frequent of each name)."""
    ent = [s for s in stats if s["name"] == "grad_total"]
    if not ent:
        return None
    e = max(ent, key=lambda s: s["launches"])
    return e["total_ms"] / e["launches"]


def run_cufft_reference(args) -> None:
    """cuFFT timing reference for the gradient at the 256^2 x 32 (plain, one
    chain) and 1024^2 x 64 (ADA-PT groups of three chains) shapes."""
    import numpy as np
    import torch
    from synth import make_workload
    import paper_1905_08468_gb300 as pkg
    torch.cuda.set_device(0)
    rows = []
    for wl, chains in (("c2_256x256x32", 1), ("c3_1024x1024x64", 3)):
        c = make_workload(wl)
        dev = torch.device("cuda")
        psf = torch.from_numpy(c.psf).to(dev)
        dirty = torch.from_numpy(c.dirty).to(dev)
        with pkg.Plan(c.n, c.L, psf, sure=chains == 3) as plan:
            x = torch.zeros_like(dirty)
            plan.profile(True)
            if chains == 3:
                plan.sure_tune(dirty, torch.from_numpy(c.delta).to(dev), c.noise_var, x,
                               THETA0, 20, window=10, eta=(0.0, 0.0),
                               eps=float(np.sqrt(np.mean(c.noise_var))) * 0.1)
            else:
                plan.solve(dirty, x, 20, 1e-2, 1e-2)
            stats = plan.profile_stats()
            plan.profile(False)
        ours = muffin_gradient_ms(stats, None)
        xs = torch.rand((chains * c.L, c.n, c.n), device=dev)
        b = torch.rand((c.L, c.n, c.n), device=dev)
        ref = cufft_gradient_ms(torch, psf, xs, b)
        rows.append({"workload": wl, "images": chains * c.L, "n": c.n,
                     "muffin_ms": ours, "cufft_ms": ref,
                     "speedup_vs_cufft": ref / ours if ours else None})
        del psf, dirty, x, xs, b
        torch.cuda.empty_cache()
    out = {"metric": "gradient H^T(Hx - y) per launch: library FFT kernels vs cuFFT (torch.fft)",
           "value": rows[-1]["speedup_vs_cufft"], "unit": "x (cuFFT time / library time)",
           "n_gpus": 1, "steps": 10, "warmup": 3, "higher_is_better": True,
           "data": "synthetic", "dtype": "f32", "rows": rows}
    print(json.dumps(out), flush=True)


def run_gpu(args) -> None:
    import numpy as np
    import torch
    from synth import fdmc_eps, make_workload
    import paper_1905_08468_gb300 as pkg

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist_init("nccl")
    dev = torch.device("cuda", local_rank)
    mode = "plain" if args.plain else "adapt"
    c = make_workload(args.workload)
    vox = c.voxels
    psf = torch.from_numpy(c.psf).to(dev)
    dirty = torch.from_numpy(c.dirty).to(dev)
    delta = torch.from_numpy(c.delta).to(dev) if mode == "adapt" else None
    x = torch.zeros_like(dirty)
    plan = pkg.Plan(c.n, c.L, psf, sure=mode == "adapt", dictionary=args.dictionary,
                    precision=args.precision)
    del psf
    tuning = None
    if args.tuning:
        sp, dc = (int(v) for v in args.tuning.split(","))
        plan.set_tuning(sp, dc)
        tuning = {"syn_packed": sp, "dct_ctas_per_sm": dc, "candidates": 0}
    elif not args.no_autotune:
        ti = plan.autotune()            # launch variants for this shape (results unchanged)
        tuning = {"syn_packed": ti.syn_packed, "dct_ctas_per_sm": ti.dct_ctas_per_sm,
                  "spectral_tcgen05": ti.spectral_tcgen05,
                  "candidates": ti.candidates, "iter_ms_default": ti.ms_default,
                  "iter_ms_tuned": ti.ms_best}
    if args.grad_chunk >= 0:
        plan.set_schedule(grad_chunk=args.grad_chunk)
    if args.schedule:
        plan.set_schedule(**{k: int(v) for k, v in
                             (kv.split("=") for kv in args.schedule.split(","))})
    if tuning is not None:
        tuning["schedule"] = plan.schedule()
    if mode == "adapt":
        eps = fdmc_eps(c.noise_var)
        kw = dict(window=args.window, eta=ETA, eps=eps)

        def step(xb, d, dl):
            th, _, _ = plan.sure_tune(d, dl, c.noise_var, xb, THETA0, args.iters, **kw)
            return th
    else:
        def step(xb, d, dl):
            plan.solve(d, xb, args.iters, args.mu, args.mu)
            return (args.mu, args.mu)

    for _ in range(args.warmup):
        x.zero_()
        step(x, dirty, delta)
    torch.cuda.synchronize()

    # ---- device-resident timed region (captured graphs, no per-launch events)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        x.zero_()
        theta = step(x, dirty, delta)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, dev)
    secs = ms / 1e3
    value = job_value(vox * args.iters * args.steps, world, secs)

    # ---- one more step with CUDA events around every launch (on the plan's
    # stream): per-kernel durations, shares and the launch count of a step
    plan.profile(True)
    x.zero_()
    torch.cuda.synchronize()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record()
    step(x, dirty, delta)
    pe1.record()
    torch.cuda.synchronize()
    profiled_ms = pe0.elapsed_time(pe1)
    stats = plan.profile_stats()
    plan.profile(False)
    # "grad_total" brackets the gradient's launches (an aggregate, not a kernel)
    stats = [s for s in stats if s["name"] != "grad_total"] + \
        [dict(s, aggregate=True) for s in stats if s["name"] == "grad_total"]
    kstats = [s for s in stats if not s.get("aggregate")]
    launches = sum(s["launches"] for s in kstats) * args.steps
    dom = max(kstats, key=lambda s: s["total_ms"])
    tot_ms = sum(s["total_ms"] for s in kstats)
    avg_ms = dom["total_ms"] / dom["launches"]
    peak, peak_kind = measured_peak_gbs()
    attr = attributable_bytes(dom["name"], dom["bytes_per_launch"])
    achieved = attr / (avg_ms / 1e3) / 1e9
    chains = 3.0 if mode == "adapt" else 1.0
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": captured_traffic(dom["name"], chains * vox),
                "bytes_per_launch": attr, "design_bytes_per_launch": dom["bytes_per_launch"],
                "avg_launch_ms": avg_ms, "share": dom["total_ms"] / tot_ms,
                "timing": "CUDA events around each launch on the plan's stream, one "
                          "profiled step after the timed region"}
    floor = FLOOR_BYTES[mode]
    iteration_roofline = {"floor_bytes_per_voxel_iter": floor,
                          "achieved_GBps": floor * value / 1e9,
                          "frac": floor * value / 1e9 / peak}
    kernels = sorted(({"name": s["name"], "launches": s["launches"],
                       "ms": round(s["total_ms"], 3),
                       "share": round(s["total_ms"] / tot_ms, 4),
                       "GBps_design": round(s["bytes_per_launch"] * s["launches"] /
                                            (s["total_ms"] / 1e3) / 1e9, 1) if s["total_ms"] else None,
                       "GBps_attributable": round(attributable_bytes(s["name"], s["bytes_per_launch"])
                                                  * s["launches"] / (s["total_ms"] / 1e3) / 1e9, 1)
                       if s["total_ms"] else None}
                      for s in kstats), key=lambda s: -s["ms"])

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        hd = torch.from_numpy(c.dirty).pin_memory()
        hdl = torch.from_numpy(c.delta).pin_memory() if mode == "adapt" else None
        hx = torch.zeros(c.dirty.shape, dtype=torch.float32).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            hx.zero_()
            step(hx, hd, hdl)
        torch.cuda.synchronize()
        barrier()
        es = max_over_ranks(time.perf_counter() - t0, dev)
        nbytes = c.dirty.nbytes
        e2e = {"value": job_value(vox * args.iters * args.e2e_steps, world, es),
               "unit": UNIT, "h2d_bytes_per_step": (3 if mode == "adapt" else 2) * nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps}

    cufft = None
    if mode == "adapt" and rank == 0 and not args.no_cufft:
        ours = muffin_gradient_ms(stats, None)
        xs = torch.rand((3 * c.L, c.n, c.n), device=dev)
        ref = cufft_gradient_ms(torch, torch.from_numpy(c.psf).to(dev), xs, dirty)
        cufft = {"images": 3 * c.L, "n": c.n, "muffin_gradient_ms": ours,
                 "cufft_gradient_ms": ref, "speedup_vs_cufft": ref / ours if ours else None}
        del xs

    cpu = cpu1 = None
    if mode == "adapt" and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_obj(oracle_sample(args.workload, parallel=True, cube=c))
        cpu1 = cpu_baseline_obj(oracle_sample(args.workload, parallel=False, cube=c))

    if rank == 0:
        metric = METRIC if mode == "adapt" else \
            f"voxel-iters/s (px x bands x iters) at {c.n}^2 x {c.L}, plain MUFFIN (Algorithm 2)"
        out = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": dict(workload_config(args), tuning=tuning),
               "roofline": roofline, "iteration_roofline": iteration_roofline,
               "cpu_baseline": cpu, "cpu_baseline_1core": cpu1, "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks,
               "theta": list(theta), "kernels": kernels,
               "iter_ms": ms / args.steps / args.iters,
               "profiled_step_ms": profiled_ms, "cufft_reference": cufft}
        print(json.dumps(out), flush=True)
    plan.close()


if __name__ == "__main__":
    main()
