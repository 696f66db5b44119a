"""Host-side logic of bench.py: the multi-rank timing reduction (gloo,
world size 2 on CPU), whole-job throughput, clock-sample parsing and the
reference arm's rank handling."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    bench.dist_init("gloo")
    bench.barrier()
    m = bench.max_over_ranks(10.0 + 5.0 * rank)
    v = bench.job_value(100.0, world, m)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]            # slowest rank's time
    assert all(abs(r[2] - 100.0 * 2 / 15.0) < 1e-12 for r in res)


def test_job_value_single_rank():
    assert bench.job_value(3e9, 1, 1.5) == 2e9


def test_parse_clocks():
    text = ("0, 1980, 2070, 900.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
            "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1995, 2070, 940.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.parse_clocks(text)
    assert c["sm_mhz"] == 1995 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.parse_clocks("")["sm_mhz"] is None


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_minimum_enforced():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "1"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "warmup" in r.stderr
