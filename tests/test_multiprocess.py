"""The N>1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

bench.py runs one independent replica of the step per rank (no data-path
collective); ranks meet only at the timing barriers and in the max over
ranks of the step time.  These tests run those helpers as two real
processes, and check that the reference arm prints from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_env()
dist = bench.init_dist(world, "gloo")
bench.barrier(dist)
t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
value = bench.job_value(world, 1000, 4, t)
bench.barrier(dist)
print(json.dumps({{"rank": rank, "max": t, "value": value, "seed_base": bench.replica_seed_base(rank)}}))
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ)
    env.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    return env


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    code = WORKER.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=240) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    recs = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda r: r["rank"])
    assert [r["max"] for r in recs] == [15.0, 15.0]
    # whole-job value: all ranks' packages over the slowest rank's time
    assert recs[0]["value"] == pytest.approx(2 * 1000 * 4 / 15e-3)
    assert recs[0]["value"] == recs[1]["value"]
    assert recs[0]["seed_base"] != recs[1]["seed_base"]


def test_reference_arm_prints_from_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--ref-seconds", "0.3"]
    r1 = subprocess.run(cmd, env=_env(1, 2, port), capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr[-2000:]
    assert r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, env=_env(0, 2, port), capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0, r0.stderr[-2000:]
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
