"""Host logic of bench.py's multi-rank path (no GPU): two gloo ranks on the CPU.  Each rank
runs its own replica of the batched workload (problems are independent, no data-path
collective); the step time is the maximum over the ranks, and only rank 0 reports."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
rank = dist.get_rank()
t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
single = bench.max_over_ranks(3.5)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "max": t, "single": single}))
"""


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_step_time_is_the_maximum_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["max"] == 15.0 for o in outs)
    assert all(o["single"] == 3.5 for o in outs)


def test_reference_arm_other_ranks_exit_without_output():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=240)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_json_line_on_rank_0():
    """The reference arm (the FP64 oracle on the host cores) prints one JSON line with the
    same metric and config as the GPU arm, marked "impl": "reference", with its own
    cpu_baseline and an e2e that moves no bytes."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--cpu-sample-s", "1"], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["unit"] == "s" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("batched")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the value is extrapolated from the sample, and says so; a step is one bounded sample,
    # so the timed region (steps x ms_per_step) is what the run actually spent
    assert d["extrapolated"] is True and cb["extrapolated"] is True
    assert d["sampled_grid_point_steps"] > 0 and d["sample_wall_s"] > 0
    assert d["ms_per_step"] * d["steps"] / 1e3 <= 10 * 60
    assert d["ms_per_step"] / 1e3 == pytest.approx(d["sample_wall_s"], rel=1e-6)
