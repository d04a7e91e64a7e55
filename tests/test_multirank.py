"""The N > 1 path of bench.py on the CPU: two gloo ranks (replicas only, no
collective on the data path).  Checked: the timed durations are reduced to
the slowest rank's on every rank, the whole-job rate counts every rank's
units, and the reference arm runs on rank 0 alone."""
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
import torch.distributed as dist
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]),
                        world_size=int(os.environ["WORLD_SIZE"]))
r = dist.get_rank()
mine = [10.0 + r, 3.0 - r]           # rank 1 is slower on the first, faster on the second
got = bench.max_over_ranks(mine, dist, device="cpu")
rate = bench.whole_job_rate(1000, dist.get_world_size(), got[0])
dist.barrier()
print(json.dumps({{"rank": r, "max": got, "rate": rate}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code, world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    outs = _launch(WORKER.format(root=ROOT), 2)
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["max"] == [11.0, 3.0]            # the slowest rank's time, everywhere
        assert d["rate"] == pytest.approx(2 * 1000 / 11.0)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    # the oracle arm of a small workload under two ranks: rank 1 exits 0
    # without work or output, rank 0 prints one JSON line
    env_common = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    outs = []
    for r in (1, 0):
        env = dict(env_common, RANK=str(r), LOCAL_RANK=str(r))
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                            "reference", "--workload", "c1", "--steps", "3", "--warmup", "3",
                            "--gpus", "2"], env=env, capture_output=True, text=True,
                           timeout=300, cwd=ROOT)
        assert p.returncode == 0, p.stderr
        outs.append(p.stdout.strip())
    assert outs[0] == ""
    line = json.loads(outs[1].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    # the reference line describes its own run: the oracle on the host cores,
    # the same metric as the GPU arm, no host-device copies
    assert line["metric"] == "coupled-LB MLUPS" and line["unit"] == "MLUPS"
    assert line["higher_is_better"] is True and line["steps"] == 3 and line["warmup"] == 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
