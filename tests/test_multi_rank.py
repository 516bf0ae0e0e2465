"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as torchrun launches
them) run independent replicas with their own seeds; the job time is the slowest rank's
(element-wise maximum over ranks); the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as tdist
import bench
rank, world, local = bench.dist_env()
tdist.init_process_group("gloo")
tdist.barrier()
times = bench.max_over_ranks([10.0 + rank, 5.0 - rank, float(rank)], world, "cpu")
seeds = bench.graph_seeds(rank)
tdist.barrier()
print(json.dumps({"rank": rank, "world": world, "times": times, "seeds": seeds}), flush=True)
tdist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code: str, world: int, extra_env=None, args=()):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT)
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code, *args], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_rank_and_own_seeds():
    pytest.importorskip("torch")
    outs = _launch(RANK_SCRIPT, 2)
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for ln in lines:
        assert ln["world"] == 2
        assert ln["times"] == [11.0, 5.0, 1.0]  # element-wise max over ranks 0 and 1
    s0, s1 = sorted(lines, key=lambda x: x["rank"])
    assert s0["seeds"] != s1["seeds"]  # independent replicas
    assert [p for p, _ in s0["seeds"]] == [p for p, _ in s1["seeds"]]


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under two ranks: rank 0 times the oracle on its graphs and
    prints the line, rank 1 exits 0 at once without output."""
    pytest.importorskip("torch")
    code = r"""
import os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import bench
rank, world, local = bench.dist_env()
class A: steps = 1; warmup = 0
bench.run_reference(A(), rank, world)
print("done", flush=True)
"""
    outs = _launch(code, 2)
    assert outs[1].strip() == "done"
    line = json.loads(outs[0].strip().splitlines()[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
