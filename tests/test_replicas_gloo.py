"""The multi-GPU form is replicas only (streams are independent: no data-path
collective).  Its host logic is checked here on CPU with world-size-2 `gloo`
ranks, started the way torchrun starts them (RANK / WORLD_SIZE / MASTER_* in
the environment, rendezvous on 127.0.0.1):

* bench.py's timing is the slowest rank's (max over ranks, on every rank) and
  its value counts every rank's streams;
* each rank draws its own stream seeds and inputs (replicas, not copies);
* a torchrun launch of the reference arm prints exactly one line, from rank 0,
  and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch
import torch.distributed as dist
import bench
from paper_2204_07064_gb300 import workloads as W
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = 10.0 * (rank + 1) + 0.25
got = bench.max_over_ranks(ms, dist, torch.device("cpu"))
value = bench.whole_job_streams(256, world, 100, 2048, got)
seeds = W.stream_seeds(1000 + rank, 4)
# the seeds of every rank, to check that replicas draw different streams
gathered = [None] * world
dist.all_gather_object(gathered, seeds)
dist.barrier()
print(json.dumps({{"rank": rank, "world": world, "max": got, "value": value, "seeds": gathered}}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_max_over_ranks_and_whole_job_value_gloo():
    world, port = 2, _free_port()
    code = RANK_CODE.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, world, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(world)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r, d in enumerate(outs):
        assert d["rank"] == r and d["world"] == world
        assert d["max"] == 20.25  # the slowest rank's time, on every rank
        assert abs(d["value"] - 256 * 2 * 2048 * 100 / 0.02025 / 48000) < 1e-6
    seeds = outs[0]["seeds"]
    assert seeds == outs[1]["seeds"] and not set(seeds[0]) & set(seeds[1])


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert abs(bench.whole_job_streams(256, 1, 10, 2048, 1000.0) - 256 * 2048 * 10 / 48000) < 1e-9


def test_torchrun_reference_arm_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
