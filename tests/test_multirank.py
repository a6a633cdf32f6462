"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Walkers shard across ranks with no data-path collective; the only exchange
is the timing maximum over ranks (and a barrier).  These tests run that
logic in two CPU processes, and the reference arm under torch.distributed.run
(rank 0 measures and prints one JSON line, the other rank exits cleanly).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    got = bench.ranks_max([1.0 + rank, 10.0 - rank, 0.5 * rank], world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got))


def test_ranks_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 0.5]


def test_ranks_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max([3.0, 4.0], 1) == [3.0, 4.0]


def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "heg3d_sc_n54"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                      # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype", "data"):
        assert key in d, key
    # the reference arm names the same configuration as the GPU arm: the
    # workload's sizes and parameters, built by the one function both use
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from paper_2507_02888_gb300 import inputs
    args = argparse.Namespace(workload="heg3d_sc_n54", moves=4)
    assert d["config"] == bench.workload_config(args, inputs.workload("heg3d_sc_n54"), 2)
