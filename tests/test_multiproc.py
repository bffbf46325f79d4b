"""The N > 1 bench path on CPU: world-size-2 gloo process groups.

The GPU arm runs one independent replica per rank (its own seeded box, no
data-path collective) and combines the ranks only through the barrier and the
max-over-ranks time; those host steps are exercised here with gloo.  The
reference arm (the float64 oracle) is launched under torchrun exactly as for a
multi-GPU run: rank 0 prints the one JSON line, the other rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    w, r, local = bench.dist_setup(argparse.Namespace(impl="reference"))
    local_ms = [120.0, 150.0][r]                      # rank 1 is the slower replica
    bench.barrier(w)
    ms_max = bench.max_over_ranks(local_ms, w)
    bench.barrier(w)
    q.put(dict(rank=r, world=w, local=local, ms_max=ms_max, seed=bench.replica_seed(r),
               value=bench.whole_job_ms_per_solve(ms_max, 5, w)))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_replicas_combine_by_max_over_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [d["world"] for d in out] == [2, 2]
    assert [d["ms_max"] for d in out] == [150.0, 150.0]       # both ranks see the slowest replica
    assert [d["seed"] for d in out] == [0, 1]                 # independent particle sets
    assert out[0]["value"] == pytest.approx(150.0 / (5 * 2))  # 10 solves in 150 ms


def test_reference_arm_under_torchrun_world_2():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--box-side", "8"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
