"""The multi-process path of bench.py on CPU: two ranks over gloo.

A lattice is not sharded: N GPUs run N replicas of the same gauge fixing, with
a barrier on both sides of the timed region and the maximum of the ranks'
times.  These tests run the host side of that path (process-group setup,
barrier, max over ranks, rank-0-only output of the reference arm) as two
CPU processes; the GPU work itself is not involved.
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, local = bench.dist_setup(world)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    mx = bench.max_over_ranks(1.5 * (rank + 1), w)
    bench.barrier(w)
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "max": mx}, f)
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [g["rank"] for g in got] == [0, 1]
    assert all(g["world"] == 2 for g in got)
    # every rank reports the slowest rank's time
    assert all(g["max"] == pytest.approx(3.0) for g in got)


def test_reference_arm_prints_on_rank_zero_only(tmp_path, monkeypatch):
    """Rank 1 of the reference arm returns without work or output."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 0

    printed = []
    monkeypatch.setattr("builtins.print", lambda *a, **k: printed.append(a))
    bench.reference_arm(Args(), rank=1, world=2)
    assert printed == []


def test_torchrun_two_ranks_reference_arm_single_line(tmp_path):
    """bench.py --impl reference under torchrun with two CPU ranks: one JSON
    line, from rank 0, and both ranks exit 0 (small lattice for speed)."""
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2",
           "--warmup", "1", "--dims", "4", "4", "4", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=str(tmp_path), env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the reference arm reports on the GPU arm's metric, unit and workload
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == "site-updates/s" and d["higher_is_better"]
    ref = bench.headline_config(2)
    assert {k: v for k, v in d["config"].items() if k not in ("workload", "lattice")} == \
        {k: v for k, v in ref.items() if k not in ("workload", "lattice")}
    assert d["config"]["lattice"] == [4, 4, 4, 4]
