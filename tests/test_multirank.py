"""The N > 1 bench path on CPU: replicas combined over two gloo ranks (the
timed region is the slowest rank's, the value counts every rank's graphs),
and the reference arm printing on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 80.0][rank]          # rank 0 is the slow one
    got = bench.combine_over_ranks(local_ms, steps=10, world=world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_replicas_take_the_slowest_rank_and_count_every_graph():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        max_ms, value = res[r]
        assert max_ms == 120.0
        assert value == pytest.approx(2 * 10 / 0.120)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.combine_over_ranks(50.0, 5, 1) == (50.0, 5 / 0.05)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    monkeypatch.setattr(bench, "cpu_oracle_run", lambda steps, warmup: (0.5, 2000.0, 123))
    out = io.StringIO()
    with redirect_stdout(out):
        bench.reference_main(Args, rank=1, world=2)
    assert out.getvalue() == ""
    with redirect_stdout(out):
        bench.reference_main(Args, rank=0, world=2)
    line = out.getvalue().strip()
    assert line.count("\\n") == 0 and '"impl": "reference"' in line and '"n_gpus": 2' in line


def test_batch_shards_cover_every_graph_once_and_balance():
    import bench
    rng = __import__("numpy").random.default_rng(4)
    costs = rng.integers(40, 1500, size=4096).tolist()
    for world in (1, 2, 3, 8):
        parts = bench.shard_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: no rank carries more than the average plus the largest item
        assert max(loads) <= sum(costs) / world + max(costs)


def _search_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = {"queries": [100, 60][rank], "nodes": [5000, 7000][rank], "ms_wall": [30.0, 45.0][rank],
             "ms_kernel": [25.0, 40.0][rank], "wrong": 0, "over": rank, "bytes": 1000 * (rank + 1)}
    out = bench.combine_search(local, world, group=bench.host_group())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_sharded_search_results_gather_on_the_host():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_search_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        out = res[r]
        assert out["queries"] == 160 and out["nodes"] == 12000 and out["over"] == 1 and out["bytes"] == 3000
        assert out["ms_wall"] == 45.0 and out["ms_kernel"] == 40.0
        assert out["per_rank_queries"] == [100, 60]


def test_main_with_two_gpus_starts_two_ranks():
    # `bench.py --gpus 2` without a launcher starts two ranks itself (under
    # torchrun, gloo-free here: the reference arm needs no process group);
    # rank 0 prints the single JSON line for both
    import json
    import subprocess
    pytest.importorskip("torch")
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["config"]["answer"] == 21258
