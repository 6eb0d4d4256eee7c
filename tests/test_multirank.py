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
