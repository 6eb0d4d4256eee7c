"""The CPU baselines the bench reports beside the GPU numbers: the oracle over
every host core (a thread per core; the oracle is reentrant) must give the
same answers as the single-threaded oracle, count budget overruns, and stop
taking new work once its time bound has passed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


def test_all_cores_oracle_runs_every_job():
    gs = [gg.gnm(40, 80, s) for s in range(24)]
    r = bench.cpu_oracle_all_cores([(g, -1) for g in gs])
    assert r["jobs"] == r["of"] == 24 and r["over_budget"] == 0
    assert r["cores"] == (os.cpu_count() or 1) and r["per_s"] > 0


def test_threads_give_the_single_threaded_answers():
    # the same oracle calls from many threads at once: reentrant C, no shared state
    import concurrent.futures as cf
    gs = [gg.gnm(60, 130, 100 + s) for s in range(32)]
    want = [oracle.mvc(g.n, g.row_ptr, g.col)[0] for g in gs]
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        got = list(ex.map(lambda g: oracle.mvc(g.n, g.row_ptr, g.col)[0], gs))
    assert got == want


def test_budget_overruns_are_counted_and_time_bound_stops_early():
    hard = gg.gnm(200, 700, 3)            # far beyond 50 search-tree nodes
    easy = gg.path(10)
    jobs = [(hard, -1)] * 4 + [(easy, 5)] * 4
    r = bench.cpu_oracle_all_cores(jobs, budget=50)
    assert r["jobs"] == 8 and r["over_budget"] == 4
    many = [(easy, -1)] * 10_000
    r = bench.cpu_oracle_all_cores(many, max_s=0.0)   # one wave, then the bound stops it
    assert r["jobs"] == min(10_000, os.cpu_count() or 1)


def test_host_cpu_reports_cores_and_model():
    h = bench.host_cpu()
    assert h["nproc"] == (os.cpu_count() or 1) and isinstance(h["model"], str) and h["model"]
