"""The synthetic input recipes stand in for the paper's datasets; these checks
pin each recipe to its stated shape (sizes, degree targets, structure), so a
drift in a generator shows up here and not as a silent change of workload."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402


def _simple(g):
    u, v = gg.edges_of(g)
    assert np.all(u < v) and np.all(v < g.n)            # no loops, ids in range
    keys = u.astype(np.int64) * g.n + v
    assert np.unique(keys).size == keys.size             # no repeated pairs
    rp, c = g.row_ptr, g.col
    for x in range(g.n):
        row = c[rp[x]:rp[x + 1]]
        assert np.all(np.diff(row) > 0)                  # rows sorted ascending
    return u, v


def test_chung_lu_ids_are_shuffled_and_degree_capped():
    g = gg.chung_lu(20_000, 2.5, 6.0, 800.0, 4)
    _simple(g)
    d = g.degrees().astype(np.float64)
    assert 5.0 < d.mean() < 6.5 and d.max() <= 1.05 * 800
    # degree does not follow the vertex index (ids are permuted)
    idx = np.arange(g.n, dtype=np.float64)
    assert abs(np.corrcoef(idx, d)[0, 1]) < 0.05
    # heavy tail: the largest degree is far above the mean
    assert d.max() > 20 * d.mean()


def test_component_heavy_structure():
    copies, copy_n, chain = 12, 20, 6
    g = gg.component_heavy(3, copies=copies, copy_n=copy_n, p=0.15, chain=chain)
    assert g.n == chain + copies * copy_n
    u, v = _simple(g)
    pairs = set(zip(u.tolist(), v.tolist()))
    assert all((i, i + 1) in pairs for i in range(chain - 1))      # the chain is a path
    for k in range(copies):
        lo, hi = chain + k * copy_n, chain + (k + 1) * copy_n
        inside_u = (u >= lo) & (u < hi)
        inside_v = (v >= lo) & (v < hi)
        # edges leave a copy only towards the chain, through 1 to 3 bridges
        assert not np.any(inside_u & ~inside_v & (v >= chain))
        assert not np.any(inside_v & ~inside_u & (u >= chain))
        bridges = np.sum((inside_u & (v < chain)) | (inside_v & (u < chain)))
        assert 1 <= bridges <= 3


def test_batch_mix_sizes_and_halves():
    gs = gg.batch_pvc_mix(40, 11, n_lo=40, n_hi=400)
    assert len(gs) == 40
    for i, g in enumerate(gs):
        assert 40 <= g.n <= 400
        _simple(g)
        assert ("gnp" in g.name) == (i % 2 == 0) and ("chung_lu" in g.name) == (i % 2 == 1)


def test_stream_arrivals_and_sizes():
    rate = 500.0
    t, specs = gg.stream_requests(4000, 5, rate)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    mean_gap = t[-1] / (len(t) - 1)
    assert abs(mean_gap - 1.0 / rate) < 0.1 / rate          # Poisson arrivals at the rate
    ns = np.array([s[0] for s in specs], dtype=np.float64)
    assert ns.min() >= 30 and ns.max() <= 20000
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(math.log(np.median(ns)) - 0.5 * (math.log(30) + math.log(20000))) < 0.3
    assert all(2.2 <= s[1] <= 3.0 and 4.0 <= s[2] <= 10.0 for s in specs)


def test_gnp_sparse_unranking_covers_the_pair_space():
    # every pair index maps to a distinct valid pair: a dense draw hits them all
    g = gg.gnp_sparse(30, 1.0, 0)
    assert g.m == 30 * 29 // 2
    _simple(g)
