"""The search phase launched from a CUDA graph (vc_options.cuda_graph).

The graph is captured on the second call in a row with one launch shape and
replayed on later calls with that shape; the queries, the graphs and the
bounds behind its buffers are read when it runs.  Every answer must equal the
oracle's and the one of kernel-by-kernel launches, on capture, on replay and
when the data changes between replays; covers are verified edge by edge.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_18334_gb300 import build
    build.build()
    import paper_2512_18334_gb300 as m
    return m


def opt_of(g):
    return oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]


def check_cover(g, cover, bound):
    flags = np.zeros(max(g.n, 1), np.uint8)
    flags[cover] = 1
    assert len(np.unique(cover)) == len(cover) <= bound
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags[:g.n])


def searched_graph(vc):
    # a graph the root phase leaves to the search, so that there is a search phase
    for s in range(20):
        g = gg.gnm(80, 200, 100 + s)
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        _, _, st = vc.solve_min(dg, cuda_graph=0)
        if st["n_induced"] > 0 and st["nodes"] > 0:
            return g, dg
        dg.close()
    pytest.skip("no searched graph among the seeds")


def test_repeated_solves_replay_one_graph(vc):
    g, dg = searched_graph(vc)
    opt = opt_of(g)
    vc.trim()   # no workspace (and no graph) is left from earlier tests
    states = []
    for _ in range(4):
        size, cover, st = vc.solve_min(dg)
        assert size == opt
        check_cover(g, cover, opt)
        assert st["nodes"] > 0 and st["ms_search"] > 0.0   # the events inside the graph were recorded
        states.append(st["cuda_graph"])
    assert states == [0, 1, 2, 2]   # direct, captured, replayed, replayed
    size, cover, st = vc.solve_min(dg, cuda_graph=0)
    assert size == opt and st["cuda_graph"] == 0
    check_cover(g, cover, opt)
    dg.close()


def test_replay_reads_the_current_queries(vc):
    # the same graph twice with its decision bounds swapped between calls:
    # the launch shape is unchanged, the answers are not
    g, dg = searched_graph(vc)
    opt = opt_of(g)
    plans = [[opt, opt - 1], [opt - 1, opt], [-1, opt - 1], [opt - 1, -1], [-1, -1]]
    for ks in plans * 3:
        sizes, yes, status, covers, st = vc.solve_batch([dg, dg], ks)
        assert list(status) == [vc.VC_OK, vc.VC_OK]
        for i, k in enumerate(ks):
            if k < 0:
                assert sizes[i] == opt and yes[i]
                check_cover(g, covers[i], opt)
            elif k >= opt:
                assert yes[i]
                check_cover(g, covers[i], k)
            else:
                assert not yes[i] and len(covers[i]) == 0
    dg.close()


def test_batches_match_direct_launches(vc):
    gs = [gg.gnm(80, 200, s) for s in range(6)]
    gs += [gg.component_heavy(3, copies=4, copy_n=24, p=0.2, chain=2), gg.chung_lu(600, 2.5, 4.0, 100.0, 5)]
    opts = [opt_of(g) for g in gs]
    dgs = [vc.Graph.from_csr(g.row_ptr, g.col) for g in gs]
    seen = set()
    for rep in range(3):
        for flag in (1, 0):
            sizes, yes, status, covers, st = vc.solve_batch(dgs, cuda_graph=flag)
            assert list(sizes) == opts and all(status == vc.VC_OK)
            for g, c, o in zip(gs, covers, opts):
                check_cover(g, c, o)
            if flag == 0:
                assert st["cuda_graph"] == 0
            else:
                seen.add(st["cuda_graph"])
    assert 2 in seen
    for d in dgs:
        d.close()


@pytest.mark.parametrize("big", [False, True])
def test_root_phase_replayed_with_new_descriptors(vc, big):
    # The root phase is one graph launch once a shape (query count, largest
    # n and degree) comes twice in a row.  Relabelled copies share the shape
    # but not the CSR, and the decision bound changes between calls: each
    # replay must read the descriptors of its own call.  big: n >= 8192, the
    # root phase on a thread-block cluster.
    if big:
        parts = [gg.random_forest(9000, 40, 3)] + [gg.gnm(40, 90, s) for s in range(12)]
        base = gg.disjoint_union(parts)
        want = sum(oracle.mvc(p.n, p.row_ptr, p.col)[0] for p in parts)
    else:
        base = gg.chung_lu(3000, 2.5, 6.0, 300.0, 9)
        want = opt_of(base)
    gs = [base, gg.relabel(base, 1), gg.relabel(base, 2)]
    dgs = [vc.Graph.from_csr(g.row_ptr, g.col) for g in gs]
    try:
        for rep in range(3):
            for g, dg in zip(gs, dgs):
                size, cover, _ = vc.solve_min(dg)
                assert size == want
                check_cover(g, cover, size)
                yes, cover, _ = vc.solve_k(dg, want)
                assert yes
                check_cover(g, cover, want)
                assert not vc.solve_k(dg, want - 1)[0]
        # the same calls launched kernel by kernel agree
        assert vc.solve_min(dgs[0], cuda_graph=0)[0] == want
    finally:
        for dg in dgs:
            dg.close()
