"""The paper's optimisations switched off one at a time (its ablation of
components, root reduction with the induced subgraph, non-zero bounds and
load balancing) must leave every answer unchanged; the execution-time
breakdown and the maximum-independent-set wrapper are checked here too."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

SWITCHES = [dict(disable_bounds=1), dict(disable_root_rules=1), dict(use_components=0), dict(load_balance=0),
            dict(disable_dyn_bounds=1), dict(label_propagation=1), dict(label_propagation=1, team=32),
            dict(disable_bounds=1, disable_root_rules=1), dict(disable_bounds=1, team=256),
            dict(disable_root_rules=1, team=32)]


@pytest.fixture(scope="module")
def vc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_18334_gb300 import build
    build.build()
    import paper_2512_18334_gb300 as m
    return m


def check_cover(g, cover, size):
    flags = np.zeros(max(g.n, 1), np.uint8)
    flags[cover] = 1
    assert len(cover) == size and len(np.unique(cover)) == size
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags[:g.n])


def graphs():
    gs = [gg.gnm(80, 200, s) for s in range(4)]
    gs += [gg.chung_lu(600, 2.5, 4.0, 100.0, 3), gg.component_heavy(2, copies=4, copy_n=24, p=0.2, chain=2),
           gg.random_forest(1500, 4, 2), gg.disjoint_union([gg.cycle(7), gg.complete(5), gg.petersen()])]
    return gs


@pytest.mark.parametrize("sw", SWITCHES, ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_switches_leave_answers_unchanged(vc, sw):
    for g in graphs():
        want = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        size, cover, st = vc.solve_min(dg, **sw)
        check_cover(g, cover, size)
        assert size == want, (g.name, sw)
        yes, cover2, _ = vc.solve_k(dg, want, **sw)
        assert yes
        check_cover(g, cover2, len(cover2))
        assert not vc.solve_k(dg, want - 1, **sw)[0]
        dg.close()


def test_root_rules_off_on_the_cluster_path(vc):
    # n >= 8192: the root phase runs on a thread-block cluster; without its
    # rules the search starts from all 12,000 vertices
    parts = [gg.gnm(40, 90, s) for s in range(300)]
    g = gg.disjoint_union(parts)
    want = sum(oracle.mvc(p.n, p.row_ptr, p.col)[0] for p in parts)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, cover, st = vc.solve_min(dg, disable_root_rules=1)
    _, _, st_on = vc.solve_min(dg)
    dg.close()
    assert size == want
    check_cover(g, cover, size)
    with_edges = int(np.count_nonzero(np.diff(g.row_ptr)))
    assert st["forced"] == 0 and st["n_induced"] == with_edges
    assert st_on["n_induced"] < g.n


def test_bounds_off_keeps_the_whole_array(vc):
    g = gg.component_heavy(3, copies=4, copy_n=24, p=0.2, chain=2)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    s_on, _, st_on = vc.solve_min(dg)
    s_off, _, st_off = vc.solve_min(dg, disable_bounds=1)
    dg.close()
    assert s_on == s_off
    # the same slots carry the whole array: more bytes per node
    assert st_off["search_bytes"] / st_off["nodes"] > st_on["search_bytes"] / st_on["nodes"]


def test_breakdown_counts_every_activity(vc):
    g = gg.component_heavy(1, copies=4, copy_n=32, p=0.15, chain=2)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, _, st = vc.solve_min(dg, breakdown=1)
    plain, _, st0 = vc.solve_min(dg)
    dg.close()
    assert size == plain
    ph = st["phase_cycles"]
    assert ph["reduce"] > 0 and ph["pop"] > 0 and ph["branch"] > 0 and ph["components"] > 0
    assert all(v >= 0 for v in ph.values())
    assert sum(st0["phase_cycles"].values()) == 0          # off unless asked for


def test_maximum_independent_set(vc):
    rng = np.random.default_rng(5)
    cases = [gg.gnp(int(rng.integers(8, 21)), 0.3, s) for s in range(20)]
    cases += [gg.petersen(), gg.cycle(9), gg.complete(6), gg.star(30), gg.from_edges(4, [], []),
              gg.gnm(80, 200, 9), gg.component_heavy(1, copies=4, copy_n=24, p=0.2, chain=2)]
    for g in cases:
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        size, iset, _ = vc.solve_mis(dg)
        dg.close()
        opt = oracle.brute_mvc(g.n, g.row_ptr, g.col)[0] if g.n <= 22 else \
            oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
        assert size == g.n - opt
        assert len(iset) == size and np.all(np.diff(iset) > 0)
        inside = np.zeros(max(g.n, 1), bool)
        inside[iset] = True
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        assert not np.any(inside[src] & inside[g.col])      # no edge inside the set


def test_autotuner_picks_a_working_configuration(vc):
    gs = [gg.gnm(80, 200, s) for s in range(16)] + [gg.component_heavy(1, copies=4, copy_n=24, p=0.2, chain=2)]
    dgs = [vc.Graph.from_csr(g.row_ptr, g.col) for g in gs]
    best, best_ms, table = vc.autotune(dgs, repeats=1)
    assert best_ms > 0 and len(table) >= 5
    assert best_ms <= table[0][1] + 1e-9            # never worse than where it started
    sizes, _, status, covers, _ = vc.solve_batch(dgs, opts=best)
    for g, s, st, cov in zip(gs, sizes, status, covers):
        assert st == 0 and s == oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
        check_cover(g, cov, s)
    for d in dgs:
        d.close()


def crown_graphs():
    gs = graphs()
    gs += [gg.random_bipartite_chung_lu(300, 200, 2.5, 3.0, 50.0, s) for s in range(3)]
    gs += [gg.complete_bipartite(5, 9), gg.star(40), gg.cycle(11), gg.complete(7), gg.petersen()]
    return gs


def test_crown_reduction_keeps_answers(vc):
    for g in crown_graphs():
        want = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        size, cover, st = vc.solve_min(dg, crown=1)
        assert st["crown_skipped"] == 0, g.name
        assert size == want, g.name
        check_cover(g, cover, size)
        yes, cover2, _ = vc.solve_k(dg, want, crown=1)
        assert yes
        check_cover(g, cover2, len(cover2))
        assert not vc.solve_k(dg, want - 1, crown=1)[0]
        dg.close()


def test_crown_removes_a_known_crown(vc):
    # K_{2,5} beside a Petersen graph: no degree-one vertex, no triangle and a
    # loose greedy bound, so the other root rules keep all 17 vertices; the
    # LP optimum of K_{2,5} is integral (hubs 1, the rest 0) while Petersen's
    # is all 1/2, so the crown reduction removes exactly K_{2,5}
    g = gg.disjoint_union([gg.complete_bipartite(2, 5), gg.petersen()])
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, cover, st = vc.solve_min(dg, crown=1)
    _, _, st_off = vc.solve_min(dg)
    dg.close()
    assert size == 8
    check_cover(g, cover, size)
    assert st_off["n_induced"] == 17
    assert st["crown_forced"] == 2 and st["crown_removed"] == 7 and st["n_induced"] == 10
    # K_{2,4} beside an odd cycle (all 1/2 in the LP): the greedy bound 5 is
    # optimal, and the hubs' degree 4 stays within the high-degree budget 4,
    # so the root keeps both; the crown reduction leaves only the cycle
    u = gg.disjoint_union([gg.complete_bipartite(2, 4), gg.cycle(5)])
    du = vc.Graph.from_csr(u.row_ptr, u.col)
    size, cover, st = vc.solve_min(du, crown=1)
    du.close()
    assert size == 5 and st["crown_forced"] == 2 and st["crown_removed"] == 6 and st["n_induced"] == 5
    check_cover(u, cover, size)


def test_node_arrays_in_global_memory_when_too_large(vc):
    # without root rules the induced graph keeps every vertex with an edge:
    # ~45k here, too many for a worker's arrays to fit in shared memory, so
    # the search keeps degrees, marks, labels and cover in global memory
    g = gg.chung_lu(50_000, 2.5, 6.0, 2000.0, 0)
    want = oracle.mvc(g.n, g.row_ptr, g.col)[0]
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, cover, st = vc.solve_min(dg, disable_root_rules=1)
    dg.close()
    assert st["n_induced"] > 40_000
    assert size == want
    check_cover(g, cover, size)
    # the same with a real branch on ~1,000 components at the first node
    parts = [gg.gnm(45, 110, 900 + s) for s in range(1000)]
    u = gg.disjoint_union(parts)
    want = sum(oracle.mvc(p.n, p.row_ptr, p.col)[0] for p in parts)
    du = vc.Graph.from_csr(u.row_ptr, u.col)
    size, cover, st = vc.solve_min(du, disable_root_rules=1)
    du.close()
    assert st["n_induced"] > 40_000 and st["component_branches"] >= 1
    assert size == want
    check_cover(u, cover, size)
