"""GPU parity: the CUDA solver (through the C ABI) against the CPU oracle.

Answers (minimum cover size, PVC yes/no) must match bit-exactly; covers are
not unique, so every returned cover is verified edge by edge and its size
checked against the answer.
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


def check_cover(g, cover, size):
    flags = np.zeros(max(g.n, 1), np.uint8)
    flags[cover] = 1
    assert len(cover) == size
    assert len(np.unique(cover)) == len(cover)
    assert np.all(np.diff(cover) > 0)                       # ascending ids
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags[:g.n])


def gpu_min(vc, g, **kw):
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        size, cover, st = vc.solve_min(dg, **kw)
    finally:
        dg.close()
    check_cover(g, cover, size)
    return size, st


# ------------------------------------------------ Erdos-Renyi G(80, 200)

@pytest.mark.parametrize("seed", range(24))
def test_gnm_80_200(vc, seed):
    g = gg.gnm(80, 200, seed)
    want = oracle.mvc(g.n, g.row_ptr, g.col)[0]
    assert gpu_min(vc, g)[0] == want


def test_brute_force_small_random(vc):
    rng = np.random.default_rng(11)
    for seed in range(120):
        n = int(rng.integers(8, 23))
        g = gg.gnp(n, [0.1, 0.2, 0.3, 0.45, 0.6][seed % 5], seed)
        assert gpu_min(vc, g)[0] == oracle.brute_mvc(g.n, g.row_ptr, g.col)[0], (n, seed)


def test_closed_forms(vc):
    cases = [(gg.path(2001), 1000), (gg.cycle(1001), 501), (gg.cycle(1000), 500),
             (gg.complete(40), 39), (gg.complete_bipartite(30, 45), 30), (gg.petersen(), 6),
             (gg.star(500), 1), (gg.complete(2), 1), (gg.cycle(3), 2), (gg.cycle(5), 3)]
    for g, want in cases:
        assert gpu_min(vc, g)[0] == want, g.name


def test_forests(vc):
    for seed in range(6):
        g = gg.random_forest(5000, 1 + 3 * seed, seed)
        assert gpu_min(vc, g)[0] == oracle.mvc(g.n, g.row_ptr, g.col)[0]


def test_components_cliques_cycles(vc):
    parts = [gg.cycle(5), gg.cycle(7), gg.cycle(4), gg.complete(4), gg.complete(6),
             gg.cycle(9), gg.complete(3), gg.petersen(), gg.gnm(30, 70, 3), gg.gnm(25, 60, 4)]
    u = gg.disjoint_union(parts)
    want = oracle.mvc(u.n, u.row_ptr, u.col)[0]
    assert gpu_min(vc, u)[0] == want
    # hang the parts off one hub so the split happens inside the search
    uu, vv = gg.edges_of(u)
    hub = u.n
    offs = np.cumsum([0] + [p.n for p in parts[:-1]])
    h = gg.from_edges(u.n + 1, np.concatenate([uu, np.full(len(parts), hub)]),
                      np.concatenate([vv, offs]))
    assert gpu_min(vc, h)[0] == oracle.mvc(h.n, h.row_ptr, h.col)[0]


def test_edge_cases(vc):
    empty = gg.from_edges(0, [], [])
    dg = vc.Graph.from_csr(empty.row_ptr, empty.col)
    assert vc.solve_min(dg)[0] == 0
    dg.close()
    iso = gg.from_edges(7, [], [])
    assert gpu_min(vc, iso)[0] == 0
    assert gpu_min(vc, gg.path(2))[0] == 1
    k2s = gg.disjoint_union([gg.path(2)] * 9 + [gg.from_edges(3, [], [])])
    assert gpu_min(vc, k2s)[0] == 9


# disjoint random graphs hung on a chain of articulation vertices: forces
# nested branches on components; shapes small enough for the oracle
@pytest.mark.parametrize("copies,copy_n,p,chain", [(3, 48, 0.12, 2), (4, 48, 0.12, 2), (8, 24, 0.2, 3),
                                                   (12, 24, 0.2, 3), (16, 20, 0.2, 4), (32, 16, 0.25, 6)])
def test_component_heavy_small(vc, copies, copy_n, p, chain):
    g = gg.component_heavy(1, copies=copies, copy_n=copy_n, p=p, chain=chain)
    want = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
    for team in (32, 256):
        size, st = gpu_min(vc, g, team=team)
        assert size == want, team
        assert st["component_branches"] + st["trivial_components"] > 0


def test_large_graph_with_core(vc):
    # n >= 8192: the root phase runs on a thread-block cluster; the core left
    # after the unbounded rules exercises the greedy bound, the bounded rules
    # and the induced-subgraph build
    parts = [gg.gnm(40, 90, s) for s in range(300)]
    g = gg.disjoint_union(parts)
    want = sum(oracle.mvc(p.n, p.row_ptr, p.col)[0] for p in parts)
    size, st = gpu_min(vc, g)
    assert size == want
    assert st["n_induced"] > 0


def test_chung_lu_50k(vc):
    g = gg.chung_lu(50_000, 2.5, 6.0, 2000.0, 0)
    want = oracle.mvc(g.n, g.row_ptr, g.col)[0]
    size, st = gpu_min(vc, g)
    assert size == want
    assert st["n_induced"] <= 64


def _spiders(hubs, legs, leg_len):
    # hubs, each with `legs` paths of leg_len vertices hanging off it: the
    # leaves peel inwards until the hubs, still of high degree, are forced
    u, v, n = [], [], 0
    for _ in range(hubs):
        h = n
        n += 1
        for _ in range(legs):
            prev = h
            for _ in range(leg_len):
                u.append(prev)
                v.append(n)
                prev = n
                n += 1
    return gg.from_edges(n, u, v, "spiders")


def test_residual_rounds_on_one_cta(vc):
    # n >= 8192: once the live graph fits in one CTA's shared memory, the last
    # rounds of the unbounded rules run there on a renumbered copy; answers
    # (and witnesses) must stay exact whether the graph vanishes, keeps a
    # core for the greedy bound, bounded rules and search, or keeps hubs
    # whose long rows are applied by whole warps
    cases = [gg.chung_lu(20_000, 2.5, 6.0, 800.0, 7), gg.chung_lu(60_000, 2.5, 6.0, 2000.0, 3),
             gg.chung_lu(30_000, 2.2, 8.0, 3000.0, 5), _spiders(12, 300, 3), _spiders(40, 120, 2)]
    for g in cases:
        want = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=2_000_000)[0]
        for _ in range(2):
            assert gpu_min(vc, g)[0] == want, g.name
    parts = [gg.random_forest(9000, 40, 11)] + [gg.gnm(40, 90, s) for s in range(20)] + [_spiders(3, 200, 3)]
    g = gg.disjoint_union(parts)
    want = sum(oracle.mvc(p.n, p.row_ptr, p.col)[0] for p in parts)
    size, st = gpu_min(vc, g)
    assert size == want and st["n_induced"] > 0
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        yes, cover, _ = vc.solve_k(dg, want)
        assert yes and len(cover) <= want
        check_cover(g, cover, len(cover))
        assert not vc.solve_k(dg, want - 1)[0]
    finally:
        dg.close()


def test_cluster_rows_too_many_to_stage(vc):
    # 9,048 vertices, 1,024 per CTA.  The first CTA's vertices are nine
    # copies of K(56, 56): about 56k row entries, more than its shared memory
    # holds, so it reads its rows from the global CSR.  The second CTA's are
    # twelve copies of K(40, 40): about 38k entries, staged, but with no room
    # for the per-entry source index, so its degree updates walk the rows.
    # The rest is a forest and two paths for the rule rounds to peel.
    # A minimum cover of K(a, a) has a vertices.
    forest = gg.random_forest(7000, 60, 13)
    parts = ([gg.complete_bipartite(56, 56) for _ in range(9)] + [gg.path(16)] +
             [gg.complete_bipartite(40, 40) for _ in range(12)] + [gg.path(64)] + [forest])
    g = gg.disjoint_union(parts)
    assert g.n == 9048
    want = 9 * 56 + 8 + 12 * 40 + 32 + oracle.mvc(forest.n, forest.row_ptr, forest.col)[0]
    for _ in range(2):
        size, st = gpu_min(vc, g)
        assert size == want
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        yes, cover, _ = vc.solve_k(dg, want)
        assert yes and len(cover) <= want
        check_cover(g, cover, len(cover))
        assert not vc.solve_k(dg, want - 1)[0]
    finally:
        dg.close()


def test_chung_lu_50k_decision_and_independent_set(vc):
    # the cluster root phase settles this graph and writes the cover list
    # itself; the decision form and the complement go through finalisation
    g = gg.chung_lu(50_000, 2.5, 6.0, 2000.0, 0)
    opt = oracle.mvc(g.n, g.row_ptr, g.col)[0]
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        for _ in range(2):
            size, cover, _ = vc.solve_min(dg)
            assert size == opt and np.all(np.diff(cover) > 0)
            check_cover(g, cover, size)
        yes, cover, _ = vc.solve_k(dg, opt)
        assert yes and len(cover) <= opt and np.all(np.diff(cover) > 0)
        check_cover(g, cover, len(cover))
        assert not vc.solve_k(dg, opt - 1)[0]
        alpha, iset, _ = vc.solve_mis(dg)
        assert alpha == g.n - opt and len(iset) == alpha and np.all(np.diff(iset) > 0)
        inside = np.zeros(g.n, bool)
        inside[iset] = True
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        assert not np.any(inside[src] & inside[g.col])
        sizes, yes_b, status, covers, _ = vc.solve_batch([dg, dg], [-1, opt])
        assert list(sizes[:1]) == [opt] and all(status == vc.VC_OK) and yes_b[1]
        for c in covers:
            check_cover(g, c, len(c))
    finally:
        dg.close()


def test_options_same_answers(vc):
    for seed in range(6):
        g = gg.gnm(80, 200, 100 + seed)
        want = oracle.mvc(g.n, g.row_ptr, g.col)[0]
        for kw in [dict(use_components=0), dict(team=32), dict(team=256), dict(dtype_bytes=2),
                   dict(dtype_bytes=4), dict(load_balance=0), dict(stack_depth=2, worklist_capacity=64)]:
            assert gpu_min(vc, g, **kw)[0] == want, kw


def test_pvc_at_opt_and_opt_minus_one(vc):
    for seed in range(10):
        g = gg.gnm(80, 200, seed)
        opt = oracle.mvc(g.n, g.row_ptr, g.col)[0]
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        yes, cover, _ = vc.solve_k(dg, opt)
        assert yes
        assert len(cover) <= opt
        check_cover(g, cover, len(cover))
        no, cover2, _ = vc.solve_k(dg, opt - 1)
        assert not no and cover2 is None
        assert vc.solve_k(dg, opt + 5)[0]
        dg.close()


@pytest.mark.parametrize("copies,copy_n,p,chain", [(4, 48, 0.12, 2), (8, 24, 0.2, 3), (16, 20, 0.2, 4),
                                                   (32, 16, 0.25, 6)])
def test_pvc_component_heavy(vc, copies, copy_n, p, chain):
    # improvements inside components are pushed to the root (Section 3.5):
    # the answer and the witness must stay exact
    g = gg.component_heavy(2, copies=copies, copy_n=copy_n, p=p, chain=chain)
    opt = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    for team in (32, 256):
        yes, cover, st = vc.solve_k(dg, opt, team=team)
        assert yes and len(cover) <= opt
        check_cover(g, cover, len(cover))
        assert not vc.solve_k(dg, opt - 1, team=team)[0]
        yes2, cover2, _ = vc.solve_k(dg, opt + 2, team=team)
        assert yes2 and len(cover2) <= opt + 2
        check_cover(g, cover2, len(cover2))
    dg.close()


def test_pvc_k_zero(vc):
    g = gg.from_edges(5, [], [])
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    assert vc.solve_k(dg, 0)[0]
    dg.close()
    g = gg.path(3)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    assert not vc.solve_k(dg, 0)[0]
    with pytest.raises(vc.VcError):
        vc.solve_k(dg, -1)
    dg.close()


def test_batch_matches_single(vc):
    graphs = [gg.gnm(80, 200, s) for s in range(12)] + [gg.chung_lu(600, 2.5, 4.0, 100.0, s) for s in range(4)]
    opts = [oracle.mvc(g.n, g.row_ptr, g.col)[0] for g in graphs]
    dgs = [vc.Graph.from_csr(g.row_ptr, g.col) for g in graphs]
    # each graph at minimum, at k = opt and at k = opt - 1
    qg = dgs + dgs + dgs
    ks = [-1] * len(dgs) + opts + [o - 1 for o in opts]
    sizes, yes, status, covers, st = vc.solve_batch(qg, ks)
    assert np.all(status == 0)
    n = len(dgs)
    for i, g in enumerate(graphs):
        assert sizes[i] == opts[i]
        check_cover(g, covers[i], sizes[i])
        assert yes[n + i] and len(covers[n + i]) <= opts[i]
        check_cover(g, covers[n + i], len(covers[n + i]))
        assert not yes[2 * n + i] and len(covers[2 * n + i]) == 0
    for d in dgs:
        d.close()


def test_device_resident_input(vc):
    import torch
    g = gg.gnm(80, 200, 5)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    dg = vc.Graph.from_device(rp, col)
    size, cover, _ = vc.solve_min(dg)
    dg.close()
    assert size == oracle.mvc(g.n, g.row_ptr, g.col)[0]
    check_cover(g, cover, size)


def test_invalid_csr_rejected(vc):
    bad = [
        (np.array([0, 1, 1], np.int32), np.array([1], np.int32)),          # asymmetric
        (np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32)),       # self-loops
        (np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32)),  # duplicates
        (np.array([0, 1, 2], np.int32), np.array([5, 0], np.int32)),       # out of range
        (np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32)),       # row_ptr decreasing
    ]
    for rp, col in bad:
        with pytest.raises(vc.VcError) as ei:
            vc.Graph.from_csr(rp, col)
        assert ei.value.status == vc.VC_EINVAL


def test_node_budget_reports_cleanly(vc):
    g = gg.gnm(120, 330, 0)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    with pytest.raises(vc.VcError) as ei:
        vc.solve_min(dg, node_budget=1)
    assert ei.value.status in (vc.VC_EBUDGET,)
    # the handle stays usable
    size, cover, _ = vc.solve_min(dg)
    dg.close()
    assert size == oracle.mvc(g.n, g.row_ptr, g.col)[0]


def test_registry_exhaustion_reports_cleanly(vc):
    g = gg.component_heavy(1, copies=8, copy_n=24, p=0.2, chain=3)
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    with pytest.raises(vc.VcError) as ei:
        vc.solve_min(dg, registry_capacity=1, capacity_retries=0)
    assert ei.value.status == vc.VC_ECAPACITY
    size, _, _ = vc.solve_min(dg)
    dg.close()
    assert size == oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]


def test_capacity_retries_grow_the_capacities(vc):
    # a registry of one entry, a two-slot stack and a small worklist: the
    # solve is repeated with doubled capacities until they suffice; the
    # answer is exact
    import torch
    g = gg.component_heavy(1, copies=8, copy_n=24, p=0.2, chain=3)
    want = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        vc.solve_min(dg)   # a pooled workspace at the default sizes
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        size, cover, st = vc.solve_min(dg, registry_capacity=1, stack_depth=2, worklist_capacity=64,
                                       capacity_retries=30)
        assert size == want and st["retries"] >= 1
        check_cover(g, cover, size)
        # the retried solve freed the workspace it grew
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
        sizes, _, status, covers, bst = vc.solve_batch([dg, dg], [-1, want], registry_capacity=1,
                                                       capacity_retries=30)
        assert list(status) == [vc.VC_OK, vc.VC_OK] and sizes[0] == want and bst["retries"] >= 1
        for c in covers:
            check_cover(g, c, len(c))
        # registry exhaustion grows only the registry: a one-entry registry
        # with ample slots needs retries but reaches the answer
        size, _, st = vc.solve_min(dg, registry_capacity=1, capacity_retries=30)
        assert size == want and st["retries"] >= 1
    finally:
        dg.close()


@pytest.mark.parametrize("team", [64, 128, 256, 512, 1024])
def test_component_labels_with_every_block_size(vc, team):
    # one block labels every vertex of a node's components; with path
    # halving in the final pass, vertices could keep a stale (non-root)
    # label and a cycle was counted short -- nearly every run at 128+ threads
    for g, want in [(gg.cycle(1001), 501), (gg.cycle(1000), 500)]:
        for _ in range(5):
            assert gpu_min(vc, g, team=team)[0] == want
    u = gg.disjoint_union([gg.cycle(5 + (s % 7)) for s in range(300)] + [gg.complete(4 + s % 3) for s in range(50)])
    want = oracle.mvc(u.n, u.row_ptr, u.col)[0]
    for _ in range(3):
        assert gpu_min(vc, u, team=team)[0] == want


@pytest.mark.parametrize("team", [32, 128, 1024])
def test_label_propagation_finds_the_same_components(vc, team):
    # the two ways of splitting a node into components (union-find, label
    # propagation) must give the same components: long cycles need many
    # label rounds, the union splits into 350 pieces at its first node, all
    # closed by the clique and cycle rules
    for g, want in [(gg.cycle(1001), 501), (gg.cycle(1000), 500), (gg.path(777), 388)]:
        assert gpu_min(vc, g, team=team, label_propagation=1)[0] == want
    u = gg.disjoint_union([gg.cycle(5 + (s % 7)) for s in range(300)] + [gg.complete(4 + s % 3) for s in range(50)])
    want = oracle.mvc(u.n, u.row_ptr, u.col)[0]
    size, st = gpu_min(vc, u, team=team, label_propagation=1)
    size_uf, st_uf = gpu_min(vc, u, team=team)
    assert size == size_uf == want
    assert st["trivial_components"] == st_uf["trivial_components"]
    if st_uf["nodes"] > 0:
        assert st_uf["trivial_components"] == 350
    g = gg.component_heavy(3, copies=6, copy_n=30, p=0.15, chain=3)
    opt = oracle.mvc(g.n, g.row_ptr, g.col, node_budget=5_000_000)[0]
    assert gpu_min(vc, g, team=team, label_propagation=1)[0] == opt
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    try:
        yes, cover, _ = vc.solve_k(dg, opt, team=team, label_propagation=1)
        assert yes and len(cover) <= opt
        check_cover(g, cover, len(cover))
        assert not vc.solve_k(dg, opt - 1, team=team, label_propagation=1)[0]
    finally:
        dg.close()


def test_workspace_pool_reuse_and_trim(vc):
    # solves on different handles share pooled workspaces; trimming between
    # solves is safe and the next solve rebuilds what it needs
    gs = [gg.gnm(80, 200, 60 + s) for s in range(6)]
    for i, g in enumerate(gs):
        assert gpu_min(vc, g)[0] == oracle.mvc(g.n, g.row_ptr, g.col)[0]
        if i == 2:
            assert vc.trim() >= 1
    assert gpu_min(vc, gg.cycle(501))[0] == 251
