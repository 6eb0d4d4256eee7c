"""The served form (vc_server_*): continuous batching over a resident search.

Every served answer must equal the oracle's and the plain single-graph call's
on the same graph, whatever else is in flight; covers are verified edge by
edge.  Short time slices force requests to be preempted and resumed across
steps; a small arena forces admission to wait for retirements; small slot
counts force slot recycling after requests that leave nodes behind (PVC
answered early, node budget exhausted).
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


def verify(g, res):
    cover = res["cover"]
    assert len(np.unique(cover)) == len(cover)
    assert np.all(np.diff(cover) > 0)
    flags = np.zeros(max(g.n, 1), np.uint8)
    flags[cover] = 1
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags[:g.n])


def mixed_graphs():
    gs = [gg.gnm(80, 200, s) for s in range(10)]
    gs += [gg.chung_lu(600, 2.5, 4.0, 100.0, s) for s in range(3)]
    gs += [gg.component_heavy(1, copies=4, copy_n=24, p=0.2, chain=2), gg.random_forest(2000, 5, 1)]
    gs += [gg.cycle(31), gg.complete(12), gg.petersen(), gg.path(2), gg.from_edges(5, [], []),
           gg.from_edges(0, [], [])]
    return gs


def test_served_answers_match_oracle_and_plain(vc):
    graphs = mixed_graphs()
    opts = [opt_of(g) for g in graphs]
    srv = vc.Server(quantum_us=500)
    tags = {}
    for i, g in enumerate(graphs):
        tags[srv.submit(g.row_ptr, g.col, -1)] = ("min", i)
    for i, g in enumerate(graphs[:10]):
        tags[srv.submit(g.row_ptr, g.col, opts[i])] = ("yes", i)
        tags[srv.submit(g.row_ptr, g.col, opts[i] - 1)] = ("no", i)
    res = srv.drain()
    assert len(res) == len(tags)
    for r in res:
        kind, i = tags[r["tag"]]
        g = graphs[i]
        assert r["status"] == vc.VC_OK, (kind, i, r)
        if kind == "min":
            assert r["size"] == opts[i], (i, r["size"], opts[i])
            assert r["yes"] == 1 and r["cover_len"] == opts[i]
            verify(g, r)
            if g.n > 0:   # the plain path on the same graph gives the same answer
                dg = vc.Graph.from_csr(g.row_ptr, g.col)
                assert vc.solve_min(dg)[0] == r["size"]
                dg.close()
        elif kind == "yes":
            assert r["yes"] == 1 and 0 < r["cover_len"] <= opts[i]
            verify(g, r)
        else:
            assert r["yes"] == 0 and r["cover_len"] == 0
    st = srv.stats()
    assert st["completed"] == len(tags) and st["admitted"] == len(tags)
    srv.close()


def test_requests_join_while_others_are_in_flight(vc):
    # component-heavy graphs need many nodes: with a 100 us slice they span
    # several steps, and new requests are admitted beside them
    heavy = [gg.component_heavy(s, copies=8, copy_n=24, p=0.2, chain=3) for s in range(3)]
    light = [gg.gnm(80, 200, 40 + s) for s in range(12)]
    want = {}
    srv = vc.Server(quantum_us=100)
    for g in heavy:
        want[srv.submit(g.row_ptr, g.col)] = g
    srv.step()
    joined_in_flight = 0
    results = srv.poll()
    for g in light:
        q, f, _ = srv.counts()
        joined_in_flight += f > 0
        want[srv.submit(g.row_ptr, g.col)] = g
        srv.step()
        results += srv.poll()
    results += srv.drain()
    assert joined_in_flight > 0
    assert len(results) == len(want)
    for r in results:
        g = want[r["tag"]]
        assert r["status"] == vc.VC_OK
        assert r["size"] == opt_of(g)
        verify(g, r)
    # a heavy request still in flight after a slice was stored at the deadline
    # and resumed later; its answer is exact
    assert srv.stats()["slices"] >= 2
    srv.close()


def test_admission_waits_for_device_memory(vc):
    graphs = [gg.chung_lu(3000, 2.5, 5.0, 300.0, s) for s in range(12)]
    arena = 256 << 10    # room for about two of these at a time
    srv = vc.Server(arena_bytes=arena, quantum_us=200)
    for g in graphs:
        srv.submit(g.row_ptr, g.col)
    most_in_flight = 0
    results = []
    for _ in range(10000):
        q, f, _ = srv.counts()
        if q == 0 and f == 0:
            break
        srv.step()
        most_in_flight = max(most_in_flight, srv.counts()[1])
        results += srv.poll()
    results += srv.poll()
    assert len(results) == len(graphs)
    assert most_in_flight < len(graphs)
    for r in results:
        g = graphs[r["tag"]]
        assert r["status"] == vc.VC_OK and r["size"] == opt_of(g)
        verify(g, r)
    # a request larger than the whole arena is refused at submission
    big = gg.path(20000)
    with pytest.raises(vc.VcError) as ei:
        srv.submit(big.row_ptr, big.col)
    assert ei.value.status == vc.VC_ECAPACITY
    srv.close()


def test_malformed_oversized_and_over_budget_requests(vc):
    srv = vc.Server(max_induced=64, max_induced_large=0, node_budget=50, quantum_us=300)
    good = gg.random_forest(40, 3, 1)           # settled by the root phase
    bad_rp = np.array([0, 1, 2, 2], np.int32)   # 0-1 and 1-2 listed once each: not mirrored
    bad_col = np.array([1, 2], np.int32)
    big_core = gg.gnm(200, 600, 1)              # induced graph above 64 vertices
    hard = gg.gnm(64, 190, 7)                   # more than 50 nodes
    t_good = srv.submit(good.row_ptr, good.col)
    t_bad = srv.submit(bad_rp, bad_col)
    t_big = srv.submit(big_core.row_ptr, big_core.col)
    t_hard = srv.submit(hard.row_ptr, hard.col)
    res = {r["tag"]: r for r in srv.drain()}
    assert res[t_bad]["status"] == vc.VC_EINVAL
    assert res[t_big]["status"] == vc.VC_ECAPACITY and res[t_big]["n_induced"] > 64
    assert res[t_hard]["status"] == vc.VC_EBUDGET and res[t_hard]["nodes"] > 50
    assert res[t_good]["status"] == vc.VC_OK and res[t_good]["size"] == opt_of(good)
    verify(good, res[t_good])
    srv.close()


def test_size_classes_serve_small_and_large_induced_graphs_together(vc):
    # two classes: induced graphs of up to 64 vertices, and up to 512; the
    # small and large requests are in flight together and each answer equals
    # the oracle's and the plain call's; one above 512 is refused
    srv = vc.Server(max_induced=64, max_induced_large=512, quantum_us=300)
    small = [gg.gnm(40, 90, s) for s in range(6)]
    large = [gg.disjoint_union([gg.gnm(40, 90, 10 * s + j) for j in range(4)]) for s in range(4)]
    too_big = gg.disjoint_union([gg.gnm(40, 90, 100 + j) for j in range(40)])
    graphs = []
    for i in range(6):
        graphs.append(small[i])
        if i < 4:
            graphs.append(large[i])
    tags = {srv.submit(g.row_ptr, g.col): g for g in graphs}
    t_big = srv.submit(too_big.row_ptr, too_big.col)
    res = {r["tag"]: r for r in srv.drain()}
    sizes = []
    for t, g in tags.items():
        r = res[t]
        dg = vc.Graph.from_csr(g.row_ptr, g.col)
        want, _, st = vc.solve_min(dg)
        dg.close()
        assert r["status"] == vc.VC_OK and r["size"] == want == opt_of(g)
        assert r["n_induced"] == st["n_induced"]
        verify(g, r)
        sizes.append(r["n_induced"])
    assert max(sizes) > 64 and min(sizes) <= 64    # both classes were used
    assert res[t_big]["status"] == vc.VC_ECAPACITY and res[t_big]["n_induced"] > 512
    st = srv.stats()
    assert st["max_induced"] == 512
    srv.close()


def test_running_out_of_room_ends_only_that_request(vc):
    # a one-slot stack and a 16-slot worklist: requests whose search needs
    # more room finish with VC_ECAPACITY on their own; every answer given is
    # exact, and the server keeps serving afterwards
    srv = vc.Server(stack_depth=1, worklist_capacity=16, max_inflight=8, quantum_us=300)
    hard = [gg.component_heavy(s, copies=6, copy_n=24, p=0.2, chain=3) for s in range(1, 4)]
    easy = [gg.random_forest(200, 3, s) for s in range(3)] + [gg.cycle(41), gg.complete(9)]
    graphs = hard + easy
    tags = {srv.submit(g.row_ptr, g.col): g for g in graphs}
    res = {r["tag"]: r for r in srv.drain()}
    statuses = {r["status"] for r in res.values()}
    assert statuses <= {vc.VC_OK, vc.VC_ECAPACITY}
    for t, g in tags.items():
        if res[t]["status"] == vc.VC_OK:
            assert res[t]["size"] == opt_of(g)
            verify(g, res[t])
    for g in easy:   # settled at the root or closed at once: never short of room
        t = [k for k, v in tags.items() if v is g][0]
        assert res[t]["status"] == vc.VC_OK
    g = gg.gnm(80, 200, 3)
    t = srv.submit(g.row_ptr, g.col)
    r = {x["tag"]: x for x in srv.drain()}[t]
    assert r["status"] in (vc.VC_OK, vc.VC_ECAPACITY)
    if r["status"] == vc.VC_OK:
        assert r["size"] == opt_of(g)
    srv.close()


def test_slot_recycling_after_requests_that_leave_nodes(vc):
    # 2 slots: PVC requests answered early and over-budget requests leave
    # nodes in the stacks and the worklist; the requests that reuse their
    # slots must not see them
    srv = vc.Server(max_inflight=2, node_budget=4000, quantum_us=200)
    graphs = [gg.gnm(60, 120, s) for s in range(8)]
    opts = [opt_of(g) for g in graphs]
    hard = gg.gnm(80, 260, 11)
    plan = []
    for i, g in enumerate(graphs):
        # k = opt: the search stops as soon as a cover of size opt is found
        plan.append((srv.submit(g.row_ptr, g.col, opts[i]), "easy_yes", i))
        plan.append((srv.submit(hard.row_ptr, hard.col), "budget", -1))
        plan.append((srv.submit(g.row_ptr, g.col), "min", i))
    res = {r["tag"]: r for r in srv.drain()}
    assert len(res) == len(plan)
    for tag, kind, i in plan:
        r = res[tag]
        if kind == "easy_yes":
            assert r["status"] == vc.VC_OK and r["yes"] == 1 and r["cover_len"] <= opts[i]
            verify(graphs[i], r)
        elif kind == "budget":
            assert r["status"] in (vc.VC_EBUDGET, vc.VC_OK)
            if r["status"] == vc.VC_OK:
                assert r["size"] == opt_of(hard)
        else:
            assert r["status"] == vc.VC_OK and r["size"] == opts[i]
            verify(graphs[i], r)
    srv.close()


def test_leftover_nodes_are_never_expanded_against_a_new_graph(vc):
    # One slot.  A hard request stops on its node budget with right children
    # (pending "remove N(v)" operations over its own 80-vertex graph) left in
    # the stacks and the worklist; the slot then holds tiny graphs.  Expanding
    # a leftover node against the new graph would read rows that do not exist
    # there and run for seconds; it must be dropped unexpanded instead.
    srv = vc.Server(max_inflight=1, node_budget=3000, quantum_us=200)
    hard = gg.gnm(80, 260, 11)
    tiny = [gg.gnm(12, 20, s) for s in range(6)]
    plan = []
    for g in tiny:
        plan.append((srv.submit(hard.row_ptr, hard.col), None))
        plan.append((srv.submit(g.row_ptr, g.col), g))
    res = {r["tag"]: r for r in srv.drain()}
    for tag, g in plan:
        if g is None:
            assert res[tag]["status"] in (vc.VC_EBUDGET, vc.VC_OK)
            continue
        assert res[tag]["status"] == vc.VC_OK and res[tag]["size"] == opt_of(g)
        verify(g, res[tag])
    st = srv.stats()
    assert st["ms_search"] / max(1, st["slices"]) < 20.0     # slices end at their deadline
    srv.close()
