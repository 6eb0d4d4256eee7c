"""Pins for the CPU oracle: things the mathematics fixes, independent of the
oracle's own code.

- brute force (subset enumeration) is checked against closed forms and against
  a second, separately written enumeration of independent sets (OPT = n - alpha);
- Algorithm 2 (``oracle.mvc``) is checked against brute force on every labelled
  graph with n <= 6 and on random graphs with n <= 22;
- closed forms at sizes brute force cannot reach: P_n, C_n, K_n, K_{a,b},
  Petersen, forests (leaf-greedy, exact on forests by the degree-one exchange);
- Koenig's theorem on large bipartite graphs: OPT = maximum matching, with the
  matching itself checked against scipy's bipartite matching;
- additivity over disjoint unions (exercises branching on components and the
  clique / cycle component rules) and invariance under relabelling;
- PVC consistency: yes at k = OPT, no at k = OPT - 1;
- planted mistakes (``ORC_MUTANT``) are each caught by at least one pin.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle


def opt(g, **kw):
    k, cover, _ = oracle.mvc(g.n, g.row_ptr, g.col, **kw)
    return k, cover


def brute(g):
    return oracle.brute_mvc(g.n, g.row_ptr, g.col)[0]


# ------------------------------------------------------------------ generators

def test_csr_canonical():
    g = gg.from_edges(5, [0, 1, 1, 2, 4, 3, 3], [1, 0, 2, 2, 3, 4, 0])
    assert g.row_ptr.dtype == np.int32 and g.col.dtype == np.int32
    for v in range(g.n):
        row = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.all(np.diff(row) > 0)          # sorted, no duplicates
        assert v not in row                      # no loops
        for u in row:
            assert v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]  # symmetric
    assert g.m == 4


def test_gnp_sparse_pairs_valid():
    for seed in range(5):
        g = gg.gnp_sparse(300, 0.02, seed)
        u, v = gg.edges_of(g)
        assert np.all(u < v) and np.all(v < 300)
        assert abs(g.m - 0.02 * 300 * 299 / 2) < 6 * math.sqrt(0.02 * 300 * 299 / 2)


def test_gnm_exact_edge_count():
    g = gg.gnm(80, 200, 3)
    assert g.n == 80 and g.m == 200


def test_chung_lu_shape():
    g = gg.chung_lu(50_000, 2.5, 6.0, 2000.0, 0)
    d = g.degrees()
    assert 5.0 < d.mean() < 6.5
    assert d.max() <= 2100


# ----------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", range(1, 21))
def test_brute_closed_forms_paths_cycles(n):
    assert brute(gg.path(n)) == n // 2
    if n >= 3:
        assert brute(gg.cycle(n)) == (n + 1) // 2


def test_brute_closed_forms_other():
    for n in range(1, 13):
        assert brute(gg.complete(n)) == max(n - 1, 0)
    for a in range(1, 7):
        for b in range(1, 7):
            assert brute(gg.complete_bipartite(a, b)) == min(a, b)
    assert brute(gg.petersen()) == 6
    assert brute(gg.star(9)) == 1
    assert brute(gg.from_edges(7, [], [])) == 0


def _alpha_by_independent_sets(g):
    """Largest independent set by plain enumeration (a different formulation)."""
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    for size in range(g.n, -1, -1):
        for sub in itertools.combinations(range(g.n), size):
            s = set(sub)
            if all(not (adj[v] & s) for v in sub):
                return size
    return 0


def test_brute_equals_n_minus_alpha():
    for seed in range(40):
        g = gg.gnp(10, 0.1 + 0.5 * (seed % 6) / 5, seed)
        assert brute(g) == g.n - _alpha_by_independent_sets(g)


# ---------------------------------------------------- Algorithm 2 vs brute force

def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        u = [pairs[i][0] for i in range(len(pairs)) if mask >> i & 1]
        v = [pairs[i][1] for i in range(len(pairs)) if mask >> i & 1]
        yield gg.from_edges(n, u, v)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_mvc_all_labelled_graphs(n):
    for g in _all_graphs(n):
        k, cover = opt(g)
        assert k == brute(g)
        assert oracle.verify_cover(g.n, g.row_ptr, g.col, cover) and cover.sum() == k


def _covers_by_edges(g, flags):
    """Definition of a cover (Section 2.1) restated with numpy over the edge list."""
    u, v = gg.edges_of(g)
    f = np.asarray(flags, dtype=bool)
    return bool(np.all(f[u] | f[v])) if u.size else True


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_verify_rejects_a_minimum_cover_minus_one_vertex(n):
    # every labelled graph with an edge: drop each vertex of a minimum cover
    # in turn; the edges to the dropped vertex's non-cover neighbours are bare
    checked = 0
    for g in _all_graphs(n):
        if g.m == 0:
            continue
        _, cover = opt(g)
        for v in np.flatnonzero(cover):
            bad = cover.copy()
            bad[v] = 0
            assert not oracle.verify_cover(g.n, g.row_ptr, g.col, bad)
            checked += 1
    assert checked > 0


def test_verify_rejects_the_empty_set():
    for g in [gg.path(2), gg.cycle(5), gg.complete(4), gg.petersen(), gg.gnm(80, 200, 0)]:
        assert not oracle.verify_cover(g.n, g.row_ptr, g.col, np.zeros(g.n, np.uint8))
    g = gg.from_edges(4, [], [])
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, np.zeros(g.n, np.uint8))


def test_verify_matches_edge_test_on_random_subsets():
    rng = np.random.default_rng(11)
    seen = {True: 0, False: 0}
    for seed in range(200):
        n = int(rng.integers(2, 40))
        g = gg.gnp(n, [0.05, 0.1, 0.2, 0.4][seed % 4], seed)
        for _ in range(10):
            flags = (rng.random(n) < rng.uniform(0.3, 0.95)).astype(np.uint8)
            want = _covers_by_edges(g, flags)
            assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags) == want
            seen[want] += 1
    assert seen[True] > 100 and seen[False] > 100


def _verify_pins_fail(mutant):
    """The negative pins above, run against a (possibly mutant) oracle build."""
    for n in (3, 4):
        for g in _all_graphs(n):
            _, cover = opt(g)
            for v in np.flatnonzero(cover):
                bad = cover.copy()
                bad[v] = 0
                if oracle.verify_cover(g.n, g.row_ptr, g.col, bad, mutant=mutant):
                    return True
    rng = np.random.default_rng(5)
    for seed in range(40):
        g = gg.gnp(20, 0.2, seed)
        flags = (rng.random(g.n) < 0.7).astype(np.uint8)
        if oracle.verify_cover(g.n, g.row_ptr, g.col, flags, mutant=mutant) != _covers_by_edges(g, flags):
            return True
    return False


def test_verify_mutant_is_caught():
    # a planted early acceptance in the cover check (ORC_MUTANT 8) fails the
    # negative pins; the normal build passes them
    assert _verify_pins_fail(8)
    assert not _verify_pins_fail(0)


def test_mvc_random_vs_brute():
    rng = np.random.default_rng(7)
    for seed in range(300):
        n = int(rng.integers(8, 23))
        p = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6][seed % 6]
        g = gg.gnp(n, p, seed)
        k, cover = opt(g)
        assert k == brute(g), (n, p, seed)
        assert oracle.verify_cover(g.n, g.row_ptr, g.col, cover) and cover.sum() == k


def test_mvc_without_components_same_answer():
    for seed in range(60):
        g = gg.gnp(18, 0.15, seed)
        assert opt(g)[0] == opt(g, use_components=False)[0]


# ---------------------------------------------------------------- closed forms

def test_closed_forms_large():
    assert opt(gg.path(2001))[0] == 1000
    assert opt(gg.cycle(1001))[0] == 501
    assert opt(gg.cycle(1000))[0] == 500
    assert opt(gg.complete(40))[0] == 39
    assert opt(gg.complete_bipartite(30, 45))[0] == 30
    assert opt(gg.petersen())[0] == 6
    assert opt(gg.star(500))[0] == 1


def _leaf_greedy_forest(g):
    """Exact MVC of a forest: repeatedly put the neighbour of a leaf in the cover."""
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    size = 0
    leaves = [v for v in range(g.n) if len(adj[v]) == 1]
    while leaves:
        v = leaves.pop()
        if len(adj[v]) != 1:
            continue
        (u,) = adj[v]
        size += 1
        for w in list(adj[u]):
            adj[w].discard(u)
            if len(adj[w]) == 1:
                leaves.append(w)
        adj[u] = set()
    return size


def test_forests_leaf_greedy():
    for seed in range(20):
        g = gg.random_forest(3000, 1 + seed, seed)
        assert opt(g)[0] == _leaf_greedy_forest(g)


# -------------------------------------------------------------------- Koenig

def test_matching_vs_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(10):
        na, nb = 300, 400
        g = gg.random_bipartite_chung_lu(na, nb, 2.7, 3.0, 60.0, seed)
        k, mate = oracle.max_matching(g.n, g.row_ptr, g.col)
        u, v = gg.edges_of(g)
        bi = sp.csr_matrix((np.ones(u.size), (u, v - na)), shape=(na, nb))
        ref = csgraph.maximum_bipartite_matching(bi, perm_type="column")
        assert k == int((ref >= 0).sum())
        # the returned matching is a matching of the graph
        for a in range(g.n):
            if mate[a] >= 0:
                assert mate[mate[a]] == a
                assert mate[a] in g.col[g.row_ptr[a]:g.row_ptr[a + 1]]


def test_matching_not_bipartite():
    assert oracle.max_matching(3, gg.cycle(3).row_ptr, gg.cycle(3).col)[0] == -1


def test_koenig_bipartite_small_brute():
    for seed in range(40):
        g = gg.random_bipartite_chung_lu(9, 11, 2.5, 2.5, 6.0, seed)
        assert oracle.max_matching(g.n, g.row_ptr, g.col)[0] == brute(g)


def test_koenig_bipartite_large():
    for seed in range(6):
        g = gg.random_bipartite_chung_lu(1500, 2000, 2.5, 2.2, 200.0, seed)
        k, cover = opt(g, node_budget=2_000_000)
        assert k == oracle.max_matching(g.n, g.row_ptr, g.col)[0]
        assert oracle.verify_cover(g.n, g.row_ptr, g.col, cover)


# -------------------------------------------------------- additivity, relabel

def test_additivity_disjoint_union():
    for seed in range(30):
        a = gg.gnp(12, 0.3, seed)
        b = gg.gnp(14, 0.25, seed + 1000)
        c = gg.gnp(9, 0.4, seed + 2000)
        u = gg.disjoint_union([a, b, c])
        assert opt(u)[0] == brute(a) + brute(b) + brute(c)


def test_additivity_cycles_and_cliques():
    parts = [gg.cycle(5), gg.cycle(7), gg.cycle(4), gg.complete(4), gg.complete(6),
             gg.cycle(9), gg.complete(3), gg.petersen()]
    u = gg.disjoint_union(parts)
    want = 3 + 4 + 2 + 3 + 5 + 5 + 2 + 6
    k, cover = opt(u)
    assert k == want
    assert oracle.verify_cover(u.n, u.row_ptr, u.col, cover) and cover.sum() == k
    # the same pieces hung off a hub: the hub's removal splits them apart
    g = gg.disjoint_union([gg.star(0)] + parts)
    uu, vv = gg.edges_of(g)
    hub_edges_u = [0] * len(parts)
    off, hub_edges_v = 1, []
    for p in parts:
        hub_edges_v.append(off)
        off += p.n
    g2 = gg.from_edges(g.n, np.concatenate([uu, hub_edges_u]), np.concatenate([vv, hub_edges_v]))
    k2, cover2 = opt(g2)
    assert oracle.verify_cover(g2.n, g2.row_ptr, g2.col, cover2) and cover2.sum() == k2
    assert k2 in (want, want + 1)


def test_relabel_invariance():
    for seed in range(20):
        g = gg.gnm(60, 110, seed)
        assert opt(g)[0] == opt(gg.relabel(g, seed + 5))[0]


def test_component_heavy_small():
    g = gg.component_heavy(0, copies=12, copy_n=20, p=0.15, chain=6)
    k, cover = opt(g)
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, cover) and cover.sum() == k
    # matching lower bound and greedy upper bound bracket it
    gk = oracle.greedy(g.n, g.row_ptr, g.col)[0]
    assert k <= gk


# ------------------------------------------------------------------------ PVC

def test_pvc_consistency():
    for seed in range(30):
        g = gg.gnp(16, 0.25, seed)
        k = brute(g)
        yes, size, cover = oracle.pvc(g.n, g.row_ptr, g.col, k)
        assert yes and size <= k
        assert oracle.verify_cover(g.n, g.row_ptr, g.col, cover) and cover.sum() == size
        if k > 0:
            assert not oracle.pvc(g.n, g.row_ptr, g.col, k - 1)[0]
        assert oracle.pvc(g.n, g.row_ptr, g.col, k + 3)[0]


def test_pvc_k_zero():
    g = gg.from_edges(4, [], [])
    assert oracle.pvc(g.n, g.row_ptr, g.col, 0)[0]
    g = gg.path(2)
    assert not oracle.pvc(g.n, g.row_ptr, g.col, 0)[0]


# ---------------------------------------------------------------- rule checker

def test_rule_violation():
    g = gg.path(3)
    assert oracle.rule_violation(g.n, g.row_ptr, g.col, np.zeros(3, np.uint8), -1) == (0, "degree-one")
    g = gg.complete(3)
    assert oracle.rule_violation(g.n, g.row_ptr, g.col, np.zeros(3, np.uint8), -1) == (0, "triangle")
    g = gg.cycle(5)
    assert oracle.rule_violation(g.n, g.row_ptr, g.col, np.zeros(5, np.uint8), -1) is None
    assert oracle.rule_violation(g.n, g.row_ptr, g.col, np.zeros(5, np.uint8), 1) == (0, "high-degree")


# ----------------------------------------------------------- planted mistakes

def _hub_of_cycles(count, length):
    parts = gg.disjoint_union([gg.cycle(length)] * count)
    u, v = gg.edges_of(parts)
    hub = parts.n
    return gg.from_edges(parts.n + 1, np.concatenate([u, [hub] * count]),
                         np.concatenate([v, [i * length for i in range(count)]]))


def test_hub_of_cycles():
    g = _hub_of_cycles(3, 5)
    assert brute(g) == 9 and opt(g)[0] == 9


def _pins_fail(mutant):
    """Run a cheap subset of the pins against a mutant oracle build; True if any fails."""
    def mk(g):
        return oracle.mvc(g.n, g.row_ptr, g.col, mutant=mutant)
    checks = []
    for seed in range(120):
        g = gg.gnp(10 + seed % 9, [0.15, 0.25, 0.35][seed % 3], seed)
        checks.append((g, brute(g)))
    parts = [gg.cycle(5), gg.cycle(7), gg.complete(4), gg.complete(5), gg.cycle(9)]
    u = gg.disjoint_union(parts)
    checks.append((u, 3 + 4 + 3 + 4 + 5))
    # a hub joined to one vertex of each of three 5-cycles: branching on the
    # hub leaves |S| = 1 before the branch on components
    h = _hub_of_cycles(3, 5)
    checks.append((h, brute(h)))
    for g, want in checks:
        try:
            k, cover, _ = mk(g)
        except Exception:
            return True
        if k != want or not oracle.verify_cover(g.n, g.row_ptr, g.col, cover) or cover.sum() != k:
            return True
    return False


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_planted_mistakes_are_caught(mutant):
    assert _pins_fail(mutant)


def test_unmutated_passes_the_same_checks():
    assert not _pins_fail(0)


# ------------------------------------------------ branching-factor sanity note

def test_branching_factor_example():
    # Section 3.1: beta = 1.5, rho = 0.02, eta = 0.5 gives beta_e ~= 1.494 and
    # (beta / beta_e)^200 ~= 2.25 times fewer nodes.
    beta_e = 1.5 ** (1 - 0.02 * 0.5)
    assert abs(beta_e - 1.494) < 1e-3
    assert abs((1.5 / beta_e) ** 200 - 2.25) < 0.03
