"""The paper's worked example (tests/golden/search_tree_example.txt): the
oracle, brute force and -- on a GPU -- the library must reproduce what the
paper states about it."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = "abcdefghi"


def load():
    spec = {}
    with open(os.path.join(HERE, "golden", "search_tree_example.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, *vals = line.split()
                spec[key] = vals
    n = int(spec["vertices"][0])
    u, v = zip(*[(NAMES.index(e[0]), NAMES.index(e[2])) for e in spec["edges"]])
    return gg.from_edges(n, u, v), spec


def ids(names):
    return sorted(NAMES.index(x) for x in names)


def test_example_statements_hold():
    g, spec = load()
    deg = np.diff(g.row_ptr)
    e = NAMES.index(spec["max_degree_vertex"][0])
    assert deg[e] == deg.max() and np.count_nonzero(deg == deg.max()) == 1
    assert sorted(g.col[g.row_ptr[e]:g.row_ptr[e + 1]].tolist()) == ids(spec["neighbourhood_of_e"])
    for cov in (spec["cover_right_branch"], spec["minimum_cover"]):
        flags = np.zeros(g.n, np.uint8)
        flags[ids(cov)] = 1
        assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags)
    # components of G - e (isolated vertices are not components)
    keep = [x for x in range(g.n) if x != e]
    adj = {x: set() for x in keep}
    for x in keep:
        for y in g.col[g.row_ptr[x]:g.row_ptr[x + 1]]:
            if y != e:
                adj[x].add(int(y))
    seen, comps = set(), []
    for x in keep:
        if x in seen or not adj[x]:
            continue
        stack, comp = [x], set()
        while stack:
            z = stack.pop()
            if z not in comp:
                comp.add(z)
                stack.extend(adj[z] - comp)
        seen |= comp
        comps.append(sorted(comp))
    want = sorted(ids(c.split(",")) for c in spec["components_after_removing_e"])
    assert sorted(comps) == want


def test_oracle_and_brute_force_find_the_papers_minimum():
    g, spec = load()
    size = int(spec["minimum_size"][0])
    assert oracle.brute_mvc(g.n, g.row_ptr, g.col)[0] == size
    got, flags, _ = oracle.mvc(g.n, g.row_ptr, g.col)
    assert got == size
    assert oracle.verify_cover(g.n, g.row_ptr, g.col, flags[:g.n])
    # {b, e, h} is the only minimum cover of this graph
    assert sorted(np.nonzero(flags[:g.n])[0].tolist()) == ids(spec["minimum_cover"])


@pytest.mark.gpu
def test_library_finds_the_papers_minimum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_18334_gb300 import build
    build.build()
    import paper_2512_18334_gb300 as vc
    g, spec = load()
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, cover, _ = vc.solve_min(dg)
    yes, _, _ = vc.solve_k(dg, 3)
    no, _, _ = vc.solve_k(dg, 2)
    dg.close()
    assert size == 3 and sorted(cover.tolist()) == ids(spec["minimum_cover"])
    assert yes and not no
