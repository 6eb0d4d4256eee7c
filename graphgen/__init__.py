"""Seeded synthetic graph generators.

This module only draws graphs; it holds none of the vertex-cover method's
arithmetic.  Both the CPU oracle and the CUDA solver take their inputs from
here, and nothing here imports either of them.

Every graph is returned as a simple undirected graph in CSR form:
``row_ptr`` (int32, n+1 entries) and ``col`` (int32, row_ptr[n] entries), each
row sorted strictly ascending, symmetric, with no self-loops.  This is the
input contract of ``vc_load_csr``.

The workload shapes follow the paper's setting (sparse graphs of low density
that fragment during the search, Section 5.6 notes the method wins below about
10% density); the paper's own datasets are not available, so these seeded
families stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Graph", "from_edges", "edges_of", "relabel", "disjoint_union",
    "gnm", "gnp", "chung_lu", "component_heavy",
    "path", "cycle", "complete", "complete_bipartite", "petersen", "star",
    "random_forest", "random_bipartite_chung_lu",
    "batch_pvc_mix", "stream_requests",
]


@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [row_ptr[n]]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def from_edges(n: int, u, v, name: str = "") -> Graph:
    """Canonical CSR from an undirected edge list (drops loops and duplicates)."""
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    if u.size:
        if u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n:
            raise ValueError("edge endpoint out of range")
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * max(n, 1) + b)
    a = key // max(n, 1)
    b = key % max(n, 1)
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for int32 CSR")
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), name)


def edges_of(g: Graph):
    """Edge list (u < v) of a CSR graph."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    keep = src < dst
    return src[keep], dst[keep]


def relabel(g: Graph, seed: int) -> Graph:
    """The same graph with vertex ids permuted by a seeded permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    u, v = edges_of(g)
    return from_edges(g.n, perm[u], perm[v], g.name + f"/perm{seed}")


def disjoint_union(graphs, name: str = "") -> Graph:
    us, vs, off = [], [], 0
    for h in graphs:
        u, v = edges_of(h)
        us.append(u + off)
        vs.append(v + off)
        off += h.n
    if not us:
        return from_edges(0, [], [], name)
    return from_edges(off, np.concatenate(us), np.concatenate(vs), name)


# ---------------------------------------------------------------- random families

def gnm(n: int, m: int, seed: int) -> Graph:
    """Erdos-Renyi G(n, m): m distinct unordered pairs drawn uniformly."""
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("m exceeds n choose 2")
    rng = np.random.default_rng(seed)
    chosen = set()
    out_u, out_v = [], []
    while len(chosen) < m:
        k = m - len(chosen)
        u = rng.integers(0, n, size=2 * k + 8)
        v = rng.integers(0, n, size=2 * k + 8)
        for a, b in zip(u.tolist(), v.tolist()):
            if a == b:
                continue
            key = (a, b) if a < b else (b, a)
            if key in chosen:
                continue
            chosen.add(key)
            out_u.append(key[0])
            out_v.append(key[1])
            if len(chosen) == m:
                break
    return from_edges(n, out_u, out_v, f"gnm({n},{m},s{seed})")


def gnp(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p), each pair independently with probability p."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    return from_edges(n, iu[keep], ju[keep], f"gnp({n},{p},s{seed})")


def _chung_lu_weights(n: int, gamma: float, avg_deg: float, max_deg: float):
    # w_i proportional to (i + i0)^(-1/(gamma-1)); i0 is solved so that after
    # scaling to mean avg_deg the largest weight equals max_deg (or no shift
    # when the plain power law already stays below the cap).
    alpha = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def wts(i0):
        w = (idx + i0) ** (-alpha)
        return w * (avg_deg * n / w.sum())

    lo, hi = 1e-9, float(n)
    if wts(lo)[0] <= max_deg:
        return wts(lo)
    for _ in range(200):
        mid = math.sqrt(lo * hi) if lo > 0 else hi / 2
        if wts(mid)[0] > max_deg:
            lo = mid
        else:
            hi = mid
    return np.minimum(wts(hi), max_deg)


def chung_lu(n: int, gamma: float, avg_deg: float, max_deg: float, seed: int) -> Graph:
    """Chung-Lu power-law graph (fast edge-sampling form).

    Expected degrees w_i follow a power law with exponent ``gamma`` scaled to
    mean ``avg_deg`` and capped at ``max_deg``.  M ~ Poisson(sum(w)/2) edge
    draws pick both endpoints independently with probability w_i / sum(w);
    loops and repeated pairs are dropped.  Vertex ids are shuffled so degree
    does not correlate with index.
    """
    rng = np.random.default_rng(seed)
    w = _chung_lu_weights(n, gamma, avg_deg, max_deg)
    total = w.sum()
    M = rng.poisson(total / 2.0)
    p = w / total
    u = rng.choice(n, size=M, p=p)
    v = rng.choice(n, size=M, p=p)
    perm = rng.permutation(n)
    return from_edges(n, perm[u], perm[v], f"chung_lu({n},{gamma},{avg_deg},{max_deg},s{seed})")


def random_bipartite_chung_lu(na: int, nb: int, gamma: float, avg_deg: float,
                              max_deg: float, seed: int) -> Graph:
    """Bipartite power-law graph: sides [0, na) and [na, na+nb)."""
    rng = np.random.default_rng(seed)
    wa = _chung_lu_weights(na, gamma, avg_deg, max_deg)
    wb = _chung_lu_weights(nb, gamma, avg_deg * na / max(nb, 1), max_deg)
    M = rng.poisson(wa.sum())
    u = rng.choice(na, size=M, p=wa / wa.sum())
    v = na + rng.choice(nb, size=M, p=wb / wb.sum())
    g = from_edges(na + nb, u, v, f"bip_chung_lu({na},{nb},s{seed})")
    return g


def component_heavy(seed: int, copies: int = 256, copy_n: int = 48, p: float = 0.12,
                    chain: int = 32) -> Graph:
    """Disjoint copies of G(copy_n, p) hung on a path of articulation vertices.

    Vertices [0, chain) form a path.  Each copy gets 1-3 bridge edges, each
    from a random vertex of the copy to a uniformly chosen chain vertex.
    """
    rng = np.random.default_rng(seed)
    us = [np.arange(chain - 1)]
    vs = [np.arange(1, chain)]
    off = chain
    iu, ju = np.triu_indices(copy_n, 1)
    for _ in range(copies):
        keep = rng.random(iu.size) < p
        us.append(iu[keep] + off)
        vs.append(ju[keep] + off)
        nb = int(rng.integers(1, 4))
        us.append(rng.integers(0, copy_n, size=nb) + off)
        vs.append(rng.integers(0, chain, size=nb))
        off += copy_n
    return from_edges(off, np.concatenate(us), np.concatenate(vs),
                      f"component_heavy({copies}x{copy_n},{p},chain{chain},s{seed})")


# ---------------------------------------------------------------- closed forms

def path(n: int) -> Graph:
    a = np.arange(max(n - 1, 0))
    return from_edges(n, a, a + 1, f"P{n}")


def cycle(n: int) -> Graph:
    if n < 3:
        raise ValueError("cycle needs n >= 3")
    a = np.arange(n)
    return from_edges(n, a, (a + 1) % n, f"C{n}")


def complete(n: int) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    u = np.repeat(np.arange(a), b)
    v = a + np.tile(np.arange(b), a)
    return from_edges(a + b, u, v, f"K{a},{b}")


def star(leaves: int) -> Graph:
    return from_edges(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1),
                      f"S{leaves}")


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(10, e[:, 0], e[:, 1], "Petersen")


def random_forest(n: int, trees: int, seed: int) -> Graph:
    """Uniform random recursive forest: vertex i>=trees attaches to a random earlier vertex."""
    rng = np.random.default_rng(seed)
    us, vs = [], []
    for i in range(trees, n):
        us.append(i)
        vs.append(int(rng.integers(0, i)))
    perm = rng.permutation(n)
    return from_edges(n, perm[np.array(us, np.int64)] if us else [],
                      perm[np.array(vs, np.int64)] if vs else [], f"forest({n},{trees},s{seed})")


# ---------------------------------------------------------------- workload mixes

def batch_pvc_mix(count: int, seed: int, n_lo: int = 40, n_hi: int = 1500):
    """Mixed batch: n ~ U[n_lo, n_hi]; half G(n,p) with mean degree U[3,8],
    half Chung-Lu with exponent 2.5 (mean degree U[3,8], cap n/4)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = float(rng.uniform(3.0, 8.0))
        s = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            out.append(gnp_sparse(n, d / (n - 1), s))
        else:
            out.append(chung_lu(n, 2.5, d, max(4.0, n / 4.0), s))
    return out


def gnp_sparse(n: int, p: float, seed: int) -> Graph:
    """G(n, p) by geometric skipping over the pair list (O(n + m))."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if p <= 0 or total == 0:
        return from_edges(n, [], [], f"gnp({n},{p:.4g},s{seed})")
    # number of edges, then a uniform sample of that many distinct pairs
    m = int(rng.binomial(total, min(p, 1.0)))
    idx = rng.choice(total, size=m, replace=False) if m else np.zeros(0, np.int64)
    # unrank pair index k -> (i, j), i < j, row-major over the upper triangle
    k = idx.astype(np.float64)
    i = (n - 2 - np.floor(np.sqrt(-8 * k + 4 * n * (n - 1) - 7) / 2.0 - 0.5)).astype(np.int64)
    j = (idx + i + 1 - n * (n - 1) // 2 + (n - i) * ((n - i) - 1) // 2).astype(np.int64)
    return from_edges(n, i, j, f"gnp({n},{p:.4g},s{seed})")


def stream_requests(count: int, seed: int, rate: float, n_lo: int = 30, n_hi: int = 20000):
    """Served stream: Poisson arrivals at ``rate`` per second, n log-uniform on
    [n_lo, n_hi], Chung-Lu with exponent U[2.2, 3.0] and mean degree U[4, 10].
    Returns (arrival_seconds, list of (n, gamma, avg_deg, seed)) so that graphs
    can be drawn lazily."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    specs = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        specs.append((n, float(rng.uniform(2.2, 3.0)), float(rng.uniform(4.0, 10.0)),
                      int(rng.integers(0, 2**31 - 1))))
    return t, specs
