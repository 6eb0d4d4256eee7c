/*
 * CPU oracle for exact vertex cover -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call this file.  The CUDA solver shares no
 * code, header, table or helper with it.
 *
 * Everything here is plain, sequential and slow on purpose, written from the
 * paper "Faster Vertex Cover Algorithms on GPUs with Component-Aware Parallel
 * Branching" (arXiv 2512.18334):
 *
 *   orc_verify_cover   definition of a vertex cover            (Section 2.1)
 *   orc_brute_mvc      MVC by its definition: the smallest cover, found by
 *                      enumerating subsets in increasing size  (Section 2.1)
 *   orc_greedy         the initial upper bound: the size of some cover
 *                      found quickly and without optimality    (Section 2.2)
 *   orc_mvc            Algorithm 2 (component-aware branch-and-reduce), with
 *                      the three reduction rules of Section 2.2, the stopping
 *                      condition of Algorithm 1/2, and the clique and
 *                      chordless-cycle component rules of Section 3.4
 *   orc_pvc            the parameterized problem (Section 2.1, 2.2): MVC run
 *                      with best = k + 1; answer yes iff a cover <= k exists
 *   orc_max_matching   Hopcroft-Karp maximum matching on a bipartite graph;
 *                      with Koenig's theorem it pins OPT on bipartite inputs
 *   orc_rule_violation which reduction rule of Section 2.2 still applies to a
 *                      graph (used to check that a reduced graph is a fixpoint)
 *
 * Readings of points where the paper is silent or garbled (each is listed in
 * the design notes):
 *   - stopping condition: prune when |S| >= best or |E| > b*b with
 *     b = best - |S| - 1 (Algorithm 1 prints b this way; the prose of
 *     Section 2.2 prints the sign reversed, which cannot be meant).
 *   - high-degree rule: add v when d(v) > b, same b.
 *   - reduce() sweeps the vertices in ascending order, trying degree-one, then
 *     degree-two-triangle, then high-degree at each vertex, and repeats the
 *     sweep until nothing changes.
 *   - v_max is the lowest-index vertex of maximum degree.
 *   - component children get best_i = min(best - sum, |V_i| - 1) in order of
 *     their smallest vertex (Algorithm 2 as printed, sequential).
 *   - the clique / cycle rules are applied to each component of a branch on
 *     components (Section 3.4 introduces them for that case).
 *
 * ORC_MUTANT (compile-time, default 0) plants one known mistake so that the
 * pin tests can show they catch it; the normal build never defines it.
 *
 * Graph input: CSR (row_ptr[n+1], col[row_ptr[n]]), simple and symmetric.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EBUDGET (-2)
#define ORC_ENOMEM (-3)
#define ORC_EARG (-4)

/* --------------------------------------------------------------- definition */

/* 1 iff every edge uv has u or v in the cover (cover[v] != 0). */
int orc_verify_cover(int n, const int32_t *rp, const int32_t *col, const uint8_t *cover)
{
    for (int v = 0; v < n; v++) {
        if (cover[v]) continue;
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            if (!cover[col[e]]) return 0;
#if ORC_MUTANT == 8
            return 1;   /* planted: stops after the first edge it checks */
#endif
        }
    }
    return 1;
}

/* Minimum vertex cover by definition: try every subset of size 0, 1, 2, ...
 * and return the first size that covers every edge.  n <= 30. */
int orc_brute_mvc(int n, const int32_t *rp, const int32_t *col, uint8_t *out_cover)
{
    if (n < 0 || n > 30) return ORC_EARG;
    uint32_t adj[30];
    for (int v = 0; v < n; v++) {
        adj[v] = 0;
        for (int e = rp[v]; e < rp[v + 1]; e++) adj[v] |= 1u << col[e];
    }
    for (int k = 0; k <= n; k++) {
        /* all n-bit masks with k bits set, in increasing order (Gosper) */
        uint64_t limit = 1ull << n;
        uint64_t s = (k == 0) ? 0 : ((1ull << k) - 1);
        while (s < limit) {
            uint32_t mask = (uint32_t)s;
            int ok = 1;
            for (int v = 0; v < n && ok; v++)
                if (!(mask >> v & 1u) && (adj[v] & ~mask)) ok = 0;
            if (ok) {
                if (out_cover)
                    for (int v = 0; v < n; v++) out_cover[v] = (uint8_t)(mask >> v & 1u);
                return k;
            }
            if (k == 0) break;
            uint64_t c = s & (~s + 1);
            uint64_t r = s + c;
            s = (((r ^ s) >> 2) / c) | r;
        }
    }
    return n; /* unreachable: the full set is a cover */
}

/* ------------------------------------------------------------ graph state */

/* A search-tree node's graph: the vertices still in G and their degrees in G.
 * in_g[v]  = 1 iff v is a vertex of G (not yet removed),
 * deg[v]   = number of neighbours u of v with in_g[u] (valid when in_g[v]),
 * in_s[v]  = 1 iff v was put in S by this node or its ancestors (in the
 *            current component context).                                     */
typedef struct {
    int n;
    const int32_t *rp, *col;
    long long nodes, node_budget;
    long long comp_branches;
    int stop; /* budget exhausted */
} orc_ctx;

typedef struct {
    uint8_t *in_g;
    uint8_t *in_s;
    int32_t *deg;
    int s_size;
} orc_state;

static int state_alloc(orc_state *st, int n)
{
    size_t sz = (size_t)(n > 0 ? n : 1);
    st->in_g = (uint8_t *)malloc(sz);
    st->in_s = (uint8_t *)malloc(sz);
    st->deg = (int32_t *)malloc(sz * sizeof(int32_t));
    st->s_size = 0;
    return (st->in_g && st->in_s && st->deg) ? ORC_OK : ORC_ENOMEM;
}

static void state_free(orc_state *st)
{
    free(st->in_g); free(st->in_s); free(st->deg);
}

static void state_copy(orc_state *dst, const orc_state *src, int n)
{
    memcpy(dst->in_g, src->in_g, (size_t)n);
    memcpy(dst->in_s, src->in_s, (size_t)n);
    memcpy(dst->deg, src->deg, (size_t)n * sizeof(int32_t));
    dst->s_size = src->s_size;
}

/* G - {v}, S + {v} */
static void put_in_cover(const orc_ctx *cx, orc_state *st, int v)
{
    st->in_g[v] = 0;
    st->in_s[v] = 1;
    st->s_size++;
    for (int e = cx->rp[v]; e < cx->rp[v + 1]; e++) {
        int u = cx->col[e];
        if (st->in_g[u]) st->deg[u]--;
    }
    st->deg[v] = 0;
}

static long long edge_count(const orc_ctx *cx, const orc_state *st)
{
    long long twice = 0;
    for (int v = 0; v < cx->n; v++)
        if (st->in_g[v]) twice += st->deg[v];
    return twice / 2;
}

static int adjacent(const orc_ctx *cx, int a, int b)
{
    for (int e = cx->rp[a]; e < cx->rp[a + 1]; e++)
        if (cx->col[e] == b) return 1;
    return 0;
}

/* The live neighbours of v (at most `cap` of them) into out[]; returns count. */
static int live_neighbours(const orc_ctx *cx, const orc_state *st, int v, int *out, int cap)
{
    int c = 0;
    for (int e = cx->rp[v]; e < cx->rp[v + 1] && c < cap; e++) {
        int u = cx->col[e];
        if (st->in_g[u]) out[c++] = u;
    }
    return c;
}

/* reduce(G, S, best) of Algorithm 1/2 with the three rules of Section 2.2,
 * repeated until no rule applies (or until |S| >= best, where the branch is
 * dead anyway). */
static void reduce(const orc_ctx *cx, orc_state *st, int best)
{
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int v = 0; v < cx->n; v++) {
            if (st->s_size >= best) return;
            if (!st->in_g[v] || st->deg[v] == 0) continue;
            int nb[2];
            if (st->deg[v] == 1) {                 /* degree-one rule */
                live_neighbours(cx, st, v, nb, 1);
#if ORC_MUTANT == 1
                put_in_cover(cx, st, v);         /* planted mistake: the leaf */
#else
                put_in_cover(cx, st, nb[0]);
#endif
                changed = 1;
            } else if (st->deg[v] == 2) {          /* degree-two-triangle rule */
                live_neighbours(cx, st, v, nb, 2);
#if ORC_MUTANT == 2
                if (1) {                         /* planted mistake: no triangle test */
#else
                if (adjacent(cx, nb[0], nb[1])) {
#endif
                    put_in_cover(cx, st, nb[0]);
                    put_in_cover(cx, st, nb[1]);
                    changed = 1;
                }
            }
            if (st->in_g[v] && st->deg[v] > 0) {   /* high-degree rule */
                int b = best - st->s_size - 1;
#if ORC_MUTANT == 3
                b -= 1;                          /* planted mistake: threshold off by one */
#endif
                if (st->deg[v] > b) {
                    put_in_cover(cx, st, v);
                    changed = 1;
                }
            }
        }
    }
}

/* Connected components of the vertices of G with non-zero degree (BFS).
 * comp[v] = component id (0..count-1) in order of smallest vertex, -1 else. */
static int find_components(const orc_ctx *cx, const orc_state *st, int32_t *comp, int32_t *queue)
{
    int count = 0;
    for (int v = 0; v < cx->n; v++) comp[v] = -1;
    for (int s = 0; s < cx->n; s++) {
        if (!st->in_g[s] || st->deg[s] == 0 || comp[s] >= 0) continue;
        int head = 0, tail = 0;
        queue[tail++] = s;
        comp[s] = count;
        while (head < tail) {
            int v = queue[head++];
            for (int e = cx->rp[v]; e < cx->rp[v + 1]; e++) {
                int u = cx->col[e];
                if (st->in_g[u] && comp[u] < 0) {
                    comp[u] = count;
                    queue[tail++] = u;
                }
            }
        }
        count++;
    }
    return count;
}

/* Algorithm 2.  `best` and `best_cover` play the role of the by-reference
 * best; `best_cover` holds a cover of the current component context of size
 * `*best` whenever `*best_has_cover` is set. */
static void mvc(orc_ctx *cx, orc_state *g, int *best, uint8_t *best_cover, int *best_has_cover,
                int use_components)
{
    const int n = cx->n;
    if (cx->stop) return;
    if (++cx->nodes > cx->node_budget) { cx->stop = 1; return; }

    reduce(cx, g, *best);
    long long m = edge_count(cx, g);
    long long b = (long long)*best - g->s_size - 1;
#if ORC_MUTANT == 4
    b -= 1;                                                /* planted mistake */
#endif
    if (g->s_size >= *best || m > b * b) return;          /* stopping condition */
    if (m == 0) {                                          /* new best cover */
        *best = g->s_size;
        memcpy(best_cover, g->in_s, (size_t)n);
        *best_has_cover = 1;
        return;
    }

    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!comp || !queue) { free(comp); free(queue); cx->stop = 1; return; }
    int ncomp = use_components ? find_components(cx, g, comp, queue) : 1;

    if (ncomp <= 1) {
        /* branch on a vertex of maximum degree (lowest index among ties) */
        int vmax = -1;
        for (int v = 0; v < n; v++)
            if (g->in_g[v] && (vmax < 0 || g->deg[v] > g->deg[vmax])) vmax = v;
        free(comp); free(queue);
        orc_state child;
        if (state_alloc(&child, n) != ORC_OK) { state_free(&child); cx->stop = 1; return; }
        state_copy(&child, g, n);
        put_in_cover(cx, &child, vmax);                     /* G - v_max */
        mvc(cx, &child, best, best_cover, best_has_cover, use_components);
        state_copy(&child, g, n);                           /* G - N(v_max) */
        for (int e = cx->rp[vmax]; e < cx->rp[vmax + 1]; e++) {
            int u = cx->col[e];
            if (child.in_g[u]) put_in_cover(cx, &child, u);
        }
        mvc(cx, &child, best, best_cover, best_has_cover, use_components);
        state_free(&child);
        return;
    }

    /* branch on components */
    cx->comp_branches++;
    int sum = g->s_size;
#if ORC_MUTANT == 5
    sum = 0;                                               /* planted mistake: S dropped */
#endif
    uint8_t *acc = (uint8_t *)malloc((size_t)n);           /* S plus each component's cover */
    uint8_t *cov_i = (uint8_t *)malloc((size_t)n);
    orc_state child;
    int ok = acc && cov_i && state_alloc(&child, n) == ORC_OK;
    if (!ok) { free(acc); free(cov_i); state_free(&child); free(comp); free(queue); cx->stop = 1; return; }
    memcpy(acc, g->in_s, (size_t)n);

    for (int i = 0; i < ncomp && !cx->stop; i++) {
        int size_i = 0, last = -1, clique = 1, cyc = 1;
        for (int v = 0; v < n; v++)
            if (comp[v] == i) { size_i++; last = v; }
        for (int v = 0; v < n; v++) {
            if (comp[v] != i) continue;
            if (g->deg[v] != size_i - 1) clique = 0;
            if (g->deg[v] != 2) cyc = 0;
        }
        int best_i = (*best - sum < size_i - 1) ? (*best - sum) : (size_i - 1);
        int has_i = (best_i == size_i - 1);
        /* the achievable starting cover: every vertex of the component but one */
        memset(cov_i, 0, (size_t)n);
        for (int v = 0; v < n; v++)
            if (comp[v] == i && v != last) cov_i[v] = 1;

        if (clique || cyc) {
            /* Section 3.4: a clique needs |C|-1 vertices (all but one), a
             * chordless cycle needs ceil(|C|/2) (every other vertex). */
            int need = clique ? size_i - 1 : (size_i + 1) / 2;
#if ORC_MUTANT == 6
            if (!clique) need = size_i / 2;              /* planted mistake: floor */
#endif
#if ORC_MUTANT == 7
            if (clique) need = size_i - 2;               /* planted mistake: one too few */
#endif
            if (need < best_i) {
                best_i = need;
                has_i = 1;
                memset(cov_i, 0, (size_t)n);
                if (clique) {
                    for (int v = 0; v < n; v++)
                        if (comp[v] == i && v != last) cov_i[v] = 1;
                } else {
                    /* walk the cycle from its smallest vertex, take every other */
                    int start = -1;
                    for (int v = 0; v < n && start < 0; v++)
                        if (comp[v] == i) start = v;
                    int prev = -1, cur = start, k = 0;
                    do {
                        if (k % 2 == 0) cov_i[cur] = 1;
                        int next = -1;
                        for (int e = cx->rp[cur]; e < cx->rp[cur + 1]; e++) {
                            int u = cx->col[e];
                            if (comp[u] == i && u != prev) { next = u; break; }
                        }
                        prev = cur; cur = next; k++;
                    } while (cur != start && cur >= 0);
                }
            }
        } else if (best_i > 0) {
            /* MVC(G_i, {}, best_i) */
            for (int v = 0; v < n; v++) {
                child.in_g[v] = (uint8_t)(comp[v] == i);
                child.in_s[v] = 0;
                child.deg[v] = (comp[v] == i) ? g->deg[v] : 0;
            }
            child.s_size = 0;
            mvc(cx, &child, &best_i, cov_i, &has_i, use_components);
        }
        sum += best_i;
        if (has_i)
            for (int v = 0; v < n; v++) acc[v] |= cov_i[v];
    }
    if (!cx->stop && sum < *best) {
        *best = sum;
        memcpy(best_cover, acc, (size_t)n);
        *best_has_cover = 1;
    }
    free(acc); free(cov_i); state_free(&child); free(comp); free(queue);
}

/* Greedy cover: repeatedly take a vertex of maximum degree (lowest index). */
int orc_greedy(int n, const int32_t *rp, const int32_t *col, uint8_t *out_cover)
{
    orc_ctx cx = {n, rp, col, 0, 0, 0, 0};
    orc_state st;
    if (state_alloc(&st, n) != ORC_OK) { state_free(&st); return ORC_ENOMEM; }
    for (int v = 0; v < n; v++) {
        st.in_g[v] = 1; st.in_s[v] = 0; st.deg[v] = rp[v + 1] - rp[v];
    }
    st.s_size = 0;
    for (;;) {
        int vmax = -1;
        for (int v = 0; v < n; v++)
            if (st.in_g[v] && st.deg[v] > 0 && (vmax < 0 || st.deg[v] > st.deg[vmax])) vmax = v;
        if (vmax < 0) break;
        put_in_cover(&cx, &st, vmax);
    }
    int size = st.s_size;
    if (out_cover) memcpy(out_cover, st.in_s, (size_t)n);
    state_free(&st);
    return size;
}

/* Exact minimum vertex cover by Algorithm 2, seeded with the greedy bound.
 * Returns the size (>= 0) and a cover in out_cover; ORC_EBUDGET when more
 * than node_budget search-tree nodes would be needed.  stats (nullable):
 * [0] nodes visited, [1] branches on components.  use_components = 0 runs
 * Algorithm 1 instead (no component branching). */
int orc_mvc(int n, const int32_t *rp, const int32_t *col, long long node_budget,
            int use_components, uint8_t *out_cover, long long *stats)
{
    if (n < 0) return ORC_EARG;
    orc_ctx cx = {n, rp, col, 0, node_budget > 0 ? node_budget : (1ll << 62), 0, 0};
    uint8_t *cover = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    orc_state root;
    if (!cover || state_alloc(&root, n) != ORC_OK) { free(cover); return ORC_ENOMEM; }
    int best = orc_greedy(n, rp, col, cover);
    int has = 1;
    for (int v = 0; v < n; v++) {
        root.in_g[v] = 1; root.in_s[v] = 0; root.deg[v] = rp[v + 1] - rp[v];
    }
    root.s_size = 0;
    mvc(&cx, &root, &best, cover, &has, use_components);
    state_free(&root);
    if (stats) { stats[0] = cx.nodes; stats[1] = cx.comp_branches; }
    if (cx.stop) { free(cover); return ORC_EBUDGET; }
    if (out_cover) memcpy(out_cover, cover, (size_t)n);
    free(cover);
    return best;
}

/* Parameterized vertex cover: is there a cover of size <= k?  Runs the MVC
 * search with best = k + 1, i.e. looking only for covers smaller than k + 1.
 * Returns 1 (yes, cover of size <= k in out_cover), 0 (no), or an error. */
int orc_pvc(int n, const int32_t *rp, const int32_t *col, int k, long long node_budget,
            uint8_t *out_cover, int *out_size, long long *stats)
{
    if (n < 0 || k < 0) return ORC_EARG;
    orc_ctx cx = {n, rp, col, 0, node_budget > 0 ? node_budget : (1ll << 62), 0, 0};
    uint8_t *cover = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    orc_state root;
    if (!cover || state_alloc(&root, n) != ORC_OK) { free(cover); return ORC_ENOMEM; }
    int best = k + 1, has = 0;
    for (int v = 0; v < n; v++) {
        root.in_g[v] = 1; root.in_s[v] = 0; root.deg[v] = rp[v + 1] - rp[v];
    }
    root.s_size = 0;
    mvc(&cx, &root, &best, cover, &has, 1);
    state_free(&root);
    if (stats) { stats[0] = cx.nodes; stats[1] = cx.comp_branches; }
    if (cx.stop) { free(cover); return ORC_EBUDGET; }
    int yes = has && best <= k;
    if (out_size) *out_size = yes ? best : -1;
    if (out_cover && yes) memcpy(out_cover, cover, (size_t)n);
    free(cover);
    return yes;
}

/* Which Section 2.2 rule still applies to the graph G = (V minus removed)?
 * b is the high-degree budget (a vertex with degree > b is reducible; pass a
 * negative b to skip that rule).  Returns -1 when G is a fixpoint, else
 * 4*v + r with r = 1 (degree one), 2 (degree-two triangle), 3 (high degree). */
long long orc_rule_violation(int n, const int32_t *rp, const int32_t *col,
                             const uint8_t *removed, long long b)
{
    for (int v = 0; v < n; v++) {
        if (removed[v]) continue;
        int d = 0, a = -1, c = -1;
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            int u = col[e];
            if (removed[u]) continue;
            if (d == 0) a = u; else if (d == 1) c = u;
            d++;
        }
        if (d == 1) return 4ll * v + 1;
        if (d == 2) {
            for (int e = rp[a]; e < rp[a + 1]; e++)
                if (col[e] == c) return 4ll * v + 2;
        }
        if (b >= 0 && d > 0 && d > b) return 4ll * v + 3;
    }
    return -1;
}

/* Hopcroft-Karp maximum matching.  Two-colours the graph first; returns -1
 * when it is not bipartite.  out_match (nullable): partner of each vertex or
 * -1.  Isolated vertices are fine. */
int orc_max_matching(int n, const int32_t *rp, const int32_t *col, int32_t *out_match)
{
    int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *mate = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *it = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!side || !q || !mate || !dist || !it || !stk) {
        free(side); free(q); free(mate); free(dist); free(it); free(stk);
        return ORC_ENOMEM;
    }
    for (int v = 0; v < n; v++) side[v] = -1;
    for (int s = 0; s < n; s++) {
        if (side[s] >= 0) continue;
        int h = 0, t = 0;
        q[t++] = s; side[s] = 0;
        while (h < t) {
            int v = q[h++];
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                int u = col[e];
                if (side[u] < 0) { side[u] = 1 - side[v]; q[t++] = u; }
                else if (side[u] == side[v]) {
                    free(side); free(q); free(mate); free(dist); free(it); free(stk);
                    return -1;
                }
            }
        }
    }
    for (int v = 0; v < n; v++) mate[v] = -1;
    const int INF = 0x3fffffff;
    int matching = 0;
    for (;;) {
        /* BFS layers from free left vertices */
        int h = 0, t = 0, found = 0;
        for (int v = 0; v < n; v++) {
            if (side[v] == 0 && mate[v] < 0) { dist[v] = 0; q[t++] = v; }
            else dist[v] = INF;
        }
        while (h < t) {
            int v = q[h++];
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                int u = col[e];
                int w = mate[u];
                if (w < 0) found = 1;
                else if (dist[w] == INF) { dist[w] = dist[v] + 1; q[t++] = w; }
            }
        }
        if (!found) break;
        /* DFS along layers from each free left vertex (iterative) */
        for (int v = 0; v < n; v++) it[v] = rp[v];
        for (int s = 0; s < n; s++) {
            if (side[s] != 0 || mate[s] >= 0) continue;
            int top = 0;
            stk[top++] = s;
            while (top > 0) {
                int v = stk[top - 1];
                int advanced = 0;
                while (it[v] < rp[v + 1]) {
                    int u = col[it[v]++];
                    int w = mate[u];
                    if (w < 0) {
                        /* augment along the stack: stk[0..top-1] are left vertices */
                        int cur = u;
                        for (int i = top - 1; i >= 0; i--) {
                            int lv = stk[i];
                            int prev = mate[lv];
                            mate[lv] = cur; mate[cur] = lv;
                            cur = prev;
                        }
                        matching++;
                        top = 0;
                        advanced = 1;
                        break;
                    }
                    if (dist[w] == dist[v] + 1) { stk[top++] = w; advanced = 1; break; }
                }
                if (!advanced) { dist[v] = INF; top--; }
            }
        }
    }
    if (out_match) for (int v = 0; v < n; v++) out_match[v] = mate[v];
    free(side); free(q); free(mate); free(dist); free(it); free(stk);
    return matching;
}
