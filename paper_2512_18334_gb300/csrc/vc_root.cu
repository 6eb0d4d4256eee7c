// Root phase on the device: CSR validation, exhaustive root reduction, greedy
// upper bound and the induced-subgraph build (Section 4.2, which the paper
// runs on the CPU; here it is one thread block per query).
//
// Rules (Section 2.2), applied in synchronous rounds from one snapshot of the
// degrees.  A vertex u is "marked" for the cover when
//   degree-one:  some v with d(v) = 1 has u as its only neighbour
//                (if u also has d(u) = 1, only the lower endpoint's rule fires),
//   triangle:    some v with d(v) = 2 has neighbours u, w that are adjacent
//                (only the lowest-index degree-two vertex of a triangle fires),
//   high-degree: d(u) > b with b = bound - |F| - 1 (phase 2 only).
// All marks of a round go into the cover together; the tie-breaks keep the
// simultaneous application exact (no K2 or triangle gets every vertex).
// Phase 1 uses only the first two rules (they need no bound), then a greedy
// cover gives the bound, then phase 2 adds the high-degree rule.
#include <climits>

#include "vc_common.cuh"

namespace vcg {

// ------------------------------------------------------------ validation

__device__ __forceinline__ bool bsearch_row(const int *row, int len, int key)
{
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = __ldg(row + mid);
        if (x == key) return true;
        if (x < key) lo = mid + 1; else hi = mid - 1;
    }
    return false;
}

// Grid-stride checks of the CSR contract.  err[0] collects failures,
// err[1] counts entries (v, u) with u > v.
__global__ void validate_rowptr_kernel(int n, int m2, const int *rp, int *err)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        int a = rp[v];
        bool bad = (v == 0 && a != 0) || (v == n && a != m2) || a < 0 || a > m2;
        if (v < n && rp[v + 1] < a) bad = true;
        if (bad) atomicOr(err, 1);
    }
}

__global__ void validate_col_kernel(int n, const int *rp, const int *col, int *err)
{
    if (*(volatile int *)err) return;   // row pointers are bad: rows cannot be read safely
    int up = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int a = rp[v], b = rp[v + 1];
        int prev = -1;
        bool bad = false;
        for (int e = a; e < b && !bad; e++) {
            int u = col[e];
            if (u < 0 || u >= n || u == v || u <= prev) { bad = true; break; }
            prev = u;
            if (u > v) {
                up++;
                if (!bsearch_row(col + rp[u], rp[u + 1] - rp[u], v)) bad = true;
            }
        }
        if (bad) atomicOr(err, 1);
    }
    up = __reduce_add_sync(kFull, up);
    if ((threadIdx.x & 31) == 0 && up) atomicAdd(err + 1, up);
}

// ------------------------------------------------------------ root kernel

constexpr int kRootThreads = 1024;

struct RootShared {
    int cnt;        // marks in this round
    int fcnt;       // next-frontier size
    int forced;
    int delta;      // max live degree seen in the last full scan
    int red[33];
    int flag;
};

__device__ __forceinline__ int block_sum(int x, int *red)
{
    x = __reduce_add_sync(kFull, x);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    if (w == 0) {
        int y = l < nw ? red[l] : 0;
        y = __reduce_add_sync(kFull, y);
        if (l == 0) red[32] = y;
    }
    __syncthreads();
    return red[32];
}

__device__ __forceinline__ int block_max(int x, int *red)
{
    x = __reduce_max_sync(kFull, x);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    if (w == 0) {
        int y = l < nw ? red[l] : INT_MIN;
        y = __reduce_max_sync(kFull, y);
        if (l == 0) red[32] = y;
    }
    __syncthreads();
    return red[32];
}

// exclusive scan of one value per thread (block-wide); returns the prefix and
// the total in *tot
__device__ __forceinline__ int block_excl_scan(int x, int *red, int *tot)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    int inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, inc, o);
        if (l >= o) inc += y;
    }
    __syncthreads();
    if (l == 31) red[w] = inc;
    __syncthreads();
    if (w == 0) {
        int y = l < nw ? red[l] : 0, s = y;
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(kFull, s, o);
            if (l >= o) s += z;
        }
        if (l < nw) red[l] = s - y;
        if (l == 31) red[32] = s;
    }
    __syncthreads();
    int r = red[w] + inc - x;
    *tot = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Queue u for the cover (once per round).
__device__ __forceinline__ void root_mark(const QueryDesc &Q, RootShared &sh, int u)
{
    if (atomicExch(&Q.aux[u], 1) == 0) {
        int pos = atomicAdd(&sh.cnt, 1);
        Q.forced_list[sh.forced + pos] = u;
    }
}

__device__ __forceinline__ void root_push_frontier(const QueryDesc &Q, RootShared &sh, int *next, int x)
{
    if (atomicExch(&Q.flag[x], 1) == 0) next[atomicAdd(&sh.fcnt, 1)] = x;
}

// Examine vertex v against the rules; marks go to the round's list.
__device__ __forceinline__ void root_examine(const QueryDesc &Q, RootShared &sh, int *next, int v,
                                             int bud)
{
    if (Q.st[v] != 0) return;
    const int d = Q.deg[v];
    if (d == 0) return;
    const int *col = Q.col;
    const int a = Q.rp[v], b = Q.rp[v + 1];
    if (d == 1) {
        int u = -1;
        for (int e = a; e < b; e++) {
            int x = col[e];
            if (Q.st[x] == 0 && Q.deg[x] > 0) { u = x; break; }
        }
        if (u >= 0) {
            if (Q.deg[u] == 1 && u < v) root_push_frontier(Q, sh, next, u);  // u's rule fires
            else root_mark(Q, sh, u);
        }
    } else if (d == 2) {
        int u = -1, w = -1;
        for (int e = a; e < b; e++) {
            int x = col[e];
            if (Q.st[x] == 0 && Q.deg[x] > 0) {
                if (u < 0) u = x; else { w = x; break; }
            }
        }
        if (w >= 0 && bsearch_row(col + Q.rp[u], Q.rp[u + 1] - Q.rp[u], w)) {
            int p = INT_MAX;
            if (Q.deg[u] == 2 && u < v) p = u;
            if (Q.deg[w] == 2 && w < v && w < p) p = w;
            if (p != INT_MAX) root_push_frontier(Q, sh, next, p);
            else { root_mark(Q, sh, u); root_mark(Q, sh, w); }
        }
    }
    if (d > bud) root_mark(Q, sh, v);
}

// Rounds of the rules until nothing is marked.  hd: use the high-degree rule
// with budget bound - forced - 1.  Returns false when the budget went negative
// (no cover smaller than `bound` can exist).
__device__ bool root_reduce_rounds(QueryDesc &Q, RootShared &sh, bool hd, int bound)
{
    const int n = Q.n;
    int *cur = Q.fr0, *next = Q.fr1;
    int fsize = -1;   // -1: full scan
    for (;;) {
        const int bud = hd ? bound - sh.forced - 1 : INT_MAX;
        if (hd && bud < 0) return false;
        bool full = fsize < 0 || (hd && sh.delta > bud);
        __syncthreads();
        if (threadIdx.x == 0) { sh.cnt = 0; sh.fcnt = 0; }
        __syncthreads();
        int dmax = 0;
        if (full) {
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                Q.flag[v] = 0;
                if (Q.st[v] == 0) dmax = max(dmax, Q.deg[v]);
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) root_examine(Q, sh, next, v, bud);
        } else {
            for (int i = threadIdx.x; i < fsize; i += blockDim.x) Q.flag[cur[i]] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < fsize; i += blockDim.x) root_examine(Q, sh, next, cur[i], bud);
        }
        if (full) {
            int dm = block_max(dmax, sh.red);
            if (threadIdx.x == 0) sh.delta = dm;
        }
        __syncthreads();
        const int cnt = sh.cnt;
        const int base = sh.forced;
        if (cnt == 0) {
            if (sh.fcnt == 0) return true;
            // only tie-break partners were queued: examine them next round
        }
        // apply: lower the degrees of the marked vertices' live neighbours
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            int u = Q.forced_list[base + i];
            for (int e = Q.rp[u]; e < Q.rp[u + 1]; e++) {
                int x = Q.col[e];
                if (Q.st[x] == 0 && Q.aux[x] == 0 && Q.deg[x] > 0) {
                    atomicSub(&Q.deg[x], 1);
                    root_push_frontier(Q, sh, next, x);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            int u = Q.forced_list[base + i];
            Q.st[u] = 1;
            Q.deg[u] = 0;
            Q.aux[u] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) sh.forced = base + cnt;
        fsize = sh.fcnt;
        int *t = cur; cur = next; next = t;
        __syncthreads();
        if (fsize == 0 && !(hd && sh.delta > bound - sh.forced - 1)) return true;
    }
}

// Greedy cover of the live graph: the complement of a maximal independent
// set chosen by static priority (degree, hash(id)), lowest first.  aux[v]:
// 0 undecided, 1 in the independent set, 2 in the cover.  Returns the number
// of live vertices put in the cover; flags them in cover_flags.
__device__ int root_greedy(QueryDesc &Q, RootShared &sh)
{
    const int n = Q.n;
    for (int v = threadIdx.x; v < n; v += blockDim.x)
        Q.aux[v] = (Q.st[v] == 0 && Q.deg[v] > 0) ? 0 : 3;   // 3: not part of the live graph
    __syncthreads();
    for (int round = 0;; round++) {
        __syncthreads();
        if (threadIdx.x == 0) sh.flag = 0;
        __syncthreads();
        // a vertex joins when every undecided neighbour has a larger priority
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            if (Q.aux[v] != 0) continue;
            const unsigned long long pv =
                ((unsigned long long)Q.deg[v] << 32) | mix32((unsigned)v);
            bool join = true;
            for (int e = Q.rp[v]; e < Q.rp[v + 1] && join; e++) {
                int x = Q.col[e];
                int ax = Q.aux[x];
                if (ax == 1 || ax == 4) join = false;
                else if (ax == 0) {
                    unsigned long long px = ((unsigned long long)Q.deg[x] << 32) | mix32((unsigned)x);
                    if (px < pv || (px == pv && x < v)) join = false;
                }
            }
            if (join) Q.fr0[v] = 1; else Q.fr0[v] = 0;
        }
        __syncthreads();
        for (int v = threadIdx.x; v < n; v += blockDim.x)
            if (Q.aux[v] == 0 && Q.fr0[v]) { Q.aux[v] = 4; sh.flag = 1; }   // 4: joined this round
        __syncthreads();
        if (!sh.flag) break;
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            if (Q.aux[v] != 4) continue;
            for (int e = Q.rp[v]; e < Q.rp[v + 1]; e++) {
                int x = Q.col[e];
                if (Q.aux[x] == 0) Q.aux[x] = 2;
            }
        }
        __syncthreads();
        for (int v = threadIdx.x; v < n; v += blockDim.x)
            if (Q.aux[v] == 4) Q.aux[v] = 1;
    }
    __syncthreads();
    int c = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        bool in = Q.st[v] == 1 || Q.aux[v] == 2 || Q.aux[v] == 0;
        Q.cover_flags[v] = in ? 1 : 0;
        if (Q.aux[v] == 2 || Q.aux[v] == 0) c++;
    }
    int tot = block_sum(c, sh.red);
    for (int v = threadIdx.x; v < n; v += blockDim.x) Q.aux[v] = 0;
    __syncthreads();
    return tot;
}

// Induce the subgraph on the live vertices with non-zero degree, relabelled
// in increasing original id (so rows stay sorted).
__device__ void root_induce(QueryDesc &Q, RootShared &sh)
{
    const int n = Q.n;
    const int T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int beg = min(n, threadIdx.x * chunk), end = min(n, beg + chunk);
    int cnt = 0, dsum = 0, dmax = 0;
    for (int v = beg; v < end; v++) {
        if (Q.st[v] == 0 && Q.deg[v] > 0) { cnt++; dsum += Q.deg[v]; dmax = max(dmax, Q.deg[v]); }
    }
    int np, m2p;
    int off = block_excl_scan(cnt, sh.red, &np);
    int eoff = block_excl_scan(dsum, sh.red, &m2p);
    int dm = block_max(dmax, sh.red);
    int id = off, eo = eoff;
    for (int v = beg; v < end; v++) {
        if (Q.st[v] == 0 && Q.deg[v] > 0) {
            Q.aux[v] = id;       // new id
            Q.orig[id] = v;
            Q.rp2[id] = eo;
            id++;
            eo += Q.deg[v];
        } else {
            Q.aux[v] = -1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Q.rp2[np] = m2p;
        Q.np = np;
        Q.m2p = m2p;
        Q.maxdeg = dm;
    }
    for (int i = threadIdx.x; i < np; i += T) {
        int v = Q.orig[i];
        int o = Q.rp2[i];
        for (int e = Q.rp[v]; e < Q.rp[v + 1]; e++) {
            int x = Q.col[e];
            int nx = Q.aux[x];
            if (nx >= 0) Q.col2[o++] = nx;
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += T) Q.aux[v] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(kRootThreads) root_kernel(QueryDesc *qs)
{
    __shared__ RootShared sh;
    QueryDesc &Q = qs[blockIdx.x];
    if (Q.status != VC_OK) return;
    const int n = Q.n;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        Q.deg[v] = Q.rp[v + 1] - Q.rp[v];
        Q.st[v] = 0;
        Q.aux[v] = 0;
        Q.flag[v] = 0;
        Q.cover_flags[v] = 0;
    }
    if (threadIdx.x == 0) {
        sh.forced = 0;
        sh.delta = INT_MAX;
        Q.np = 0; Q.m2p = 0; Q.maxdeg = 0; Q.answered = 0; Q.greedy = -1;
        Q.improved = 0; Q.result = -1; Q.yes = 0; Q.cover_len = 0;
    }
    __syncthreads();

    // phase 1: degree-one and degree-two-triangle rules (need no bound)
    root_reduce_rounds(Q, sh, false, INT_MAX);
    int e2 = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x)
        if (Q.st[v] == 0) e2 += Q.deg[v];
    e2 = block_sum(e2, sh.red);
    if (e2 == 0) {
        // the rules alone produced a cover; they are exact, so it is minimum
        for (int v = threadIdx.x; v < n; v += blockDim.x) Q.cover_flags[v] = Q.st[v] == 1;
        if (threadIdx.x == 0) {
            Q.forced = sh.forced;
            Q.answered = 1;
            Q.bound = sh.forced;
            if (Q.k < 0) { Q.result = sh.forced; Q.yes = 1; }
            else { Q.yes = sh.forced <= Q.k; Q.result = Q.yes ? sh.forced : -1; }
        }
        return;
    }

    // initial upper bound (Algorithm 1: "an approximate minimum ... such as a greedy one")
    int g = root_greedy(Q, sh);
    const int greedy = sh.forced + g;
    if (threadIdx.x == 0) Q.greedy = greedy;
    if (Q.k >= 0 && greedy <= Q.k) {
        if (threadIdx.x == 0) {
            Q.forced = sh.forced; Q.answered = 1; Q.bound = greedy; Q.yes = 1; Q.result = greedy;
        }
        return;
    }
    // look only for covers smaller than `bound`
    const int bound = Q.k >= 0 ? Q.k + 1 : greedy;

    // phase 2: all three rules; high-degree budget b = bound - |F| - 1
    bool feasible = root_reduce_rounds(Q, sh, true, bound);
    e2 = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x)
        if (Q.st[v] == 0) e2 += Q.deg[v];
    e2 = block_sum(e2, sh.red);
    if (!feasible || sh.forced >= bound) {
        // no cover smaller than the bound exists
        if (threadIdx.x == 0) {
            Q.forced = sh.forced; Q.answered = 1; Q.bound = bound;
            if (Q.k < 0) { Q.result = greedy; Q.yes = 1; }   // greedy flags already hold it
            else { Q.yes = 0; Q.result = -1; }
        }
        return;
    }
    if (e2 == 0) {
        for (int v = threadIdx.x; v < n; v += blockDim.x) Q.cover_flags[v] = Q.st[v] == 1;
        if (threadIdx.x == 0) {
            Q.forced = sh.forced; Q.answered = 1; Q.bound = bound;
            Q.result = sh.forced; Q.yes = 1;
        }
        return;
    }
    root_induce(Q, sh);
    if (threadIdx.x == 0) { Q.forced = sh.forced; Q.bound = bound; }
}

// ------------------------------------------------------------ final answer

// Assemble each query's cover in original ids: the root-forced vertices plus
// the witness of the induced graph's registry entry when the search improved
// on the bound; otherwise the root phase's cover (greedy or forced set).
__global__ void __launch_bounds__(kRootThreads) finalize_kernel(QueryDesc *qs, const RegEntry *reg,
                                                                 const uint32_t *reg_words, int wcap)
{
    __shared__ int red[33];
    QueryDesc &Q = qs[blockIdx.x];
    if (Q.status != VC_OK) return;
    const int n = Q.n;
    if (!Q.answered) {
        const RegEntry &R = reg[Q.root_entry];
        const bool imp = R.has_w != 0;
        if (imp) {
            for (int v = threadIdx.x; v < n; v += blockDim.x) Q.cover_flags[v] = Q.st[v] == 1;
            __syncthreads();
            const uint32_t *w = reg_words + (size_t)Q.root_entry * wcap;
            for (int i = threadIdx.x; i < Q.np; i += blockDim.x)
                if (w[(i >> 5) - R.wlo] >> (i & 31) & 1u) Q.cover_flags[Q.orig[i]] = 1;
        }
        if (threadIdx.x == 0) {
            Q.improved = imp;
            if (Q.k < 0) {
                Q.result = imp ? Q.forced + R.val : Q.greedy;
                Q.yes = 1;
            } else {
                Q.yes = imp;
                Q.result = imp ? Q.forced + R.val : -1;
            }
        }
        __syncthreads();
    }
    // compact the cover flags into an ascending id list
    const int T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int beg = min(n, threadIdx.x * chunk), end = min(n, beg + chunk);
    const bool emit = Q.yes != 0;
    int c = 0;
    if (emit)
        for (int v = beg; v < end; v++) c += Q.cover_flags[v] != 0;
    int tot;
    int off = block_excl_scan(c, red, &tot);
    if (emit)
        for (int v = beg; v < end; v++)
            if (Q.cover_flags[v]) Q.cover_list[off++] = v;
    if (threadIdx.x == 0) Q.cover_len = emit ? tot : 0;
}

}  // namespace vcg

// ------------------------------------------------------------ host wrappers

#include "vc_internal.h"

namespace vcg {

cudaError_t validate_run(int n, int m2, const int *rp, const int *col, int *d_err, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_err, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = (n + 1 + threads - 1) / threads < 4096 ? (n + 1 + threads - 1) / threads : 4096;
    validate_rowptr_kernel<<<blocks > 0 ? blocks : 1, threads, 0, s>>>(n, m2, rp, d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n > 0) {
        validate_col_kernel<<<blocks > 0 ? blocks : 1, threads, 0, s>>>(n, rp, col, d_err);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t root_run(QueryDesc *d_q, int nq, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    root_kernel<<<nq, kRootThreads, 0, s>>>(d_q);
    return cudaGetLastError();
}

cudaError_t finalize_run(QueryDesc *d_q, int nq, const RegEntry *reg, const uint32_t *reg_words, int wcap,
                         cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    finalize_kernel<<<nq, kRootThreads, 0, s>>>(d_q, reg, reg_words, wcap);
    return cudaGetLastError();
}

}  // namespace vcg
