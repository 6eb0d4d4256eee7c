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
#include <algorithm>
#include <climits>
#include <map>
#include <mutex>
#include <set>

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

// Is key in the sorted global row[0, len)?  Eight probes at a time: each
// step loads eight evenly spaced entries together (one round trip) and
// keeps the gap that can hold key, so a 2,000-entry row takes three steps
// and a short scan instead of eleven dependent loads.
__device__ bool kary_find(const int *row, int len, int key)
{
    int lo = 0, hi = len;                      // key can only be in [lo, hi)
    while (hi - lo > 16) {
        const int step = (hi - lo) / 9;        // >= 1
        int xs[8];
#pragma unroll
        for (int j = 0; j < 8; j++) xs[j] = __ldg(row + lo + (j + 1) * step);
        int below = 0;
        bool hit = false;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            below += xs[j] < key;
            hit |= xs[j] == key;
        }
        if (hit) return true;
        // the first `below` probes are < key, the rest > key
        const int nlo = below == 0 ? lo : lo + below * step + 1;
        const int nhi = below == 8 ? hi : lo + (below + 1) * step;
        lo = nlo;
        hi = nhi;
    }
    for (int e0 = lo; e0 < hi; e0 += 8) {
        int xs[8];
#pragma unroll
        for (int j = 0; j < 8; j++) xs[j] = e0 + j < hi ? __ldg(row + e0 + j) : -1;
        bool hit = false;
#pragma unroll
        for (int j = 0; j < 8; j++) hit |= xs[j] == key;
        if (hit) return true;
    }
    return false;
}

// The largest i in [lo, hi] with a[i] <= key, for a non-decreasing global
// array with a[lo] <= key; eight probes a step as in kary_find.
__device__ int kary_last_le(const int *a, int lo, int hi, int key)
{
    while (hi - lo >= 16) {
        const int step = (hi - lo) / 9;        // >= 1
        int xs[8];
#pragma unroll
        for (int j = 0; j < 8; j++) xs[j] = __ldg(a + lo + (j + 1) * step);
        int le = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) le += xs[j] <= key;
        // probes 1..le hold, the rest do not: the answer lies in
        // [lo + le * step, lo + (le + 1) * step - 1] (up to hi when all hold)
        const int nhi = le == 8 ? hi : lo + (le + 1) * step - 1;
        lo += le * step;
        hi = nhi;
    }
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= key) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Grid-stride checks of the CSR contract.  err[0] collects failures,
// err[1] counts entries (v, u) with u > v, err[2] is the maximum degree
// (row length; meaningful only when the row pointers are valid).
__global__ void validate_rowptr_kernel(int n, int m2, const int *rp, int *err)
{
    int dm = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        int a = rp[v];
        bool bad = (v == 0 && a != 0) || (v == n && a != m2) || a < 0 || a > m2;
        if (v < n) {
            const int b = rp[v + 1];
            if (b < a) bad = true;
            dm = max(dm, b - a);
        }
        if (bad) atomicOr(err, 1);
    }
    dm = __reduce_max_sync(kFull, dm);
    if ((threadIdx.x & 31) == 0 && dm) atomicMax(err + 2, dm);
}

// One entry per thread (edge-parallel, so a hub's long row is spread over
// many threads): entry e of row v must be in range, not v itself, larger
// than the entry before it in the row, and (when above the diagonal) mirrored
// in row col[e].  Needs valid row pointers (checked first).
__global__ void validate_col_kernel(int n, int m2, const int *rp, const int *col, int *err)
{
    if (*(volatile int *)err) return;   // row pointers are bad: rows cannot be read safely
    int up = 0;
    bool bad = false;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m2; e += gridDim.x * blockDim.x) {
        // the row holding e: the largest v with rp[v] <= e (rp[0] = 0)
        const int v = kary_last_le(rp, 0, n - 1, e);
        const int u = __ldg(col + e);
        if (u < 0 || u >= n || u == v) { bad = true; continue; }
        if (e > __ldg(rp + v) && __ldg(col + e - 1) >= u) { bad = true; continue; }
        if (u > v) {
            up++;
            if (!kary_find(col + __ldg(rp + u), __ldg(rp + u + 1) - __ldg(rp + u), v)) bad = true;
        }
    }
    if (bad) atomicOr(err, 1);
    up = __reduce_add_sync(kFull, up);
    if ((threadIdx.x & 31) == 0 && up) atomicAdd(err + 1, up);
}

// err[2] = maximum degree (row length)
__global__ void max_degree_kernel(int n, const int *rp, int *err)
{
    int dm = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        dm = max(dm, rp[v + 1] - rp[v]);
    dm = __reduce_max_sync(kFull, dm);
    if ((threadIdx.x & 31) == 0 && dm) atomicMax(err + 2, dm);
}

// ------------------------------------------------------------ root kernel

constexpr int kRootThreads = 1024;
// Rows longer than this are scanned by a whole warp: a thread scanning a row
// alone takes one dependent L2 round trip per 8 entries, and after the first
// rounds a round holds few vertices, so its slowest row sets its length.
constexpr int kHeavyRow = 8;
constexpr int kGiantRow = 512;   // rows longer than this are applied by the whole block

struct RootShared {
    int cnt;        // marks in this round
    int fcnt;       // next-frontier size
    int hcnt;       // heavy-row list size
    int gcnt;       // giant-row list size
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

// two block-wide sums at once (one set of barriers); both results replace
// the inputs in every thread
__device__ __forceinline__ void block_sum2(int &a, int &b, int *red, int *red2)
{
    int x = __reduce_add_sync(kFull, a), y = __reduce_add_sync(kFull, b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) { red[w] = x; red2[w] = y; }
    __syncthreads();
    if (w == 0) {
        x = l < nw ? red[l] : 0;
        y = l < nw ? red2[l] : 0;
        x = __reduce_add_sync(kFull, x);
        y = __reduce_add_sync(kFull, y);
        if (l == 0) { red[32] = x; red2[32] = y; }
    }
    __syncthreads();
    a = red[32];
    b = red2[32];
}

// exclusive running maximum of one value per thread (block-wide, in thread
// order; 0 for thread 0)
__device__ __forceinline__ int block_excl_max(int x, int *red)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    int inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, o);
        if (l >= o) inc = max(inc, y);
    }
    int exc = __shfl_up_sync(kFull, inc, 1);
    if (l == 0) exc = 0;
    __syncthreads();
    if (l == 31) red[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int y = l < nw ? red[l] : 0;
        int sc = y;
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(kFull, sc, o);
            if (l >= o) sc = max(sc, z);
        }
        int ex = __shfl_up_sync(kFull, sc, 1);
        if (l == 0) ex = 0;
        if (l < nw) red[l] = ex;
    }
    __syncthreads();
    const int r = max(red[w], exc);
    __syncthreads();
    return r;
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

// Append val to list (slot from *counter) for every lane with pred set, with
// one atomic per warp instead of one per lane.
__device__ __forceinline__ void agg_append(int *counter, int *list, int val, bool pred)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!pred) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(m, base, leader);
    list[base + __popc(m & ((1u << lane) - 1))] = val;
}

__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Ask the memory system to bring [p, p + bytes) into L2 (bulk prefetch,
// 16-byte granules); the block's threads split the range.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes)
{
    const size_t start = ((size_t)p + 15) & ~(size_t)15;
    const size_t end = ((size_t)p + bytes) & ~(size_t)15;
    constexpr size_t kPiece = 16384;
    for (size_t a = start + (size_t)threadIdx.x * kPiece; a < end; a += (size_t)blockDim.x * kPiece) {
        const size_t len = end - a < kPiece ? end - a : kPiece;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)len) : "memory");
    }
}

// Where the per-vertex root state lives.
// Global: int degrees, byte states, int mark / frontier flags in HBM (any n).
struct GlobalStore {
    int *deg;
    uint8_t *st;
    int *mark;
    int *flag;
    __device__ void bind(QueryDesc &Q, char *) { deg = Q.deg; st = Q.st; mark = Q.aux; flag = Q.flag; }
    static __host__ __device__ size_t smem_bytes(int) { return 0; }
    __device__ __forceinline__ int d(int v) const { return deg[v]; }
    __device__ __forceinline__ void set_d(int v, int x) { deg[v] = x; }
    __device__ __forceinline__ void dec(int v) { atomicSub(&deg[v], 1); }
    __device__ __forceinline__ int s(int v) const { return st[v]; }
    __device__ __forceinline__ void set_s(int v, int x) { st[v] = (uint8_t)x; }
    __device__ __forceinline__ bool try_mark(int v) { return atomicExch(&mark[v], 1) == 0; }
    __device__ __forceinline__ bool marked(int v) const { return ((volatile int *)mark)[v] != 0; }
    __device__ __forceinline__ void reset_mark(int v) { mark[v] = 0; }
    __device__ __forceinline__ bool try_flag(int v) { return atomicExch(&flag[v], 1) == 0; }
    __device__ __forceinline__ void reset_flag(int v) { flag[v] = 0; }
    __device__ void publish(QueryDesc &, int) {}
};

// Shared: 16-bit degrees, byte states and mark / frontier bitmaps in shared
// memory (about 3.3 bytes per vertex); needs max degree <= 65535.
struct SmemStore {
    uint16_t *deg;
    uint8_t *st;
    uint32_t *mark;
    uint32_t *flag;
    static __host__ __device__ size_t smem_bytes(int n)
    {
        const size_t w = (size_t)(n + 31) / 32 * 4;
        return ((size_t)n * 2 + 15) / 16 * 16 + ((size_t)n + 15) / 16 * 16 + 2 * ((w + 15) / 16 * 16);
    }
    __device__ void bind(QueryDesc &Q, char *smem)
    {
        const int n = Q.n;
        const size_t w = (size_t)(n + 31) / 32 * 4;
        char *p = smem;
        deg = (uint16_t *)p;  p += ((size_t)n * 2 + 15) / 16 * 16;
        st = (uint8_t *)p;    p += ((size_t)n + 15) / 16 * 16;
        mark = (uint32_t *)p; p += (w + 15) / 16 * 16;
        flag = (uint32_t *)p;
        for (int i = threadIdx.x; i < (n + 31) / 32; i += blockDim.x) { mark[i] = 0; flag[i] = 0; }
    }
    __device__ __forceinline__ int d(int v) const { return deg[v]; }
    __device__ __forceinline__ void set_d(int v, int x) { deg[v] = (uint16_t)x; }
    __device__ __forceinline__ void dec(int v)
    {
        unsigned *w = (unsigned *)((char *)deg + 2 * (v & ~1));
        atomicSub(w, 1u << (16 * (v & 1)));
    }
    __device__ __forceinline__ int s(int v) const { return st[v]; }
    __device__ __forceinline__ void set_s(int v, int x) { st[v] = (uint8_t)x; }
    __device__ __forceinline__ bool try_mark(int v)
    {
        const unsigned bit = 1u << (v & 31);
        return !(atomicOr(&mark[v >> 5], bit) & bit);
    }
    __device__ __forceinline__ bool marked(int v) const { return ((volatile uint32_t *)mark)[v >> 5] >> (v & 31) & 1u; }
    __device__ __forceinline__ void reset_mark(int v) { atomicAnd(&mark[v >> 5], ~(1u << (v & 31))); }
    __device__ __forceinline__ bool try_flag(int v)
    {
        const unsigned bit = 1u << (v & 31);
        return !(atomicOr(&flag[v >> 5], bit) & bit);
    }
    __device__ __forceinline__ void reset_flag(int v) { atomicAnd(&flag[v >> 5], ~(1u << (v & 31))); }
    // the answer assembly reads the states from global memory
    __device__ void publish(QueryDesc &Q, int n)
    {
        for (int v = threadIdx.x; v < n; v += blockDim.x) Q.st[v] = st[v];
    }
};

template <class Store>
struct Root {
    QueryDesc &Q;
    Store S;
    RootShared &sh;
    int n;
    const int *rp, *col;

    __device__ Root(QueryDesc &q, RootShared &s, char *smem) : Q(q), sh(s)
    {
        n = Q.n;
        rp = Q.rp;
        col = Q.col;
        S.bind(Q, smem);
    }

    __device__ __forceinline__ bool live(int x) const { return S.s(x) == 0 && S.d(x) > 0; }

    __device__ __forceinline__ void mark(int u)
    {
        agg_append(&sh.cnt, Q.forced_list + sh.forced, u, S.try_mark(u));
    }

    __device__ __forceinline__ void push_frontier(int *next, int x)
    {
        agg_append(&sh.fcnt, next, x, S.try_flag(x));
    }

    // Is u-w an edge?  The CSR is symmetric and its rows sorted: search the
    // shorter of the two rows (batched linear scan, else binary search).
    __device__ bool row_has(int u, int w) const
    {
        const int au = __ldg(rp + u), bu = __ldg(rp + u + 1);
        const int aw = __ldg(rp + w), bw = __ldg(rp + w + 1);
        const bool by_u = bu - au <= bw - aw;
        const int a = by_u ? au : aw, b = by_u ? bu : bw, key = by_u ? w : u;
        if (b - a > 16) return bsearch_row(col + a, b - a, key);
        for (int e0 = a; e0 < b; e0 += 8) {
            int xs[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? __ldg(col + e0 + j) : -1;
            bool hit = false;
#pragma unroll
            for (int j = 0; j < 8; j++) hit |= xs[j] == key;
            if (hit) return true;
        }
        return false;
    }

    // The rule decision for v once its live neighbours u (and w) are known.
    __device__ void decide(int *next, int v, int d, int u, int w)
    {
        if (d == 1) {
            if (u < 0) return;
            if (S.d(u) == 1 && u < v) push_frontier(next, u);   // u's rule fires instead
            else mark(u);
        } else if (d == 2) {
            if (w < 0) return;
            if (row_has(u, w)) {
                int p = INT_MAX;
                if (S.d(u) == 2 && u < v) p = u;
                if (S.d(w) == 2 && w < v && w < p) p = w;
                if (p != INT_MAX) push_frontier(next, p);   // the lowest degree-two vertex fires
                else { mark(u); mark(w); }
            }
        }
    }

    // Examine v against the rules; long rows of degree-1/2 vertices go to the
    // heavy list for a warp to scan.
    __device__ void examine(int *next, int *heavy, int v, int bud)
    {
        if (S.s(v) != 0) return;
        const int d = S.d(v);
        if (d == 0) return;
        if (d > bud) mark(v);
        if (d > 2) return;
        const int a = __ldg(rp + v), b = __ldg(rp + v + 1);
        if (b - a > kHeavyRow) {
            agg_append(&sh.hcnt, heavy, v, true);
            return;
        }
        // the first d live neighbours; eight independent loads in flight at a time
        int u = -1, w = -1;
        for (int e0 = a; e0 < b; e0 += 8) {
            int xs[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? __ldg(col + e0 + j) : -1;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int x = xs[j];
                if (x >= 0 && w < 0 && live(x)) {
                    if (u < 0) u = x; else w = x;
                }
            }
            if (d == 1 ? u >= 0 : w >= 0) break;
        }
        decide(next, v, d, u, w);
    }

    // Warp-cooperative: the first `need` live neighbours of v.
    __device__ void warp_live_nbrs(int v, int need, int &u, int &w) const
    {
        const int lane = threadIdx.x & 31;
        const int a = __ldg(rp + v), b = __ldg(rp + v + 1);
        u = -1;
        w = -1;
        int found = 0;
        for (int base = a; base < b && found < need; base += 32) {
            const int e = base + lane;
            const int x = e < b ? __ldg(col + e) : -1;
            unsigned m = __ballot_sync(kFull, x >= 0 && live(x));
            while (m && found < need) {
                const int pos = __ffs(m) - 1;
                const int val = __shfl_sync(kFull, x, pos);
                if (found == 0) u = val; else w = val;
                found++;
                m &= m - 1;
            }
        }
    }

    // Put u in the cover: lower the degrees of its live, unmarked neighbours.
    __device__ __forceinline__ void apply_one(int *next, int x)
    {
        if (S.s(x) == 0 && S.d(x) > 0 && !S.marked(x)) {
            S.dec(x);
            push_frontier(next, x);
        }
    }

    __device__ void apply_row(int *next, int u, int lane, int stride)
    {
        const int a = __ldg(rp + u), b = __ldg(rp + u + 1);
        if (stride == 1) {
            // one thread: eight independent loads in flight at a time
            for (int e0 = a; e0 < b; e0 += 8) {
                int xs[8];
#pragma unroll
                for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? __ldg(col + e0 + j) : -1;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (xs[j] >= 0) apply_one(next, xs[j]);
            }
            return;
        }
        for (int e = a + lane; e < b; e += stride) apply_one(next, __ldg(col + e));
    }

    // Synchronous rounds of the rules until nothing is marked.  hd: use the
    // high-degree rule with budget bound - forced - 1.  Returns false when the
    // budget went negative (no cover smaller than `bound` can exist).
    __device__ bool reduce_rounds(bool hd, int bound)
    {
        int *cur = Q.fr0, *next = Q.fr1, *heavy = Q.heavy;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
        int fsize = -1;   // -1: full scan
        for (;;) {
            const int bud = hd ? bound - sh.forced - 1 : INT_MAX;
            if (hd && bud < 0) return false;
            const bool full = fsize < 0 || (hd && sh.delta > bud);
            __syncthreads();
            if (threadIdx.x == 0) { sh.cnt = 0; sh.fcnt = 0; sh.hcnt = 0; }
            __syncthreads();
            int dmax = 0;
            if (full) {
                for (int v = threadIdx.x; v < n; v += blockDim.x) {
                    S.reset_flag(v);
                    if (S.s(v) == 0) dmax = max(dmax, S.d(v));
                }
                __syncthreads();
                for (int v = threadIdx.x; v < n; v += blockDim.x) examine(next, heavy, v, bud);
            } else {
                for (int i = threadIdx.x; i < fsize; i += blockDim.x) S.reset_flag(cur[i]);
                __syncthreads();
                for (int i = threadIdx.x; i < fsize; i += blockDim.x) examine(next, heavy, cur[i], bud);
            }
            __syncthreads();
            // heavy rows: one warp per vertex
            const int hcnt = sh.hcnt;
            for (int i = warp; i < hcnt; i += nwarps) {
                const int v = heavy[i];
                const int d = S.d(v);
                int u, w;
                warp_live_nbrs(v, d, u, w);
                if (lane == 0) decide(next, v, d, u, w);
            }
            if (full) {
                const int dm = block_max(dmax, sh.red);
                if (threadIdx.x == 0) sh.delta = dm;
            }
            __syncthreads();
            const int cnt = sh.cnt;
            const int base = sh.forced;
            if (threadIdx.x == 0) Q.rounds++;
            if (cnt == 0 && sh.fcnt == 0) return true;
            __syncthreads();
            if (threadIdx.x == 0) sh.hcnt = 0;
            __syncthreads();
            // apply: lower the degrees of the marked vertices' live neighbours;
            // short rows by one thread, long rows by a warp, giant rows (from
            // the end of the same list) by the whole block
            if (threadIdx.x == 0) sh.gcnt = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int u = Q.forced_list[base + i];
                const int len = __ldg(rp + u + 1) - __ldg(rp + u);
                agg_append(&sh.hcnt, heavy, u, len > kHeavyRow && len <= kGiantRow);
                if (len > kGiantRow) heavy[n - 1 - atomicAdd(&sh.gcnt, 1)] = u;   // rare
                if (len <= kHeavyRow) apply_row(next, u, 0, 1);
            }
            __syncthreads();
            const int hc2 = sh.hcnt, gc = sh.gcnt;
            for (int i = warp; i < hc2; i += nwarps) apply_row(next, heavy[i], lane, 32);
            for (int i = 0; i < gc; i++) apply_row(next, heavy[n - 1 - i], threadIdx.x, blockDim.x);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const int u = Q.forced_list[base + i];
                S.set_s(u, 1);
                S.set_d(u, 0);
            }
            __syncthreads();
            if (threadIdx.x == 0) sh.forced = base + cnt;
            fsize = sh.fcnt;
            int *t = cur; cur = next; next = t;
            __syncthreads();
            if (fsize == 0 && !(hd && sh.delta > bound - sh.forced - 1)) return true;
        }
    }

    __device__ int live_edges2()
    {
        int e2 = 0;
        for (int v = threadIdx.x; v < n; v += blockDim.x)
            if (S.s(v) == 0) e2 += S.d(v);
        return block_sum(e2, sh.red);
    }

    // Greedy cover of the live graph: the complement of a maximal independent
    // set chosen by static priority (degree, hash(id)), lowest first.  aux[v]:
    // 0 undecided, 1 in the set, 2 in the cover, 3 not live, 4 joining.
    // Flags the whole cover (forced + greedy) in cover_flags; returns the
    // number of live vertices it puts in the cover.
    __device__ int greedy()
    {
        int *aux = Q.aux, *join = Q.fr0;
        for (int v = threadIdx.x; v < n; v += blockDim.x) aux[v] = live(v) ? 0 : 3;
        __syncthreads();
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) sh.flag = 0;
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                if (aux[v] != 0) continue;
                const unsigned long long pv = ((unsigned long long)S.d(v) << 32) | mix32((unsigned)v);
                bool j = true;
                for (int e = __ldg(rp + v); e < __ldg(rp + v + 1) && j; e++) {
                    const int x = __ldg(col + e);
                    const int ax = aux[x];
                    if (ax == 1) j = false;
                    else if (ax == 0) {
                        const unsigned long long px = ((unsigned long long)S.d(x) << 32) | mix32((unsigned)x);
                        if (px < pv || (px == pv && x < v)) j = false;
                    }
                }
                join[v] = j;
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x)
                if (aux[v] == 0 && join[v]) { aux[v] = 4; sh.flag = 1; }
            __syncthreads();
            if (!sh.flag) break;
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                if (aux[v] != 4) continue;
                for (int e = __ldg(rp + v); e < __ldg(rp + v + 1); e++) {
                    const int x = __ldg(col + e);
                    if (aux[x] == 0) aux[x] = 2;
                }
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x)
                if (aux[v] == 4) aux[v] = 1;
        }
        __syncthreads();
        int c = 0;
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const bool g = aux[v] == 2 || aux[v] == 0;
            Q.cover_flags[v] = (S.s(v) == 1 || g) ? 1 : 0;
            c += g;
        }
        const int tot = block_sum(c, sh.red);
        for (int v = threadIdx.x; v < n; v += blockDim.x) aux[v] = 0;
        __syncthreads();
        return tot;
    }

    // Induce the subgraph on the live vertices with non-zero degree,
    // relabelled in increasing original id (rows stay sorted).
    __device__ void induce()
    {
        const int T = blockDim.x;
        const int chunk = (n + T - 1) / T;
        const int beg = min(n, (int)threadIdx.x * chunk), end = min(n, beg + chunk);
        int cnt = 0, dsum = 0, dmax = 0;
        for (int v = beg; v < end; v++)
            if (live(v)) { cnt++; dsum += S.d(v); dmax = max(dmax, S.d(v)); }
        int np, m2p;
        const int off = block_excl_scan(cnt, sh.red, &np);
        const int eoff = block_excl_scan(dsum, sh.red, &m2p);
        const int dm = block_max(dmax, sh.red);
        int *nid = Q.aux;
        int id = off, eo = eoff;
        for (int v = beg; v < end; v++) {
            if (live(v)) {
                nid[v] = id;
                Q.orig[id] = v;
                Q.rp2[id] = eo;
                id++;
                eo += S.d(v);
            } else {
                nid[v] = -1;
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
            const int v = Q.orig[i];
            int o = Q.rp2[i];
            for (int e = __ldg(rp + v); e < __ldg(rp + v + 1); e++) {
                const int nx = nid[__ldg(col + e)];
                if (nx >= 0) Q.col2[o++] = nx;
            }
        }
        __syncthreads();
        for (int v = threadIdx.x; v < n; v += T) nid[v] = 0;
        __syncthreads();
    }

    __device__ void run()
    {
        prefetch_l2(rp, (size_t)(n + 1) * 4);
        prefetch_l2(col, (size_t)Q.m2 * 4);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            S.set_d(v, __ldg(rp + v + 1) - __ldg(rp + v));
            S.set_s(v, 0);
            Q.aux[v] = 0;
            Q.flag[v] = 0;
            Q.cover_flags[v] = 0;
        }
        if (threadIdx.x == 0) {
            sh.forced = 0;
            sh.delta = INT_MAX;
            Q.np = 0; Q.m2p = 0; Q.maxdeg = 0; Q.answered = 0; Q.greedy = -1;
            Q.improved = 0; Q.result = -1; Q.yes = 0; Q.cover_len = 0;
            Q.rounds = 0;
            Q.listed = 0;
            for (int i = 0; i < 4; i++) Q.root_cycles[i] = 0;
        }
        __syncthreads();

        // phase 1: degree-one and degree-two-triangle rules (need no bound)
        long long t0 = clock64();
        if (!Q.skip_root_rules) reduce_rounds(false, INT_MAX);
        long long t1 = clock64();
        if (threadIdx.x == 0) Q.root_cycles[0] = t1 - t0;
        if (live_edges2() == 0) {
            // the rules alone produced a cover; they are exact, so it is minimum
            S.publish(Q, n);
            for (int v = threadIdx.x; v < n; v += blockDim.x) Q.cover_flags[v] = S.s(v) == 1;
            if (threadIdx.x == 0) {
                Q.forced = sh.forced;
                Q.answered = 1;
                Q.bound = sh.forced;
                if (Q.k < 0) { Q.result = sh.forced; Q.yes = 1; }
                else { Q.yes = sh.forced <= Q.k; Q.result = Q.yes ? sh.forced : -1; }
            }
            return;
        }

        // initial upper bound (Algorithm 1, Section 2.2): the size of a cover
        // found fast with no optimality claim
        const int greedy_size = sh.forced + greedy();
        t0 = clock64();
        if (threadIdx.x == 0) { Q.greedy = greedy_size; Q.root_cycles[1] = t0 - t1; }
        if (Q.k >= 0 && greedy_size <= Q.k) {
            S.publish(Q, n);
            if (threadIdx.x == 0) {
                Q.forced = sh.forced; Q.answered = 1; Q.bound = greedy_size; Q.yes = 1; Q.result = greedy_size;
            }
            return;
        }
        // look only for covers smaller than `bound`
        const int bound = Q.k >= 0 ? Q.k + 1 : greedy_size;

        // phase 2: all three rules; high-degree budget b = bound - |F| - 1
        const bool feasible = Q.skip_root_rules ? true : reduce_rounds(true, bound);
        t1 = clock64();
        if (threadIdx.x == 0) Q.root_cycles[2] = t1 - t0;
        const int e2 = live_edges2();
        S.publish(Q, n);
        if (!feasible || sh.forced >= bound) {
            // no cover smaller than the bound exists
            if (threadIdx.x == 0) {
                Q.forced = sh.forced; Q.answered = 1; Q.bound = bound;
                if (Q.k < 0) { Q.result = greedy_size; Q.yes = 1; }   // the greedy flags hold it
                else { Q.yes = 0; Q.result = -1; }
            }
            return;
        }
        if (e2 == 0) {
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) Q.cover_flags[v] = S.s(v) == 1;
            if (threadIdx.x == 0) {
                Q.forced = sh.forced; Q.answered = 1; Q.bound = bound;
                Q.result = sh.forced; Q.yes = 1;
            }
            return;
        }
        induce();
        if (threadIdx.x == 0) { Q.forced = sh.forced; Q.bound = bound; Q.root_cycles[3] = clock64() - t1; }
    }
};

template <class Store>
__global__ void __launch_bounds__(kRootThreads, 1) root_kernel(QueryDesc *qs)
{
    extern __shared__ __align__(16) char root_smem[];
    __shared__ RootShared sh;
    QueryDesc &Q = qs[blockIdx.x];
    if (Q.status != VC_OK) return;
    Root<Store> r(Q, sh, root_smem);
    __syncthreads();
    r.run();
}

// ------------------------------------------------------------ cluster root kernel
//
// The same root phase for ONE large graph on a thread-block cluster of up to
// 16 CTAs (one per SM).  Vertex v is owned by CTA v >> cs; its 16-bit degree,
// state byte, mark bit and frontier bit live in that CTA's shared memory and
// every CTA reaches them through distributed shared memory.  Each CTA examines
// the vertices it owns; marks and frontier pushes go to the owner's lists.
// Rounds are separated by cluster barriers; per-round totals are exchanged
// through rank 0's shared memory.  Decisions taken from exchanged totals are
// identical in every CTA, so all CTAs pass the same barriers.

}  // namespace vcg
#include <cooperative_groups.h>
namespace vcg {
namespace cgx = cooperative_groups;

constexpr int kClusterMax = 16;
constexpr int kClusterMinN = 8192;    // smaller graphs use one block

struct ClusterShared {
    int cnt;          // solo rounds: frontier entries listed
    int fcnt;         // solo rounds: marks listed
    int hcnt;         // heavy rows of this CTA's examination
    int tcnt;         // triangle checks of this CTA's examination
    int red[33];
    int red2[33];
    long long tot[4]; // exchanged totals (local copy)
    int slot[2][kClusterMax][4];   // rank 0's copy is the exchange area (double-buffered)
    unsigned long long rbase[kClusterMax];   // dynamic smem base of each rank
    unsigned long long rsh[kClusterMax];     // ClusterShared of each rank
    int solo_forced;  // rank 0: vertices it forced in the rounds it ran alone
};

// Per CTA of a C-CTA cluster, for chunk owned vertices: 16-bit degrees; a
// copy of the forced bitmap of the whole graph (C chunks); the vertices
// forced in the current round (whole graph); two mark bitmaps (alternate
// rounds) and the frontier bitmap of the owned vertices; the degrees at the
// end of the previous round.  Every part is a multiple of 16 bytes (chunk
// >= 1024).
__host__ __device__ inline size_t cluster_smem_bytes(int chunk, int C)
{
    return (size_t)chunk * 2 + 2 * ((size_t)C * chunk / 8) + 3 * ((size_t)chunk / 8) + (size_t)chunk * 2;
}

// The degree update of one CTA of the cluster root kernel after a round's
// marks, over its staged rows: lcol[0, E) are the row entries of its owned
// vertices, lsrc[e] the owned vertex whose row holds entry e, nw the
// vertices forced in the round (whole graph), fw the forced bits of the
// owned vertices (this round's included), dw the owned 16-bit degrees (two
// to a word).  Every owned vertex that is not forced loses one degree per
// newly forced neighbour (a fire-and-forget reduction; the next frontier is
// found afterwards by comparing degrees).  The entries are scanned flat,
// four per thread in flight.  Only local shared memory is touched.  Not
// inlined: the round loop around it keeps many values live, and this loop
// runs without spills on a register allocation of its own.
__device__ __noinline__ void cluster_pull_flat(const int *lcol, const uint16_t *lsrc, const uint32_t *nw,
                                               const uint32_t *fw, unsigned *dw, int E)
{
    const int T = blockDim.x;
    for (int e0 = threadIdx.x; e0 < E; e0 += 4 * T) {
        int xs[4];
#pragma unroll
        for (int j = 0; j < 4; j++) xs[j] = e0 + j * T < E ? lcol[e0 + j * T] : -1;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int x = xs[j];
            if (x < 0 || !((nw[x >> 5] >> (x & 31)) & 1u)) continue;
            const int v = lsrc[e0 + j * T];
            if (!((fw[v >> 5] >> (v & 31)) & 1u))        // (a forced vertex's degree is not used again)
                atomicSub(dw + (v >> 1), 1u << (16 * (v & 1)));
        }
    }
}

struct ClusterRoot {
    QueryDesc &Q;
    ClusterShared &sh;
    cgx::cluster_group cl;
    int n, C, rank, cs, chunk;
    int vbeg, vcnt;          // vertices owned here: [vbeg, vbeg + vcnt)
    const int *rp, *col;
    int ftot;                // cluster-wide forced count (same in every CTA)
    int xround;              // exchange buffer selector
    int mbuf;                // mark bitmap of the current round (0 / 1)
    int repb;                // bytes of a whole-graph bitmap (C chunks)
    // rows of the vertices owned here, staged in shared memory when they fit
    // (lrp: offsets into lcol, relative to this CTA's first entry); null:
    // the rows are read from the global CSR
    const int *lrp, *lcol;
    const uint16_t *lsrc;    // with staged rows, when it fits: the owned vertex of each row entry
    char *lsm;               // this CTA's dynamic shared memory
    int res_off, smem_cap;   // where the staged rows (or rank 0's residual graph) start; its size
    int e_first;             // global index of this CTA's first row entry

    __device__ ClusterRoot(QueryDesc &q, ClusterShared &s, char *smem, int cs_, int smem_bytes)
        : Q(q), sh(s), cl(cgx::this_cluster())
    {
        n = Q.n;
        C = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
        cs = cs_;
        chunk = 1 << cs;
        vbeg = rank << cs;
        vcnt = max(0, min(chunk, n - vbeg));
        rp = Q.rp;
        col = Q.col;
        ftot = 0;
        xround = 0;
        mbuf = 0;
        repb = C * (chunk / 8);
        if (threadIdx.x < C) {
            sh.rbase[threadIdx.x] = (unsigned long long)cl.map_shared_rank(smem, threadIdx.x);
            sh.rsh[threadIdx.x] = (unsigned long long)cl.map_shared_rank(&sh, threadIdx.x);
        }
        uint32_t *bits = (uint32_t *)(smem + 2 * (size_t)chunk);
        const int nbits = (int)((cluster_smem_bytes(chunk, C) - 2 * (size_t)chunk) / 4);
        for (int i = threadIdx.x; i < nbits; i += blockDim.x) bits[i] = 0;
        // Stage this CTA's rows: every examination and application of the
        // rules, the greedy bound and the induced graph read only rows of
        // vertices owned here (a shared-memory load instead of an L2 round
        // trip); the triangle test's rows of other vertices stay global.
        lrp = nullptr;
        lcol = nullptr;
        lsrc = nullptr;
        const size_t off = (cluster_smem_bytes(chunk, C) + 15) & ~(size_t)15;
        lsm = smem;
        res_off = (int)off;
        smem_cap = smem_bytes;
        const int e0 = vcnt > 0 ? __ldg(rp + vbeg) : 0, e1 = vcnt > 0 ? __ldg(rp + vbeg + vcnt) : 0;
        e_first = e0;
        const int E = e1 - e0;
        const long long need = 4ll * (chunk + 1) + 4ll * E;
        if (vcnt > 0 && (long long)off + need <= (long long)smem_bytes) {
            int *r = (int *)(smem + off), *c = r + chunk + 1;
            // eight independent loads in flight per thread (the CSR comes
            // from DRAM on a cold L2)
            const int T = blockDim.x;
            for (int i0 = threadIdx.x; i0 <= vcnt; i0 += 8 * T) {
                int xs[8];
#pragma unroll
                for (int j = 0; j < 8; j++) xs[j] = i0 + j * T <= vcnt ? __ldg(rp + vbeg + i0 + j * T) : 0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (i0 + j * T <= vcnt) r[i0 + j * T] = xs[j] - e0;
            }
            for (int f0 = threadIdx.x; f0 < E; f0 += 8 * T) {
                int xs[8];
#pragma unroll
                for (int j = 0; j < 8; j++) xs[j] = f0 + j * T < E ? __ldg(col + e0 + f0 + j * T) : 0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (f0 + j * T < E) c[f0 + j * T] = xs[j];
            }
            lrp = r;
            lcol = c;
            const size_t soff = (off + (size_t)need + 15) & ~(size_t)15;
            if (soff + 2 * (size_t)E <= (size_t)smem_bytes) {
                // lsrc[e]: 0 everywhere, each non-empty row's vertex at its
                // first entry, then a running maximum (rows are in vertex order)
                uint16_t *src = (uint16_t *)(smem + soff);
                for (int e = threadIdx.x; e < E; e += blockDim.x) src[e] = 0;
                __syncthreads();
                for (int i = threadIdx.x; i < vcnt; i += blockDim.x)
                    if (r[i] < r[i + 1]) src[r[i]] = (uint16_t)i;
                __syncthreads();
                const int s0 = (int)((long long)E * threadIdx.x / blockDim.x);
                const int s1 = (int)((long long)E * (threadIdx.x + 1) / blockDim.x);
                int m = 0;
                for (int e = s0; e < s1; e++) m = max(m, (int)src[e]);
                int carry = block_excl_max(m, sh.red);
                for (int e = s0; e < s1; e++) {
                    carry = max(carry, (int)src[e]);
                    src[e] = (uint16_t)carry;
                }
                lsrc = src;
            }
        }
        __syncthreads();
    }

    // Row of a vertex owned here: entries [a, b) of *cp.
    __device__ __forceinline__ void own_row(int v, int &a, int &b, const int *&cp) const
    {
        if (lcol) {
            const int i = v - vbeg;
            a = lrp[i];
            b = lrp[i + 1];
            cp = lcol;
        } else {
            a = __ldg(rp + v);
            b = __ldg(rp + v + 1);
            cp = col;
        }
    }

    // ---- distributed state
    __device__ __forceinline__ char *base(int r) const { return (char *)sh.rbase[r]; }
    __device__ __forceinline__ uint16_t *degp(int r) const { return (uint16_t *)base(r); }
    // rank r's copy of the forced bitmap (whole graph)
    __device__ __forceinline__ uint32_t *repp(int r) const { return (uint32_t *)(base(r) + 2 * (size_t)chunk); }
    // the forced bits of rank r's own vertices in rank r's copy: always current
    __device__ __forceinline__ uint32_t *forcedp(int r) const { return repp(r) + ((size_t)r << (cs - 5)); }
    __device__ __forceinline__ uint32_t *markp(int r, int b) const
    {
        return (uint32_t *)(base(r) + 2 * (size_t)chunk + 2 * (size_t)repb + (size_t)b * (chunk / 8));
    }
    __device__ __forceinline__ uint32_t *flagp(int r) const
    {
        return (uint32_t *)(base(r) + 2 * (size_t)chunk + 2 * (size_t)repb + 2 * (chunk / 8));
    }
    // this CTA's own arrays through its local shared-memory window
    __device__ __forceinline__ uint16_t *ldeg() const { return (uint16_t *)lsm; }
    __device__ __forceinline__ uint32_t *lrep() const { return (uint32_t *)(lsm + 2 * (size_t)chunk); }
    __device__ __forceinline__ uint32_t *lnew() const { return (uint32_t *)(lsm + 2 * (size_t)chunk + repb); }
    __device__ __forceinline__ uint32_t *lmark() const { return (uint32_t *)(lsm + 2 * (size_t)chunk + 2 * (size_t)repb); }
    __device__ __forceinline__ uint32_t *lflag() const { return lmark() + 2 * (chunk >> 5); }
    __device__ __forceinline__ uint16_t *lprev() const { return (uint16_t *)(lflag() + (chunk >> 5)); }
    __device__ __forceinline__ ClusterShared *shp(int r) const { return (ClusterShared *)sh.rsh[r]; }

    __device__ __forceinline__ int d(int v) const
    {
        if ((v >> cs) == rank) return ((volatile uint16_t *)ldeg())[v - vbeg];
        return ((volatile uint16_t *)degp(v >> cs))[v & (chunk - 1)];
    }
    __device__ __forceinline__ bool forced(int v) const
    {
        const int l = v & (chunk - 1);
        return ((volatile uint32_t *)forcedp(v >> cs))[l >> 5] >> (l & 31) & 1u;
    }
    // In the rule rounds every CTA's copy of the forced bitmap is complete
    // (it is refreshed when the rounds start and every round's marks are
    // added to every copy): a local load.
    __device__ __forceinline__ bool rforced(int v) const { return lrep()[v >> 5] >> (v & 31) & 1u; }
    // a vertex is in the graph when it was not forced in an earlier round
    // and has a neighbour left
    __device__ __forceinline__ bool live(int x) const { return !forced(x) && d(x) > 0; }
    __device__ __forceinline__ void set_bit(uint32_t *words, int v)
    {
        const int l = v & (chunk - 1);
        atomicOr(&words[l >> 5], 1u << (l & 31));    // result unused: a fire-and-forget reduction
    }
    __device__ __forceinline__ void mark(int u) { set_bit(markp(u >> cs, mbuf), u); }
    __device__ __forceinline__ void push_frontier(int x) { set_bit(flagp(x >> cs), x); }

    // Is u-w an edge?  The CSR is symmetric, so the shorter of the two rows
    // is searched.
    __device__ bool row_has(int u, int w) const
    {
        const int au = __ldg(rp + u), bu = __ldg(rp + u + 1);
        const int aw = __ldg(rp + w), bw = __ldg(rp + w + 1);
        const bool by_u = bu - au <= bw - aw;
        return by_u ? kary_find(col + au, bu - au, w) : kary_find(col + aw, bw - aw, u);
    }

    // The degree-one rule at v (its only live neighbour u); the lower end of
    // an edge whose ends both have degree one decides, so the other end
    // hands its turn to it.
    __device__ __forceinline__ void decide_one(int v, int u)
    {
        if (u < v && d(u) == 1) push_frontier(u);   // u's rule fires instead
        else mark(u);
    }

    // The degree-two-triangle rule at v with live neighbours u, w: lists the
    // check for the triangle pass of the round (Q.deg / Q.heavy / Q.flag
    // hold this CTA's list in its own range; at most one entry per owned
    // vertex).
    __device__ __forceinline__ void list_triangle(int v, int u, int w)
    {
        const int i = vbeg + atomicAdd(&sh.tcnt, 1);
        Q.deg[i] = v;
        Q.heavy[i] = u;
        Q.flag[i] = w;
    }

    // A listed triangle check: when u-w is an edge the lowest degree-two
    // vertex of the triangle fires (the others hand it their turn).
    __device__ __forceinline__ void decide_triangle(int v, int u, int w)
    {
        if (!row_has(u, w)) return;
        int p = INT_MAX;
        if (u < v && d(u) == 2) p = u;
        if (w < v && w < p && d(w) == 2) p = w;
        if (p != INT_MAX) push_frontier(p);
        else { mark(u); mark(w); }
    }

    // The rules at the owned vertex v.  Its live neighbours are exactly its
    // neighbours that are not forced: a live vertex's degree counts them, so
    // each of them keeps an edge (to v) and a degree of at least one.
    __device__ void examine(int *hv, int v, int bud)
    {
        const int i = v - vbeg;
        if (rforced(v)) return;
        const int dv = ldeg()[i];
        if (dv == 0) return;
        if (dv > bud) mark(v);
        if (dv > 2) return;
        int a, b;
        const int *cp;
        own_row(v, a, b, cp);
        if (b - a > kHeavyRow) {
            hv[atomicAdd(&sh.hcnt, 1)] = v;
            return;
        }
        int u = -1, w = -1;
        for (int e0 = a; e0 < b; e0 += 8) {
            int xs[8];
            bool lv[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? cp[e0 + j] : -1;
#pragma unroll
            for (int j = 0; j < 8; j++) lv[j] = xs[j] >= 0 && !rforced(xs[j]);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (lv[j] && w < 0) {
                    if (u < 0) u = xs[j]; else w = xs[j];
                }
            }
            if (dv == 1 ? u >= 0 : w >= 0) break;
        }
        if (dv == 1) {
            if (u >= 0) decide_one(v, u);
        } else if (w >= 0) {
            list_triangle(v, u, w);
        }
    }

    __device__ void warp_live_nbrs(int v, int need, int &u, int &w) const
    {
        const int lane = threadIdx.x & 31;
        int a, b;
        const int *cp;
        own_row(v, a, b, cp);
        u = -1;
        w = -1;
        int found = 0;
        for (int base0 = a; base0 < b && found < need; base0 += 32) {
            const int e = base0 + lane;
            const int x = e < b ? cp[e] : -1;
            unsigned m = __ballot_sync(kFull, x >= 0 && !rforced(x));
            while (m && found < need) {
                const int pos = __ffs(m) - 1;
                const int val = __shfl_sync(kFull, x, pos);
                if (found == 0) u = val; else w = val;
                found++;
                m &= m - 1;
            }
        }
    }

    // Row offsets and entries of the owned vertices, relative to this CTA's
    // first entry: staged in shared memory, or the global CSR.
    __device__ __forceinline__ int row_off(int i) const { return lcol ? lrp[i] : __ldg(rp + vbeg + i) - e_first; }
    __device__ __forceinline__ int row_entry(int e) const { return lcol ? lcol[e] : __ldg(col + e_first + e); }

    // This thread's share of the owned row entries for pull_walk: a
    // contiguous range [pe0, pe1) of about equal size, starting in the row of
    // owned vertex pi0 (the rows do not change, so it is found once).
    __device__ void pull_range(int &pi0, int &pe0, int &pe1) const
    {
        const int E = vcnt > 0 ? row_off(vcnt) : 0;
        pe0 = (int)((long long)E * threadIdx.x / blockDim.x);
        pe1 = (int)((long long)E * (threadIdx.x + 1) / blockDim.x);
        int lo = 0, hi = vcnt - 1;                   // the last row starting at or before pe0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_off(mid) <= pe0) lo = mid; else hi = mid - 1;
        }
        pi0 = lo;
    }

    // The degrees of the owned vertices after this round's marks (lnew()):
    // every vertex that is still live loses one per newly forced neighbour
    // (cluster_pull_flat, given lsrc).
    __device__ __forceinline__ void pull_flat()
    {
        cluster_pull_flat(lcol, lsrc, lnew(), lrep() + (rank << (cs - 5)), (unsigned *)ldeg(), row_off(vcnt));
    }

    // The same without lsrc: each thread walks its range of entries row by
    // row, skipping the rows of vertices that are forced or isolated, and
    // subtracts each row's count at once.
    __device__ void pull_walk(int pi0, int pe0, int pe1)
    {
        const uint32_t *nw = lnew(), *fw = lrep() + (rank << (cs - 5));
        int i = pi0, e = pe0;
        while (e < pe1) {
            const int re = min(row_off(i + 1), pe1);
            if (re > e) {
                if (!((fw[i >> 5] >> (i & 31)) & 1u) && ldeg()[i] > 0) {
                    int c = 0;
                    for (; e < re; e++) {
                        const int x = row_entry(e);
                        c += (nw[x >> 5] >> (x & 31)) & 1u;
                    }
                    if (c) atomicSub((unsigned *)ldeg() + (i >> 1), (unsigned)c << (16 * (i & 1)));
                }
                e = re;
            }
            i++;
        }
    }

    // Every CTA's copy of the forced bitmap from the owners' parts (the
    // owners' parts are final: called after a cluster barrier).
    __device__ void refresh_forced_copy()
    {
        const int wpr = chunk >> 5;
        uint32_t *rep = lrep();
        for (int w = threadIdx.x; w < C * wpr; w += blockDim.x) {
            const int r = w / wpr;
            if (r != rank) rep[w] = ((volatile uint32_t *)forcedp(r))[w - r * wpr];
        }
    }

    // After the marks of a round have landed: every CTA reads every CTA's
    // mark bitmap of the round, keeps the vertices not forced before in
    // lnew() and adds them to its copy of the forced bitmap; returns their
    // number (the same in every CTA).  16-byte loads.
    __device__ int gather_marks()
    {
        const int wpr = chunk >> 5;                  // a multiple of 4
        const int q4 = (C * wpr) >> 2;
        uint4 *rep = (uint4 *)lrep(), *nw = (uint4 *)lnew();
        int c = 0;
        for (int q = threadIdx.x; q < q4; q += blockDim.x) {
            const int w = q << 2, r = w / wpr;
            const uint4 m = *(const uint4 *)(markp(r, mbuf) + (w - r * wpr));
            const uint4 o = rep[q];
            uint4 x;
            x.x = m.x & ~o.x; x.y = m.y & ~o.y; x.z = m.z & ~o.z; x.w = m.w & ~o.w;
            nw[q] = x;
            rep[q] = make_uint4(o.x | x.x, o.y | x.y, o.z | x.z, o.w | x.w);
            c += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w);
        }
        return block_sum(c, sh.red);
    }

    // The bits of x (vertices base[0..31]) whose degree is 1 or 2: the only
    // frontier vertices a rule can fire at (the high-degree rule looks at
    // every vertex, in full rounds).
    __device__ __forceinline__ static uint32_t low_degree_bits(uint32_t x, const uint16_t *base)
    {
        uint32_t y = x;
        while (y) {
            const int b = __ffs(y) - 1;
            y &= y - 1;
            if ((unsigned)((const volatile uint16_t *)base)[b] - 1u > 1u) x &= ~(1u << b);
        }
        return x;
    }

    // Take the set bits of my frontier bitmap (fetched and cleared
    // atomically: other CTAs may be setting bits meanwhile) into list[] as
    // vertex ids, leaving out forced vertices; returns the count.  Each
    // thread owns words tid + j*T, j < 4 (chunk <= 4 * 32 * blockDim).
    __device__ int frontier_to_list(int *list)
    {
        uint32_t *words = lflag();
        const uint32_t *fw = lrep() + (rank << (cs - 5));
        const int nw = chunk >> 5;
        uint32_t m[4];
        int c = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int i = threadIdx.x + j * blockDim.x;
            uint32_t x = 0;
            if (i < nw) x = atomicExch(&words[i], 0u) & ~fw[i];
            m[j] = x;
            c += __popc(x);
        }
        int tot;
        int off = block_excl_scan(c, sh.red, &tot);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int i = threadIdx.x + j * blockDim.x;
            uint32_t x = m[j];
            while (x) {
                const int b = __ffs(x) - 1;
                list[off++] = vbeg + i * 32 + b;
                x &= x - 1;
            }
        }
        __syncthreads();
        return tot;
    }

    // Every CTA contributes four numbers; every CTA gets the cluster totals
    // (sum for 0..2, max for 3) in sh.tot.  One cluster barrier (the slots
    // are double-buffered).
    __device__ void exchange(long long a0, long long a1, long long a2, long long a3)
    {
        const int buf = xround & 1;
        xround++;
        if (threadIdx.x == 0) {
            int *sl = shp(0)->slot[buf][rank];
            sl[0] = (int)a0; sl[1] = (int)a1; sl[2] = (int)a2; sl[3] = (int)a3;
        }
        cl.sync();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            long long v0 = 0, v1 = 0, v2 = 0, v3 = INT_MIN;
            if (l < C) {
                const volatile int *sl = shp(0)->slot[buf][l];
                v0 = sl[0]; v1 = sl[1]; v2 = sl[2]; v3 = sl[3];
            }
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(kFull, v0, o);
                v1 += __shfl_xor_sync(kFull, v1, o);
                v2 += __shfl_xor_sync(kFull, v2, o);
                v3 = max(v3, (long long)__shfl_xor_sync(kFull, v3, o));
            }
            if (l == 0) { sh.tot[0] = v0; sh.tot[1] = v1; sh.tot[2] = v2; sh.tot[3] = v3; }
        }
        __syncthreads();
    }

    // The same exchange in two halves around a barrier the caller passes
    // anyway: publish() writes this CTA's four numbers, collect() (after the
    // next cluster barrier) reduces every CTA's into sh.tot.
    __device__ void publish(long long a0, long long a1, long long a2, long long a3)
    {
        const int buf = xround & 1;
        xround++;
        if (threadIdx.x == 0) {
            int *sl = shp(0)->slot[buf][rank];
            sl[0] = (int)a0; sl[1] = (int)a1; sl[2] = (int)a2; sl[3] = (int)a3;
        }
    }
    __device__ void collect()
    {
        const int buf = (xround - 1) & 1;
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            long long v0 = 0, v1 = 0, v2 = 0, v3 = INT_MIN;
            if (l < C) {
                const volatile int *sl = shp(0)->slot[buf][l];
                v0 = sl[0]; v1 = sl[1]; v2 = sl[2]; v3 = sl[3];
            }
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(kFull, v0, o);
                v1 += __shfl_xor_sync(kFull, v1, o);
                v2 += __shfl_xor_sync(kFull, v2, o);
                v3 = max(v3, (long long)__shfl_xor_sync(kFull, v3, o));
            }
            if (l == 0) { sh.tot[0] = v0; sh.tot[1] = v1; sh.tot[2] = v2; sh.tot[3] = v3; }
        }
        __syncthreads();
    }

    // Prefix over ranks of two per-CTA values (exclusive) and their totals.
    __device__ void exchange_prefix(int mine, int mine2, int &off, int &tot, int &off2, int &tot2)
    {
        const int buf = xround & 1;
        xround++;
        if (threadIdx.x == 0) {
            int *sl = shp(0)->slot[buf][rank];
            sl[0] = mine; sl[1] = mine2;
        }
        cl.sync();
        if (threadIdx.x == 0) {
            int o = 0, t = 0, o2 = 0, t2 = 0;
            for (int r = 0; r < C; r++) {
                const int x = ((volatile int *)shp(0)->slot[buf][r])[0];
                const int y = ((volatile int *)shp(0)->slot[buf][r])[1];
                if (r < rank) { o += x; o2 += y; }
                t += x;
                t2 += y;
            }
            sh.red[0] = o; sh.red[1] = t; sh.red[2] = o2; sh.red[3] = t2;
        }
        __syncthreads();
        off = sh.red[0]; tot = sh.red[1]; off2 = sh.red[2]; tot2 = sh.red[3];
        __syncthreads();
    }

    // ---- the residual graph on rank 0
    //
    // Once the live graph is small, rank 0 takes it over as a compact CSR in
    // its own shared memory and runs the remaining rounds of the unbounded
    // rules alone: block barriers and local shared-memory atomics instead of
    // cluster barriers and remote ones, while the other CTAs wait at one
    // cluster barrier.  The live vertices are renumbered in increasing order,
    // so every tie-break (lowest index) decides as it would have in the
    // cluster, and the rounds reach the same fixpoint.  The forced bits and
    // degrees go back to their owners afterwards, so the later stages (greedy
    // bound, bounded rules, induced graph, forced list) see the state the
    // cluster rounds would have left.  Row entries and degrees are 16-bit.
    static constexpr int kResHeavyRow = 32;     // longer rows are applied by a whole warp
    static constexpr int kResPerVertex = 11;    // bound on the layout's bytes per vertex
    static constexpr int kResSlack = 128;
    static constexpr int kResNever = 1 << 26;   // a per-CTA bound that never fits
    static constexpr int kResNone = 0xffff;     // no vertex (ids are below it); sorts last
    static constexpr int kResWarpScan = 8;      // longer original rows are compacted by a warp at the hand-off

    __device__ static size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    // rank 0's layout: row offsets (int), row entries (u16), degrees (u16),
    // forced / mark / frontier bitmaps, one vertex list; at most
    // kResPerVertex * np + 2 * m2p + kResSlack bytes
    __device__ static size_t residual_bytes(int np, long long m2p)
    {
        const size_t w = (size_t)(np + 31) / 32 * 4;
        return a16(4 * ((size_t)np + 1)) + a16(2 * (size_t)m2p) + a16(2 * (size_t)np) + 3 * a16(w) +
               a16(4 * (size_t)np);
    }
    __device__ int residual_room() const { return smem_cap - res_off; }

    // The rounds on the residual graph run on the whole of rank 0's block
    // (named barrier 1).  Even a round of a few dozen vertices is faster on
    // the block than on one warp: its cost is the dependent shared-memory
    // chain of examining one vertex, and a warp examines several in turn.
    static constexpr int kSoloThreads = kRootThreads;
    template <int NT>
    __device__ __forceinline__ static void solo_sync()
    {
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    }

    // rank 0's residual graph and its state (new ids)
    struct Solo {
        int *rrp;
        uint16_t *rcol, *rdeg;
        uint32_t *rforced, *rmark, *rflag;
        int *rlist;
        int np, nw;
    };

    // Append the set bits of words[0, nw) (cleared here) that are not in
    // forced[] to list as indices, in any order, counting in *counter; with
    // fold, forced[] gets them, else (a frontier) only those of degree 1 or 2
    // are kept.  Called by the first NT threads.
    template <int NT>
    __device__ __forceinline__ static void solo_list(uint32_t *words, int nw, uint32_t *forced, bool fold,
                                                     const uint16_t *deg, int *list, int *counter)
    {
        for (int j = threadIdx.x; j < nw; j += NT) {
            uint32_t x = words[j];
            if (!x) continue;
            words[j] = 0;
            x &= ~forced[j];
            if (fold) forced[j] |= x;
            else x = low_degree_bits(x, deg + j * 32);
            if (!x) continue;
            int k = atomicAdd(counter, __popc(x));
            while (x) {
                list[k++] = j * 32 + __ffs(x) - 1;
                x &= x - 1;
            }
        }
    }

    // One round of the unbounded rules on the listed frontier rlist[0,
    // fsize), by the first NT threads of rank 0: examine, list the marks
    // (folded into the forced bits), apply their rows.  Three barriers;
    // returns the number of vertices forced.
    template <int NT>
    __device__ int solo_round(const Solo &R, int fsize)
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int np = R.np;
        const int *rrp = R.rrp;
        const uint16_t *rcol = R.rcol;
        const volatile uint16_t *vdeg = R.rdeg;
        const volatile uint32_t *vforced = R.rforced;
        auto rlive = [&](int x) { return x < np && !((vforced[x >> 5] >> (x & 31)) & 1u) && vdeg[x] > 0; };
        auto rdec = [&](int x) {
            unsigned *w = (unsigned *)((char *)R.rdeg + 2 * (x & ~1));
            atomicSub(w, 1u << (16 * (x & 1)));
        };
        auto rbit = [&](uint32_t *words, int x) { atomicOr(&words[x >> 5], 1u << (x & 31)); };
        for (int i = threadIdx.x; i < fsize; i += NT) {
            const int v = R.rlist[i];
            if ((vforced[v >> 5] >> (v & 31)) & 1u) continue;
            const int dv = vdeg[v];
            if (dv == 0 || dv > 2) continue;
            int u = -1, w = -1;
            const int a = rrp[v], b = rrp[v + 1];
            for (int e0 = a; e0 < b; e0 += 8) {
                int xs[8];
                bool lv[8];
#pragma unroll
                for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? rcol[e0 + j] : kResNone;
#pragma unroll
                for (int j = 0; j < 8; j++) lv[j] = rlive(xs[j]);
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (lv[j] && w < 0) {
                        if (u < 0) u = xs[j]; else w = xs[j];
                    }
                if (dv == 1 ? u >= 0 : w >= 0) break;
            }
            if (dv == 1) {
                if (u < 0) continue;
                if (vdeg[u] == 1 && u < v) rbit(R.rflag, u);   // u's rule fires instead
                else rbit(R.rmark, u);
            } else if (w >= 0) {
                // u-w an edge?  search the shorter row (sorted)
                const bool by_u = rrp[u + 1] - rrp[u] <= rrp[w + 1] - rrp[w];
                int lo = by_u ? rrp[u] : rrp[w], hi = (by_u ? rrp[u + 1] : rrp[w + 1]) - 1;
                const int key = by_u ? w : u;
                bool tri = false;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1, x = rcol[mid];
                    if (x == key) { tri = true; break; }
                    if (x < key) lo = mid + 1; else hi = mid - 1;
                }
                if (tri) {
                    int pv = INT_MAX;
                    if (vdeg[u] == 2 && u < v) pv = u;
                    if (vdeg[w] == 2 && w < v && w < pv) pv = w;
                    if (pv != INT_MAX) rbit(R.rflag, pv);
                    else { rbit(R.rmark, u); rbit(R.rmark, w); }
                }
            }
        }
        solo_sync<NT>();                                              // examined
        if (threadIdx.x == 0) sh.cnt = 0;   // (fsize is read; the next listing follows two barriers)
        solo_list<NT>(R.rmark, R.nw, R.rforced, true, R.rdeg, R.rlist, &sh.fcnt);
        solo_sync<NT>();                                              // marks listed
        const int cnt = *(volatile int *)&sh.fcnt;
        // apply: a row by its thread, or by the whole warp when long; a
        // forced vertex's row is applied with no test: its neighbours'
        // degrees count it, so none goes below zero
        for (int base = warp * 32; base < cnt; base += NT) {
            const int i = base + lane;
            int u = -1, a = 0, b = 0;
            if (i < cnt) {
                u = R.rlist[i];
                a = rrp[u];
                b = rrp[u + 1];
            }
            const bool wide = b - a > kResHeavyRow;
            if (!wide) {
                for (int e = a; e < b; e++) {
                    const int x = rcol[e];
                    if (x < np) { rdec(x); rbit(R.rflag, x); }
                }
            }
            unsigned hm = __ballot_sync(kFull, wide);
            while (hm) {
                const int src = __ffs(hm) - 1;
                hm &= hm - 1;
                const int aa = __shfl_sync(kFull, a, src), bb = __shfl_sync(kFull, b, src);
                for (int e = aa + lane; e < bb; e += 32) {
                    const int x = rcol[e];
                    if (x < np) { rdec(x); rbit(R.rflag, x); }
                }
            }
        }
        solo_sync<NT>();                                              // applied
        if (threadIdx.x == 0) sh.fcnt = 0;  // (cnt is read; the next listing follows two barriers)
        return cnt;
    }

    // The unbounded rules on the residual graph (rank 0 alone); the owners
    // read the results from rank 0's shared memory afterwards.  Input: Q.rp2
    // / Q.col2 (the CSR, new ids), Q.fr1 (degree | frontier bit << 16).
    __device__ void solo_rounds(int np, int m2p)
    {
        Solo R;
        char *p = lsm + res_off;
        R.rrp = (int *)p;               p += a16(4 * ((size_t)np + 1));
        R.rcol = (uint16_t *)p;         p += a16(2 * (size_t)m2p);
        R.rdeg = (uint16_t *)p;         p += a16(2 * (size_t)np);
        const int nw = (np + 31) / 32;
        R.rforced = (uint32_t *)p;      p += a16(4 * (size_t)nw);
        R.rmark = (uint32_t *)p;        p += a16(4 * (size_t)nw);
        R.rflag = (uint32_t *)p;        p += a16(4 * (size_t)nw);
        R.rlist = (int *)p;
        R.np = np;
        R.nw = nw;
        const int T = blockDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        // the copy in: eight independent loads in flight per thread
        for (int i0 = threadIdx.x; i0 <= np; i0 += 8 * T) {
            int xs[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xs[j] = i0 + j * T <= np ? __ldcg(Q.rp2 + i0 + j * T) : 0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (i0 + j * T <= np) R.rrp[i0 + j * T] = xs[j];
        }
        for (int e0 = threadIdx.x; e0 < m2p; e0 += 8 * T) {
            int xs[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xs[j] = e0 + j * T < m2p ? __ldcg(Q.col2 + e0 + j * T) : 0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (e0 + j * T < m2p) R.rcol[e0 + j * T] = (uint16_t)(xs[j] >= 0 && xs[j] < np ? xs[j] : kResNone);
        }
        // degrees and frontier bits: four words per warp in flight
        const int nwarps = T >> 5;
        for (int j0 = warp; j0 < nw; j0 += 4 * nwarps) {
            int xs[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = (j0 + k * nwarps) * 32 + lane;
                xs[k] = i < np ? __ldcg(Q.fr1 + i) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int j = j0 + k * nwarps;
                if (j >= nw) break;   // (uniform over the warp)
                const int i = j * 32 + lane;
                if (i < np) R.rdeg[i] = (uint16_t)(xs[k] & 0xffff);
                const unsigned f = __ballot_sync(kFull, (xs[k] >> 16) & 1);
                if (lane == 0) { R.rflag[j] = f; R.rforced[j] = 0; R.rmark[j] = 0; }
            }
        }
        if (threadIdx.x == 0) { sh.cnt = 0; sh.fcnt = 0; }
        __syncthreads();
        int forced_cnt = 0, rounds = 0;
        for (int guard = 0; guard <= 2 * np + 2; guard++) {
            solo_list<kSoloThreads>(R.rflag, nw, R.rforced, false, R.rdeg, R.rlist, &sh.cnt);
            solo_sync<kSoloThreads>();                                // frontier listed
            const int fsize = *(volatile int *)&sh.cnt;
            if (fsize == 0) break;
            forced_cnt += solo_round<kSoloThreads>(R, fsize);
            rounds++;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            sh.solo_forced = forced_cnt;
            Q.rounds += rounds;
        }
    }

    // Hand the live graph to rank 0 when its layout fits there.  Called by
    // every thread of every CTA at the top of a round of the unbounded rules
    // (the last round's decrements have landed); returns the same in every
    // CTA: true when the rounds are finished (ftot updated), false when the
    // graph did not fit after all (nothing changed).
    __device__ bool residual_solo()
    {
        const int T = blockDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int wpr = chunk >> 5, nwa = C * wpr;
        const uint32_t *fw = lrep() + (rank << (cs - 5));
        // My live vertices as a bitmap, in my part of lnew() (the round's
        // degree update is done with it); the other CTAs read it after the
        // cluster barrier of the prefix exchange.
        uint32_t *lv = lnew();
        for (int w = warp; w < wpr; w += T >> 5) {
            const int i = w * 32 + lane;
            const bool l = i < vcnt && !((fw[w] >> lane) & 1u) && ldeg()[i] > 0;
            const unsigned b = __ballot_sync(kFull, l);
            if (lane == 0) lv[rank * wpr + w] = b;
        }
        const int per = (vcnt + T - 1) / T;
        const int beg = min(vcnt, (int)threadIdx.x * per), end = min(vcnt, ((int)threadIdx.x + 1) * per);
        int cnt = 0, dsum = 0;
        for (int i = beg; i < end; i++) {
            const int dv = ldeg()[i];
            if (dv > 0 && !((fw[i >> 5] >> (i & 31)) & 1u)) { cnt++; dsum += dv; }
        }
        int lnp, lm2;
        const int loff = block_excl_scan(cnt, sh.red, &lnp);
        const int leoff = block_excl_scan(dsum, sh.red, &lm2);
        int coff, np, ceoff, m2p;
        exchange_prefix(lnp, lm2, coff, np, ceoff, m2p);
        if (np == 0 || np >= kResNone || residual_bytes(np, m2p) > (size_t)residual_room())
            return false;
        // The whole live bitmap in every CTA, and the live vertices before
        // each word (in lprev(), whose degrees no later round needs): a live
        // vertex x gets the new id pref[x / 32] + (live vertices of its word
        // below it), the same id its owner gives it below.
        for (int w = threadIdx.x; w < nwa; w += T) {
            const int r = w / wpr;
            if (r != rank) lv[w] = ((volatile uint32_t *)(base(r) + 2 * (size_t)chunk + repb))[w];
        }
        __syncthreads();
        int *pref = (int *)lprev();
        {
            const int k = (nwa + T - 1) / T;
            const int w0 = min(nwa, (int)threadIdx.x * k), w1 = min(nwa, ((int)threadIdx.x + 1) * k);
            int c = 0;
            for (int w = w0; w < w1; w++) c += __popc(lv[w]);
            int tot;
            int o = block_excl_scan(c, sh.red, &tot);
            for (int w = w0; w < w1; w++) {
                pref[w] = o;
                o += __popc(lv[w]);
            }
        }
        __syncthreads();
        // New ids in increasing vertex order (thread ranges are in order);
        // degree and frontier bit travel in Q.fr1.  Each live vertex's row
        // is its live neighbours, renumbered, in the order of the original
        // row (its degree counts them, so the row is full when that many
        // are found): written here, or, for an original row longer than
        // kResWarpScan, listed (Q.deg / Q.heavy / Q.flag: vertex, offset,
        // degree) and written by a warp below.
        const uint32_t *flw = lflag();
        if (threadIdx.x == 0) sh.tcnt = 0;
        __syncthreads();
        int id = coff + loff, eo = ceoff + leoff;
        for (int i = beg; i < end; i++) {
            const int dv = ldeg()[i];
            if (dv == 0 || ((fw[i >> 5] >> (i & 31)) & 1u)) continue;
            const int v = vbeg + i;
            Q.rp2[id] = eo;
            Q.fr1[id] = dv | (int)(((flw[i >> 5] >> (i & 31)) & 1u) << 16);
            id++;
            int a, b;
            const int *cp;
            own_row(v, a, b, cp);
            int o = eo;
            const int lim = eo + dv;
            if (b - a > kResWarpScan) {
                const int k = vbeg + atomicAdd(&sh.tcnt, 1);
                Q.deg[k] = v;
                Q.heavy[k] = eo;
                Q.flag[k] = dv;
                eo = lim;
                continue;
            }
            for (int e0 = a; e0 < b && o < lim; e0 += 8) {
                int xs[8];
#pragma unroll
                for (int j = 0; j < 8; j++) xs[j] = e0 + j < b ? cp[e0 + j] : -1;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int x = xs[j];
                    if (x < 0 || o >= lim) continue;
                    const uint32_t word = lv[x >> 5], bit = 1u << (x & 31);
                    if (word & bit) Q.col2[o++] = pref[x >> 5] + __popc(word & (bit - 1));
                }
            }
            while (o < lim) Q.col2[o++] = -1;   // (never: the degree counts the live neighbours)
            eo = lim;
        }
        __syncthreads();
        const int nlong = sh.tcnt;
        for (int k = warp; k < nlong; k += T >> 5) {
            const int v = Q.deg[vbeg + k];
            int o = Q.heavy[vbeg + k];
            const int lim = o + Q.flag[vbeg + k];
            int a, b;
            const int *cp;
            own_row(v, a, b, cp);
            for (int e0 = a; e0 < b && o < lim; e0 += 32) {           // (o is the same in every lane)
                const int e = e0 + lane;
                const int x = e < b ? cp[e] : -1;
                uint32_t word = 0, bit = 0;
                if (x >= 0) {
                    word = lv[x >> 5];
                    bit = 1u << (x & 31);
                }
                const bool l = (word & bit) != 0;
                const unsigned m = __ballot_sync(kFull, l);
                const int at = o + __popc(m & ((1u << lane) - 1u));
                if (l && at < lim) Q.col2[at] = pref[x >> 5] + __popc(word & (bit - 1));
                o += __popc(m);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < wpr; i += T) lflag()[i] = 0;   // carried in Q.fr1 now
        if (rank == 0 && threadIdx.x == 0) Q.rp2[np] = m2p;
        cl.sync();
        if (rank == 0) solo_rounds(np, m2p);
        cl.sync();   // the residual graph's degrees and forced bits are final
        // My vertices that were live at the hand-off take their degree and
        // forced bit from rank 0's residual layout (new id from the live
        // bitmap and the prefix counts, which are unchanged); a warp takes
        // one word of my vertices.  The next cluster barrier (the caller's)
        // orders these for the other CTAs.
        {
            const char *q0 = base(0) + res_off + a16(4 * ((size_t)np + 1)) + a16(2 * (size_t)m2p);
            const volatile uint16_t *rdeg0 = (const volatile uint16_t *)q0;
            const volatile uint32_t *rforced0 = (const volatile uint32_t *)(q0 + a16(2 * (size_t)np));
            uint32_t *own = lrep() + (rank << (cs - 5));
            for (int w = warp; w < wpr; w += T >> 5) {
                const int gw = rank * wpr + w;
                const uint32_t word = lv[gw];
                bool f = false;
                if ((word >> lane) & 1u) {
                    const int nid = pref[gw] + __popc(word & ((1u << lane) - 1u));
                    ldeg()[w * 32 + lane] = rdeg0[nid];
                    f = (rforced0[nid >> 5] >> (nid & 31)) & 1u;
                }
                const unsigned fm = __ballot_sync(kFull, f);
                if (lane == 0 && fm) own[w] |= fm;
            }
        }
        ftot += *(volatile int *)&shp(0)->solo_forced;
        if (rank == 0) {
            if (threadIdx.x == 0) Q.forced = ftot;
            lrp = nullptr;   // the residual graph overwrote rank 0's staged rows
            lcol = nullptr;
            lsrc = nullptr;
        }
        return true;
    }

    // Synchronous rounds, two cluster barriers each:
    //   B1  every CTA has brought its degrees and frontier up to date with
    //       the last round's marks, and that round's totals (published
    //       before B1) are read: stop when it marked nothing and left no
    //       frontier
    //   B2  this round's marks and handed-over frontier bits have landed;
    //       every CTA then reads all of the round's marks into its copy of
    //       the forced bitmap and updates the degrees of its own vertices
    //       (no remote writes after B2)
    // Marks alternate between two bitmaps: the bitmap of round r is read by
    // every CTA between B2 of round r and the next B1, and its owner clears
    // it in round r + 1, before round r + 2 marks it again.
    __device__ bool reduce_rounds(bool hd, int bound)
    {
        int *fl = Q.fr0 + vbeg;        // my frontier list
        int *hv = Q.aux + vbeg;        // vertices whose rows are scanned by a warp
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
        uint32_t *lm = lmark();        // my two mark bitmaps (contiguous)
        if (hd) refresh_forced_copy();
        for (int i = threadIdx.x; i < chunk / 16; i += blockDim.x) lm[i] = 0;
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) lprev()[i] = ldeg()[i];
        int pi0 = 0, pe0 = 0, pe1 = 0;
        if (!lsrc) pull_range(pi0, pe0, pe1);
        bool first = true, last_full = false;
        long long delta = INT_MAX;
        int last_all = 0;
        for (int rnd = 0;; rnd++) {
            cl.sync();                                                    // B1
            if (!first) {
                collect();
                const long long tpend = sh.tot[1];
                if (last_full) delta = sh.tot[3];
                if (last_all == 0 && tpend == 0) return true;
                // the bound on the live graph's layout, from the last round
                if (!hd && sh.tot[2] + kResSlack <= residual_room() && residual_solo()) return true;
            }
            const int bud = hd ? bound - ftot - 1 : INT_MAX;
            if (hd && bud < 0) return false;
            const bool full = first || (hd && delta > bud);
            first = false;
            last_full = full;
            mbuf = rnd & 1;
            for (int i = threadIdx.x; i < (chunk >> 5); i += blockDim.x) lm[(mbuf ^ 1) * (chunk >> 5) + i] = 0;
            if (threadIdx.x == 0) { sh.hcnt = 0; sh.tcnt = 0; }
            const int fsize = frontier_to_list(fl);                       // (ends with a block barrier)
            int dmax = 0;
            if (full) {
                for (int i = threadIdx.x; i < vcnt; i += blockDim.x)
                    if (!rforced(vbeg + i)) dmax = max(dmax, (int)ldeg()[i]);
                for (int i = threadIdx.x; i < vcnt; i += blockDim.x) examine(hv, vbeg + i, bud);
            } else {
                for (int i = threadIdx.x; i < fsize; i += blockDim.x) examine(hv, fl[i], bud);
            }
            __syncthreads();
            const int hc = sh.hcnt;
            for (int i = warp; i < hc; i += nwarps) {
                const int v = hv[i];
                const int dv = ldeg()[v - vbeg];
                int u, w;
                warp_live_nbrs(v, dv, u, w);
                if (lane == 0) {
                    if (dv == 1) { if (u >= 0) decide_one(v, u); }
                    else if (w >= 0) list_triangle(v, u, w);
                }
            }
            __syncthreads();
            // the triangle checks of the round, spread evenly over the block
            const int tc = sh.tcnt;
            for (int i = threadIdx.x; i < tc; i += blockDim.x)
                decide_triangle(Q.deg[vbeg + i], Q.heavy[vbeg + i], Q.flag[vbeg + i]);
            const int dm = full ? block_max(dmax, sh.red) : 0;
            cl.sync();                                                    // B2
            const int all = gather_marks();                               // (ends with a block barrier)
            ftot += all;
            last_all = all;
            if (rank == 0 && threadIdx.x == 0) { Q.forced = ftot; Q.rounds++; }
            if (all > 0) {
                if (lsrc) pull_flat();
                else pull_walk(pi0, pe0, pe1);
            }
            int pend = 0, est = 0;
            __syncthreads();
            // The next frontier: the live vertices whose degree changed to 1
            // or 2, added to the bits other CTAs handed over (a warp takes
            // 32 consecutive vertices, one frontier word).  The live graph
            // only shrinks from here: its vertices and degrees bound the
            // residual layout at the next round.
            {
                const uint32_t *fw = lrep() + (rank << (cs - 5));
                uint16_t *pv = lprev();
                for (int w = warp; w < (chunk >> 5); w += nwarps) {
                    const int i = w * 32 + lane;
                    int dv = 0;
                    bool fr = false;
                    if (i < vcnt && !((fw[w] >> lane) & 1u)) {
                        dv = ldeg()[i];
                        fr = dv != pv[i] && (dv == 1 || dv == 2);
                        pv[i] = (uint16_t)dv;
                        if (!hd && dv > 0) est += kResPerVertex + 2 * dv;
                    }
                    const unsigned f = __ballot_sync(kFull, fr);
                    if (lane == 0) {
                        const uint32_t x = lflag()[w] | f;
                        lflag()[w] = x;
                        pend += __popc(x);
                    }
                }
            }
            block_sum2(pend, est, sh.red, sh.red2);
            publish(0, pend, hd ? kResNever : min(est, kResNever), dm);   // read by every CTA after the next B1
        }
    }

    __device__ long long live_edges2()
    {
        cl.sync();   // every decrement of the last round has landed
        int e2 = 0;
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x)
            if (!forced(vbeg + i)) e2 += d(vbeg + i);
        e2 = block_sum(e2, sh.red);
        exchange(e2, 0, 0, 0);
        return sh.tot[0];
    }

    __device__ int greedy()
    {
        int *aux = Q.aux, *join = Q.fr0;
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) aux[vbeg + i] = live(vbeg + i) ? 0 : 3;
        cl.sync();
        for (;;) {
            int any = 0;
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x) {
                const int v = vbeg + i;
                if (__ldcg(aux + v) != 0) continue;
                const unsigned long long pv = ((unsigned long long)d(v) << 32) | mix32((unsigned)v);
                bool j = true;
                int a, b;
                const int *cp;
                own_row(v, a, b, cp);
                for (int e = a; e < b && j; e++) {
                    const int x = cp[e];
                    const int ax = ((volatile int *)aux)[x];
                    if (ax == 1) j = false;
                    else if (ax == 0) {
                        const unsigned long long px = ((unsigned long long)d(x) << 32) | mix32((unsigned)x);
                        if (px < pv || (px == pv && x < v)) j = false;
                    }
                }
                join[v] = j;
            }
            cl.sync();
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x) {
                const int v = vbeg + i;
                if (__ldcg(aux + v) == 0 && join[v]) { aux[v] = 4; any = 1; }
            }
            any = block_sum(any, sh.red);
            exchange(any, 0, 0, 0);
            if (sh.tot[0] == 0) break;
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x) {
                const int v = vbeg + i;
                if (__ldcg(aux + v) != 4) continue;
                int a, b;
                const int *cp;
                own_row(v, a, b, cp);
                for (int e = a; e < b; e++) atomicCAS(&aux[cp[e]], 0, 2);
            }
            cl.sync();
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x)
                if (__ldcg(aux + vbeg + i) == 4) aux[vbeg + i] = 1;
            cl.sync();
        }
        int c = 0;
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) {
            const int v = vbeg + i;
            const int av = __ldcg(aux + v);
            const bool g = av == 2 || av == 0;
            Q.cover_flags[v] = (forced(v) || g) ? 1 : 0;
            c += g;
        }
        c = block_sum(c, sh.red);
        exchange(c, 0, 0, 0);
        const int tot = (int)sh.tot[0];
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) aux[vbeg + i] = 0;
        cl.sync();
        return tot;
    }

    __device__ void induce()
    {
        const int T = blockDim.x;
        const int per = (vcnt + T - 1) / T;
        const int beg = vbeg + min(vcnt, (int)threadIdx.x * per), end = vbeg + min(vcnt, ((int)threadIdx.x + 1) * per);
        int cnt = 0, dsum = 0, dmax = 0;
        for (int v = beg; v < end; v++)
            if (live(v)) { cnt++; dsum += d(v); dmax = max(dmax, d(v)); }
        int lnp, lm2;
        const int loff = block_excl_scan(cnt, sh.red, &lnp);
        const int leoff = block_excl_scan(dsum, sh.red, &lm2);
        const int ldm = block_max(dmax, sh.red);
        int coff, np, ceoff, m2p;
        exchange_prefix(lnp, lm2, coff, np, ceoff, m2p);
        exchange(0, 0, 0, ldm);
        const int dm = (int)sh.tot[3];
        int *nid = Q.aux;
        int id = coff + loff, eo = ceoff + leoff;
        for (int v = beg; v < end; v++) {
            if (live(v)) {
                nid[v] = id;
                Q.orig[id] = v;
                Q.rp2[id] = eo;
                id++;
                eo += d(v);
            } else {
                nid[v] = -1;
            }
        }
        if (rank == 0 && threadIdx.x == 0) {
            Q.rp2[np] = m2p;
            Q.np = np;
            Q.m2p = m2p;
            Q.maxdeg = dm;
        }
        cl.sync();
        for (int i = coff + threadIdx.x; i < coff + lnp; i += T) {
            const int v = Q.orig[i];
            int o = Q.rp2[i];
            int a, b;
            const int *cp;
            own_row(v, a, b, cp);
            for (int e = a; e < b; e++) {
                const int nx = ((volatile int *)nid)[cp[e]];
                if (nx >= 0) Q.col2[o++] = nx;
            }
        }
        cl.sync();
        for (int i = threadIdx.x; i < vcnt; i += T) nid[vbeg + i] = 0;
        cl.sync();
    }

    // forced bit of owned vertex i, through the local window
    __device__ __forceinline__ bool own_forced(int i) const
    {
        return ((const volatile uint32_t *)lrep())[(rank << (cs - 5)) + (i >> 5)] >> (i & 31) & 1u;
    }

    __device__ void publish()
    {
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) Q.st[vbeg + i] = own_forced(i) ? 1 : 0;
    }

    // The answer is the forced set: write it as the ascending output list
    // (cover_list, and cover_out when set) here instead of in a separate
    // finalisation launch.  Each thread takes four consecutive words of this
    // CTA's forced bitmap, so thread order is id order; CTAs are ordered by
    // rank.  The ids are gathered in shared memory first (the staged rows
    // are not needed any more), so that consecutive threads store
    // consecutive entries.  One cluster barrier.  Called by every thread of
    // every CTA.
    __device__ void list_forced()
    {
        const volatile uint32_t *fw = lrep() + (rank << (cs - 5));
        const int nw = chunk >> 5;
        uint32_t m[4];
        int c = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int i = threadIdx.x * 4 + j;
            m[j] = i < nw ? fw[i] : 0u;
            c += __popc(m[j]);
        }
        int mine;
        int off = block_excl_scan(c, sh.red, &mine);
        int *list = Q.cover_list, *out = Q.cover_out;
        const bool staged = (size_t)smem_cap >= (size_t)res_off + 4 * (size_t)chunk;   // (uniform)
        int *stage = (int *)(lsm + res_off);
        if (staged) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                uint32_t x = m[j];
                const int v0 = vbeg + (threadIdx.x * 4 + j) * 32;
                while (x) {
                    stage[off++] = v0 + __ffs(x) - 1;
                    x &= x - 1;
                }
            }
        }
        int cta_off, all, o2, t2;
        exchange_prefix(mine, 0, cta_off, all, o2, t2);   // (its block barriers order the staging)
        if (staged) {
            for (int k = threadIdx.x; k < mine; k += blockDim.x) {
                const int v = stage[k];
                list[cta_off + k] = v;
                if (out) out[cta_off + k] = v;
            }
        } else {
            off += cta_off;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                uint32_t x = m[j];
                const int v0 = vbeg + (threadIdx.x * 4 + j) * 32;
                while (x) {
                    const int v = v0 + __ffs(x) - 1;
                    list[off] = v;
                    if (out) out[off] = v;
                    off++;
                    x &= x - 1;
                }
            }
        }
        if (rank == 0 && threadIdx.x == 0) {
            Q.cover_len = all;
            Q.listed = 1;
        }
    }

    __device__ void run()
    {
        if (rank == 0) {
            prefetch_l2(rp, (size_t)(n + 1) * 4);
            prefetch_l2(col, (size_t)Q.m2 * 4);
        }
        for (int i = threadIdx.x; i < vcnt; i += blockDim.x) {
            const int v = vbeg + i;
            ldeg()[i] = (uint16_t)(lcol ? lrp[i + 1] - lrp[i] : __ldg(rp + v + 1) - __ldg(rp + v));
            Q.aux[v] = 0;
            Q.cover_flags[v] = 0;
        }
        if (rank == 0 && threadIdx.x == 0) {
            Q.forced = 0;
            Q.np = 0; Q.m2p = 0; Q.maxdeg = 0; Q.answered = 0; Q.greedy = -1;
            Q.improved = 0; Q.result = -1; Q.yes = 0; Q.cover_len = 0;
            Q.rounds = 0;
            Q.listed = 0;
            for (int i = 0; i < 4; i++) Q.root_cycles[i] = 0;
        }
        cl.sync();
        long long t0 = clock64();
        if (!Q.skip_root_rules) reduce_rounds(false, INT_MAX);
        long long t1 = clock64();
        if (rank == 0 && threadIdx.x == 0) Q.root_cycles[0] = t1 - t0;
        if (live_edges2() == 0) {
            publish();
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x) Q.cover_flags[vbeg + i] = own_forced(i);
            if (rank == 0 && threadIdx.x == 0) {
                Q.answered = 1;
                Q.bound = ftot;
                if (Q.k < 0) { Q.result = ftot; Q.yes = 1; }
                else { Q.yes = ftot <= Q.k; Q.result = Q.yes ? ftot : -1; }
            }
            if ((Q.k < 0 || ftot <= Q.k) && !Q.emit_complement && Q.cover_list) list_forced();   // uniform
            return;
        }
        const int greedy_size = ftot + greedy();
        t0 = clock64();
        if (rank == 0 && threadIdx.x == 0) { Q.greedy = greedy_size; Q.root_cycles[1] = t0 - t1; }
        if (Q.k >= 0 && greedy_size <= Q.k) {
            publish();
            if (rank == 0 && threadIdx.x == 0) {
                Q.answered = 1; Q.bound = greedy_size; Q.yes = 1; Q.result = greedy_size;
            }
            return;
        }
        const int bound = Q.k >= 0 ? Q.k + 1 : greedy_size;
        const bool feasible = Q.skip_root_rules ? true : reduce_rounds(true, bound);
        t1 = clock64();
        if (rank == 0 && threadIdx.x == 0) Q.root_cycles[2] = t1 - t0;
        const long long e2 = live_edges2();
        publish();
        if (!feasible || ftot >= bound) {
            if (rank == 0 && threadIdx.x == 0) {
                Q.answered = 1; Q.bound = bound;
                if (Q.k < 0) { Q.result = greedy_size; Q.yes = 1; }
                else { Q.yes = 0; Q.result = -1; }
            }
            return;
        }
        if (e2 == 0) {
            for (int i = threadIdx.x; i < vcnt; i += blockDim.x) Q.cover_flags[vbeg + i] = own_forced(i);
            if (rank == 0 && threadIdx.x == 0) {
                Q.answered = 1; Q.bound = bound; Q.result = ftot; Q.yes = 1;
            }
            if (!Q.emit_complement && Q.cover_list) list_forced();
            return;
        }
        induce();
        if (rank == 0 && threadIdx.x == 0) { Q.bound = bound; Q.root_cycles[3] = clock64() - t1; }
    }
};

__global__ void __launch_bounds__(kRootThreads, 1) root_cluster_kernel(QueryDesc *qs, int cs, int smem_bytes)
{
    extern __shared__ __align__(16) char root_smem[];
    __shared__ ClusterShared sh;
    QueryDesc &Q = qs[0];
    if (Q.status != VC_OK) return;   // uniform across the cluster
    ClusterRoot r(Q, sh, root_smem, cs, smem_bytes);
    cgx::this_cluster().sync();      // remote addresses and zeroed bitmaps everywhere
    r.run();
    cgx::this_cluster().sync();      // nobody leaves while others may touch its shared memory
}

// ------------------------------------------------------------ final answer

// Assemble each query's cover in original ids: the root-forced vertices plus
// the witness of the induced graph's registry entry when the search improved
// on the bound; otherwise the root phase's cover (greedy or forced set).
// Called by every thread of the block.
__device__ void finalize_query(QueryDesc &Q, const RegEntry *reg, const uint32_t *reg_words, int wcap, int *red)
{
    if (Q.listed) return;   // the root phase wrote the list already
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
    const bool flip = Q.emit_complement != 0;   // the vertices outside the cover
    int c = 0;
    if (emit)
        for (int v = beg; v < end; v++) c += (Q.cover_flags[v] != 0) != flip;
    int tot;
    int off = block_excl_scan(c, red, &tot);
    int *out = Q.cover_out;
    if (emit)
        for (int v = beg; v < end; v++)
            if ((Q.cover_flags[v] != 0) != flip) {
                Q.cover_list[off] = v;
                if (out) out[off] = v;
                off++;
            }
    if (threadIdx.x == 0) Q.cover_len = emit ? tot : 0;
}

// mode 0: every query; 1: only those the root phase settled; 2: only the
// searched ones (the others were finalised after the root phase)
__global__ void __launch_bounds__(kRootThreads) finalize_kernel(QueryDesc *qs, const RegEntry *reg,
                                                                 const uint32_t *reg_words, int wcap, int mode)
{
    __shared__ int red[33];
    QueryDesc &Q = qs[blockIdx.x];
    if (Q.status != VC_OK) {
        // a search stopped early keeps its incumbent as the best size known
        if (mode == 2 && !Q.answered && Q.np > 0 && threadIdx.x == 0) Q.best = Q.forced + reg[Q.root_entry].val;
        return;
    }
    if ((mode == 1 && !Q.answered) || (mode == 2 && Q.answered)) return;
    finalize_query(Q, reg, reg_words, wcap, red);
}

// ------------------------------------------------------------ crown reduction
//
// The crown rule at the root (Section 4.2; the paper cites it without
// defining it), applied as the Nemhauser-Trotter reduction, which removes
// every crown: a maximum matching of the bipartite double cover (u_L - v_R
// for every edge uv) gives, through Koenig's theorem, a minimum cover C_B of
// the double cover and so a half-integral optimal LP solution
// x_v = (|{v_L, v_R} & C_B|) / 2.  Some minimum vertex cover contains every
// vertex with x = 1 and no vertex with x = 0 (whose neighbours all have
// x = 1), so those go to the cover / are dropped and the search runs on the
// x = 1/2 part.  The matching is Hopcroft-Karp: layered BFS from the free L
// vertices, then vertex-disjoint shortest augmenting paths found by parallel
// DFS with exclusive claims on R vertices (per-vertex edge pointers and
// parent links instead of stacks).  Before anything is removed, C_B is
// checked to be a cover of the double cover of size |matching| (so it is
// minimum); if not, nothing is removed.  One block per query, on the
// induced graph of the root phase.
__global__ void __launch_bounds__(kRootThreads) crown_kernel(QueryDesc *qs)
{
    __shared__ int red[33];
    __shared__ int s_a, s_b, s_c;
    QueryDesc &Q = qs[blockIdx.x];
    if (Q.status != VC_OK || Q.answered || Q.np <= 0 || Q.crown_ws == nullptr) return;
    const int n = Q.np, T = blockDim.x, t = threadIdx.x;
    const int *rp = Q.rp2, *col = Q.col2;
    int *w = Q.crown_ws;
    int *mateL = w, *mateR = w + n, *dL = w + 2 * n, *dR = w + 3 * n, *used = w + 4 * n, *itp = w + 5 * n,
        *parL = w + 6 * n, *fa = w + 7 * n, *fb = w + 8 * n, *x2 = w + 9 * n, *rpn = w + 10 * n,
        *orn = w + 11 * n + 1, *coln = w + 12 * n + 1;
    const int INF = INT_MAX;
    for (int u = t; u < n; u += T) { mateL[u] = -1; mateR[u] = -1; }
    __syncthreads();
    for (int u = t; u < n; u += T)                       // greedy start
        for (int e = rp[u]; e < rp[u + 1]; e++)
            if (atomicCAS(&mateR[col[e]], -1, u) == -1) { mateL[u] = col[e]; break; }
    __syncthreads();

    for (int phase = 0; phase <= n; phase++) {
        // ---- layered BFS from the free L vertices
        if (t == 0) { s_a = 0; s_b = 0; }
        __syncthreads();
        for (int u = t; u < n; u += T) {
            dR[u] = INF;
            if (__ldcg(mateL + u) < 0) { dL[u] = 0; fa[atomicAdd(&s_a, 1)] = u; }
            else dL[u] = INF;
        }
        __syncthreads();
        int fsz = s_a, level = 0;
        int *cur = fa, *nxt = fb;
        for (int guard = 0; fsz > 0 && guard <= 2 * n + 2; guard++) {
            __syncthreads();
            if (t == 0) s_c = 0;
            __syncthreads();
            for (int i = t; i < fsz; i += T) {
                const int u = __ldcg(cur + i);
                for (int e = rp[u]; e < rp[u + 1]; e++) {
                    const int v = col[e];
                    if (atomicCAS(&dR[v], INF, level + 1) == INF) {
                        const int m = __ldcg(mateR + v);
                        if (m < 0) s_b = 1;
                        else { dL[m] = level + 2; nxt[atomicAdd(&s_c, 1)] = m; }
                    }
                }
            }
            __threadfence_block();
            __syncthreads();
            fsz = s_b ? 0 : s_c;      // stop at the first layer that reaches a free R vertex
            int *tmp = cur; cur = nxt; nxt = tmp;
            level += 2;
        }
        __syncthreads();
        const int found = s_b;
        __syncthreads();
        if (!found) break;
        // ---- vertex-disjoint shortest augmenting paths
        for (int v = t; v < n; v += T) { used[v] = 0; itp[v] = rp[v]; }
        __threadfence_block();
        __syncthreads();
        for (int u0 = t; u0 < n; u0 += T) {
            if (__ldcg(dL + u0) != 0) continue;
            int x = u0;
            parL[u0] = -1;
            for (int guard = 0; guard < 2 * Q.m2p + 2 * n + 8; guard++) {
                int e = __ldcg(itp + x), v = -1;
                const int end = rp[x + 1], dx = __ldcg(dL + x);
                for (; e < end; e++) {
                    const int cv = col[e];
                    if (__ldcg(dR + cv) == dx + 1 && atomicCAS(&used[cv], 0, 1) == 0) { v = cv; e++; break; }
                }
                itp[x] = e;
                if (v >= 0) {
                    const int m = __ldcg(mateR + v);
                    if (m < 0) {                        // augment back to u0
                        int cl = x, cr = v;
                        for (int g2 = 0; g2 <= n; g2++) {
                            const int nr = __ldcg(mateL + cl);
                            mateL[cl] = cr;
                            mateR[cr] = cl;
                            if (cl == u0) break;
                            cr = nr;
                            cl = __ldcg(parL + cl);
                        }
                        break;
                    }
                    parL[m] = x;
                    x = m;
                } else {
                    if (x == u0) break;
                    x = __ldcg(parL + x);
                }
            }
        }
        __threadfence_block();
        __syncthreads();
    }

    // ---- Koenig: Z = reachable from the free L vertices by alternating paths
    if (t == 0) { s_a = 0; }
    __syncthreads();
    for (int u = t; u < n; u += T) {
        dR[u] = 0;
        if (__ldcg(mateL + u) < 0) { dL[u] = 1; fa[atomicAdd(&s_a, 1)] = u; }
        else dL[u] = 0;
    }
    __threadfence_block();
    __syncthreads();
    {
        int fsz = s_a;
        int *cur = fa, *nxt = fb;
        for (int guard = 0; fsz > 0 && guard <= 2 * n + 2; guard++) {
            __syncthreads();
            if (t == 0) s_c = 0;
            __syncthreads();
            for (int i = t; i < fsz; i += T) {
                const int u = __ldcg(cur + i), mu = __ldcg(mateL + u);
                for (int e = rp[u]; e < rp[u + 1]; e++) {
                    const int v = col[e];
                    if (v == mu) continue;             // non-matching edges from L
                    if (atomicCAS(&dR[v], 0, 1) == 0) {
                        const int m = __ldcg(mateR + v);
                        if (m >= 0 && atomicCAS(&dL[m], 0, 1) == 0) nxt[atomicAdd(&s_c, 1)] = m;
                    }
                }
            }
            __threadfence_block();
            __syncthreads();
            fsz = s_c;
            int *tmp = cur; cur = nxt; nxt = tmp;
        }
    }
    __syncthreads();
    // C_B = (L \ Z) + (R & Z); check it is a cover of size |M|
    int csz = 0, msz = 0, bad = 0, v1 = 0, v0 = 0;
    for (int u = t; u < n; u += T) {
        const int inL = __ldcg(dL + u) ? 0 : 1, inR = __ldcg(dR + u) ? 1 : 0;
        csz += inL + inR;
        msz += __ldcg(mateL + u) >= 0;
        x2[u] = inL + inR;
        v1 += inL + inR == 2;
        v0 += inL + inR == 0;
        for (int e = rp[u]; e < rp[u + 1] && !bad; e++)
            if (!inL && !__ldcg(dR + col[e])) bad = 1;  // edge u_L - v_R uncovered
    }
    csz = block_sum(csz, red);
    msz = block_sum(msz, red);
    bad = block_sum(bad, red);
    v1 = block_sum(v1, red);
    v0 = block_sum(v0, red);
    __threadfence_block();
    __syncthreads();
    if (bad || csz != msz) {
        if (t == 0) Q.crown_status = -1;
        return;
    }
    if (v1 + v0 == 0) {
        if (t == 0) Q.crown_status = 0;
        return;
    }
    // ---- induce the x = 1/2 part (ids in increasing order), record x = 1
    int *nid = fa;
    int base = 0;
    for (int b = 0; b < n; b += T) {
        const int v = b + t;
        const int k = v < n && x2[v] == 1;
        int tot;
        const int off = block_excl_scan(k, red, &tot);
        if (v < n) nid[v] = k ? base + off : -1;
        base += tot;
    }
    const int n2 = base;
    __threadfence_block();
    __syncthreads();
    int ebase = 0, dmax = 0;
    for (int b = 0; b < n; b += T) {
        const int v = b + t;
        int d = 0;
        if (v < n && nid[v] >= 0)
            for (int e = rp[v]; e < rp[v + 1]; e++) d += nid[col[e]] >= 0;
        dmax = max(dmax, d);
        int tot;
        const int off = block_excl_scan(d, red, &tot);
        if (v < n && nid[v] >= 0) { rpn[nid[v]] = ebase + off; orn[nid[v]] = Q.orig[v]; }
        ebase += tot;
    }
    dmax = block_max(dmax, red);
    __threadfence_block();
    __syncthreads();
    for (int v = t; v < n; v += T) {
        if (x2[v] == 2) Q.st[Q.orig[v]] = 1;            // in the cover
        if (nid[v] < 0) continue;
        int o = rpn[nid[v]];
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            const int c2 = nid[col[e]];
            if (c2 >= 0) coln[o++] = c2;
        }
    }
    __threadfence();
    __syncthreads();
    if (t == 0) {
        rpn[n2] = ebase;
        Q.rp2 = rpn;
        Q.col2 = coln;
        Q.orig = orn;
        Q.np = n2;
        Q.m2p = ebase;
        Q.maxdeg = dmax;
        Q.forced += v1;
        Q.crown_status = 1;
        Q.crown_forced = v1;
        Q.crown_removed = v1 + v0;
    }
    __syncthreads();
    if (n2 == 0 || (Q.k >= 0 && Q.forced > Q.k)) {   // settled here
        for (int v = t; v < Q.n; v += T) Q.cover_flags[v] = Q.st[v] == 1;
        if (t == 0) {
            Q.answered = 1;
            if (Q.k < 0) { Q.result = Q.forced; Q.yes = 1; }
            else { Q.yes = Q.forced <= Q.k; Q.result = Q.yes ? Q.forced : -1; }
        }
    }
}

// ------------------------------------------------------------ served requests

// One block per staged request: the CSR checks of vc_load_csr (row pointers
// non-decreasing from 0 to 2|E|; each entry in range, not a self-loop,
// strictly ascending in its row and mirrored in the other row).  A failure
// sets the request's status to VC_EINVAL.
__global__ void __launch_bounds__(kRootThreads) serve_validate_kernel(QueryDesc *qs)
{
    QueryDesc &Q = qs[blockIdx.x];
    const int n = Q.n, m2 = Q.m2;
    const int *rp = Q.rp, *col = Q.col;
    int bad = 0;
    if (threadIdx.x == 0) bad = n < 0 || m2 < 0 || (n == 0 && m2 != 0) || (n > 0 && (rp[0] != 0 || rp[n] != m2));
    for (int v = threadIdx.x; v < n && !bad; v += blockDim.x)
        if (rp[v] > rp[v + 1]) bad = 1;
    bad = __syncthreads_or(bad);
    if (!bad) {
        for (int e = threadIdx.x; e < m2 && !bad; e += blockDim.x) {
            int lo = 0, hi = n - 1;                // the row of e: last v with rp[v] <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rp[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int v = lo, u = col[e];
            if (u < 0 || u >= n || u == v || (e > rp[v] && col[e - 1] >= u)) { bad = 1; break; }
            int a = rp[u], b = rp[u + 1] - 1;
            bool found = false;
            while (a <= b) {
                const int mid = (a + b) >> 1, x = col[mid];
                if (x == v) { found = true; break; }
                if (x < v) a = mid + 1; else b = mid - 1;
            }
            if (!found) bad = 1;
        }
        bad = __syncthreads_or(bad);
    }
    if (bad && threadIdx.x == 0) Q.status = VC_EINVAL;
}

// One block per active slot (and at least one block): finished requests are
// finalised and their covers appended to the mapped output buffer; block 0
// copies the control block's entries out as well.
__global__ void __launch_bounds__(kRootThreads) serve_retire_kernel(
    QueryDesc *slots, const int *active, int nactive, const RegEntry *reg, const uint32_t *reg_words, int wcap,
    RetireRec *rec, int *cover_out, long long cover_cap, unsigned long long *cover_ctr,
    const unsigned long long *ctl, unsigned long long *ctl_out, int lane)
{
    __shared__ int red[33];
    __shared__ long long s_off;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < kCtlEntries; i += blockDim.x) ctl_out[i] = ctl[i * kCtlStride];
    if ((int)blockIdx.x >= nactive) return;
    const int qi = active[blockIdx.x];
    QueryDesc &Q = slots[qi];
    if (Q.lane != lane) return;   // another size class retires it (uniform over the block)
    RetireRec &R = rec[blockIdx.x];
    if (!Q.done) {
        if (threadIdx.x == 0) { R.slot = qi; R.state = 0; R.lane = lane; }
        return;
    }
    const bool ok = Q.status == VC_OK;
    if (ok) finalize_query(Q, reg, reg_words, wcap, red);
    __syncthreads();
    const int len = ok ? Q.cover_len : 0;
    if (threadIdx.x == 0) s_off = len > 0 ? (long long)atomicAdd(cover_ctr, (unsigned long long)len) : 0;
    __syncthreads();
    const long long off = s_off;
    const bool fits = off + len <= cover_cap;
    if (fits)
        for (int i = threadIdx.x; i < len; i += blockDim.x) cover_out[off + i] = Q.cover_list[i];
    if (threadIdx.x == 0) {
        R.slot = qi;
        R.state = 1;
        R.status = Q.status;
        R.result = Q.result;
        R.yes = Q.yes;
        R.cover_len = len;
        R.cover_off = fits ? off : -1;
        R.nodes = Q.nodes;
        R.np = Q.np;
        R.lane = lane;
    }
}

}  // namespace vcg

// ------------------------------------------------------------ host wrappers

#include "vc_internal.h"

namespace vcg {

constexpr size_t kRootSmemMax = 200 * 1024;

cudaError_t validate_run(int n, int m2, const int *rp, const int *col, int *d_err, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_err, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = (n + 1 + threads - 1) / threads < 4096 ? (n + 1 + threads - 1) / threads : 4096;
    validate_rowptr_kernel<<<blocks > 0 ? blocks : 1, threads, 0, s>>>(n, m2, rp, d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int eblocks = std::max(1, std::min(4096, (m2 + threads - 1) / threads));
        validate_col_kernel<<<eblocks, threads, 0, s>>>(n, m2, rp, col, d_err);
        e = cudaGetLastError();   // (the row-pointer check also took the maximum degree)
    }
    return e;
}

size_t root_smem_bytes(int max_n) { return SmemStore::smem_bytes(max_n); }

// log2 of the vertices per CTA for the cluster kernel, or -1 when one block
// per query is used
int root_cluster_shift(int nq, int max_n, int max_deg)
{
    if (nq != 1 || max_n < kClusterMinN || max_deg > 65535) return -1;
    int cs = 10;
    while (((long long)kClusterMax << cs) < max_n) cs++;
    const int C = (int)((max_n + (1 << cs) - 1) >> cs);
    if (cluster_smem_bytes(1 << cs, C) > kRootSmemMax || (1 << cs) > 4 * 32 * kRootThreads) return -1;
    return cs;
}

// Host-side memo of the cluster launch set-up, per device: the function
// attributes are set once, and the cluster shape found to fit for a graph
// size is kept (each occupancy query costs host time on every solve).
struct ClusterMemo {
    std::mutex mu;
    std::set<int> attrs_set;
    std::map<int, int> smem;                     // device -> dynamic shared memory per CTA
    std::map<std::pair<int, int>, int> shift;   // (device, max_n) -> cluster shift, -1: none fits
};
static ClusterMemo &cluster_memo()
{
    static ClusterMemo m;
    return m;
}

cudaError_t root_run(QueryDesc *d_q, int nq, int max_n, int max_deg, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    int cs = root_cluster_shift(nq, max_n, max_deg);
    int dev = 0;
    bool memo_hit = false;
    size_t cluster_dyn = kRootSmemMax;
    if (cs >= 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        ClusterMemo &M = cluster_memo();
        std::lock_guard<std::mutex> lk(M.mu);
        if (!M.attrs_set.count(dev)) {
            e = cudaFuncSetAttribute(root_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
            // all the shared memory a block may have (one CTA per SM): the
            // rows, their source index and rank 0's residual graph use it
            int optin = 0;
            cudaFuncAttributes fa;
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (e != cudaSuccess) return e;
            e = cudaFuncGetAttributes(&fa, root_cluster_kernel);
            if (e != cudaSuccess) return e;
            const int dyn = std::max((int)kRootSmemMax, optin - (int)fa.sharedSizeBytes) & ~15;
            e = cudaFuncSetAttribute(root_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
            if (e != cudaSuccess) return e;
            M.smem[dev] = dyn;
            M.attrs_set.insert(dev);
        }
        cluster_dyn = M.smem[dev];
        auto it = M.shift.find({dev, max_n});
        if (it != M.shift.end()) {
            cs = it->second;
            memo_hit = true;
        }
    }
    if (cs >= 0 && !memo_hit) {
        int C = (int)((max_n + (1 << cs) - 1) >> cs);
        // a cluster wider than 8 is not guaranteed: shrink until one fits
        for (;;) {
            cudaLaunchConfig_t probe = {};
            probe.gridDim = dim3(C, 1, 1);
            probe.blockDim = dim3(kRootThreads, 1, 1);
            probe.dynamicSmemBytes = cluster_dyn;   // (the rows are staged in what is left)
            cudaLaunchAttribute pa[1];
            pa[0].id = cudaLaunchAttributeClusterDimension;
            pa[0].val.clusterDim.x = C;
            pa[0].val.clusterDim.y = 1;
            pa[0].val.clusterDim.z = 1;
            probe.attrs = pa;
            probe.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, root_cluster_kernel, &probe) == cudaSuccess && clusters > 0)
                break;
            cudaGetLastError();
            const int C2 = (int)((max_n + (2 << cs) - 1) >> (cs + 1));
            if (C <= 1 || cluster_smem_bytes(2 << cs, C2) > kRootSmemMax || (2 << cs) > 4 * 32 * kRootThreads) {
                cs = -1;
                break;
            }
            cs++;
            C = (int)((max_n + (1 << cs) - 1) >> cs);
        }
        ClusterMemo &M = cluster_memo();
        std::lock_guard<std::mutex> lk(M.mu);
        if (M.shift.size() >= 4096) M.shift.clear();   // many distinct sizes: start over
        M.shift[{dev, max_n}] = cs;
    }
    if (cs >= 0) {
        const int C = (int)((max_n + (1 << cs) - 1) >> cs);
        const size_t smem = cluster_dyn;   // one CTA per SM in any case: room for staged rows
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(kRootThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, root_cluster_kernel, d_q, cs, (int)smem);
    }
    const size_t smem = SmemStore::smem_bytes(max_n);
    if (max_deg <= 65535 && smem <= kRootSmemMax) {
        // the attribute is a ceiling shared by every launch of the kernel:
        // always set the maximum, never a smaller per-launch size
        cudaError_t e = cudaFuncSetAttribute(root_kernel<SmemStore>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kRootSmemMax);
        if (e != cudaSuccess) return e;
        root_kernel<SmemStore><<<nq, kRootThreads, smem, s>>>(d_q);
    } else {
        root_kernel<GlobalStore><<<nq, kRootThreads, 0, s>>>(d_q);
    }
    return cudaGetLastError();
}

cudaError_t finalize_run(QueryDesc *d_q, int nq, const RegEntry *reg, const uint32_t *reg_words, int wcap,
                         cudaStream_t s, int mode)
{
    if (nq <= 0) return cudaSuccess;
    finalize_kernel<<<nq, kRootThreads, 0, s>>>(d_q, reg, reg_words, wcap, mode);
    return cudaGetLastError();
}

cudaError_t crown_run(QueryDesc *d_q, int nq, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    crown_kernel<<<nq, kRootThreads, 0, s>>>(d_q);
    return cudaGetLastError();
}

cudaError_t serve_validate_run(QueryDesc *d_staging, int na, cudaStream_t s)
{
    if (na <= 0) return cudaSuccess;
    serve_validate_kernel<<<na, kRootThreads, 0, s>>>(d_staging);
    return cudaGetLastError();
}

cudaError_t serve_retire_run(QueryDesc *d_slots, const int *active, int nactive, const RegEntry *reg,
                             const uint32_t *reg_words, int wcap, RetireRec *rec, int *cover_out,
                             long long cover_cap, unsigned long long *cover_ctr,
                             const unsigned long long *ctl, unsigned long long *ctl_out, int lane, cudaStream_t s)
{
    serve_retire_kernel<<<nactive > 0 ? nactive : 1, kRootThreads, 0, s>>>(
        d_slots, active, nactive, reg, reg_words, wcap, rec, cover_out, cover_cap, cover_ctr, ctl, ctl_out, lane);
    return cudaGetLastError();
}

}  // namespace vcg

// ------------------------------------------------------------ no-allocation variant
//
// vc_root_reduce_static(): the root reduction + induced subgraph above, for
// callers that cannot allocate device memory.  Its scratch is one file-scope
// device array, shared by every call in the process and kept between calls.

#include <mutex>

namespace vcg {

constexpr int kStaticMaxN = 65536;
constexpr size_t kStaticBytes = (size_t)2 << 20;   // 2 MiB, resident on every device that loads the library
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char vc_static_scratch[kStaticBytes];

// Fixed layout inside the array, sized for kStaticMaxN vertices.
struct StaticLayout {
    static constexpr size_t kDesc = 0;                                    // QueryDesc
    static constexpr size_t kErr = 512;                                   // 4 ints
    static constexpr size_t kArr = 1024;                                  // int arrays
    static constexpr size_t kIntArr = (size_t)kStaticMaxN * 4;
    static constexpr size_t kDeg = kArr;
    static constexpr size_t kAux = kDeg + kIntArr;
    static constexpr size_t kFr0 = kAux + kIntArr;
    static constexpr size_t kFr1 = kFr0 + kIntArr;
    static constexpr size_t kFlag = kFr1 + kIntArr;
    static constexpr size_t kHeavy = kFlag + kIntArr;
    static constexpr size_t kSt = kHeavy + kIntArr;
    static constexpr size_t kCover = kSt + kStaticMaxN;
    static constexpr size_t kEnd = kCover + kStaticMaxN;
};
static_assert(StaticLayout::kEnd <= kStaticBytes, "static scratch too small");
static_assert(sizeof(QueryDesc) <= StaticLayout::kErr, "descriptor does not fit");

// One thread: clear the validation words (they must start at zero).
__global__ void static_clear_kernel(char *base)
{
    int *err = (int *)(base + StaticLayout::kErr);
    err[0] = 0; err[1] = 0; err[2] = 0; err[3] = 0;
}

// One thread: fill the descriptor from the arguments and the validation result.
__global__ void static_setup_kernel(char *base, int n, int m2, const int *rp, const int *col, int k,
                                    int *forced, int *irp, int *icol, int *iorig)
{
    QueryDesc *Q = (QueryDesc *)(base + StaticLayout::kDesc);
    const int *err = (const int *)(base + StaticLayout::kErr);
    QueryDesc q;
    memset(&q, 0, sizeof(q));
    q.n = n;
    q.m2 = m2;
    q.rp = rp;
    q.col = col;
    q.k = k;
    q.maxdeg_in = err[2];
    q.deg = (int *)(base + StaticLayout::kDeg);
    q.aux = (int *)(base + StaticLayout::kAux);
    q.fr0 = (int *)(base + StaticLayout::kFr0);
    q.fr1 = (int *)(base + StaticLayout::kFr1);
    q.flag = (int *)(base + StaticLayout::kFlag);
    q.heavy = (int *)(base + StaticLayout::kHeavy);
    q.forced_list = forced;
    q.st = (uint8_t *)(base + StaticLayout::kSt);
    q.cover_flags = (uint8_t *)(base + StaticLayout::kCover);
    q.rp2 = irp;
    q.col2 = icol;
    q.orig = iorig;
    q.status = (n > 0 && (err[0] != 0 || (long long)err[1] * 2 != m2)) ? VC_EINVAL : VC_OK;
    q.greedy = -1;
    *Q = q;
}

// One thread: copy the outcome to the caller's info array.
__global__ void static_export_kernel(const char *base, int *info)
{
    const QueryDesc *Q = (const QueryDesc *)(base + StaticLayout::kDesc);
    const bool ok = Q->status == VC_OK;
    info[0] = Q->status;
    info[1] = ok ? Q->forced : 0;
    info[2] = ok ? Q->np : 0;
    info[3] = ok ? Q->m2p : 0;
    info[4] = ok ? Q->greedy : -1;
    info[5] = ok ? Q->answered : 0;
    info[6] = ok && Q->answered ? Q->result : -1;
    info[7] = ok ? Q->maxdeg : 0;
}

// Per-device set-up: the device address of the scratch array (a host-side
// use of the array's name is only a stand-in, not a device address).
static std::mutex g_static_mu;
static char *g_static_ptr[kStaticMaxDevices];

static int static_setup(char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VC_ECUDA;
    if (dev < 0 || dev >= kStaticMaxDevices) return VC_ECAPACITY;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, vc_static_scratch) != cudaSuccess || !p) return VC_ECUDA;
        if (cudaFuncSetAttribute(root_kernel<SmemStore>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRootSmemMax) != cudaSuccess)
            return VC_ECUDA;
        g_static_ptr[dev] = (char *)p;
    }
    *out = g_static_ptr[dev];
    return VC_OK;
}

}  // namespace vcg

extern "C" int vc_root_reduce_static(int32_t n, int32_t m2, const int32_t *d_row_ptr, const int32_t *d_col,
                                     int32_t k, int32_t *d_forced, int32_t *d_induced_row_ptr,
                                     int32_t *d_induced_col, int32_t *d_induced_orig, int32_t *d_info,
                                     void *cuda_stream)
{
    using namespace vcg;
    if (n < 0 || m2 < 0 || (m2 & 1) || !d_info) return VC_EINVAL;
    if (n > kStaticMaxN) return VC_ECAPACITY;
    if (n > 0 && (!d_row_ptr || !d_forced || !d_induced_row_ptr || !d_induced_orig)) return VC_EINVAL;
    if (m2 > 0 && (!d_col || !d_induced_col)) return VC_EINVAL;
    char *base = nullptr;
    int rc = static_setup(&base);
    if (rc != VC_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int *err = (int *)(base + StaticLayout::kErr);
    static_clear_kernel<<<1, 1, 0, s>>>(base);
    if (cudaGetLastError() != cudaSuccess) return VC_ECUDA;
    if (n > 0) {
        const int threads = 256;
        const int blocks = std::min(4096, (n + 1 + threads - 1) / threads);
        validate_rowptr_kernel<<<blocks, threads, 0, s>>>(n, m2, d_row_ptr, err);
        const int eblocks = std::max(1, std::min(4096, (m2 + threads - 1) / threads));
        validate_col_kernel<<<eblocks, threads, 0, s>>>(n, m2, d_row_ptr, d_col, err);
        max_degree_kernel<<<blocks, threads, 0, s>>>(n, d_row_ptr, err);
        if (cudaGetLastError() != cudaSuccess) return VC_ECUDA;
    }
    static_setup_kernel<<<1, 1, 0, s>>>(base, n, m2, d_row_ptr, d_col, k < 0 ? -1 : k, d_forced,
                                        d_induced_row_ptr, d_induced_col, d_induced_orig);
    QueryDesc *dq = (QueryDesc *)(base + StaticLayout::kDesc);
    const size_t smem = SmemStore::smem_bytes(n);
    if (smem <= kRootSmemMax)
        root_kernel<SmemStore><<<1, kRootThreads, smem, s>>>(dq);
    else
        root_kernel<GlobalStore><<<1, kRootThreads, 0, s>>>(dq);
    static_export_kernel<<<1, 1, 0, s>>>(base, d_info);
    return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}
