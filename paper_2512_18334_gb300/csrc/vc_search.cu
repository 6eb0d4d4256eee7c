// Persistent component-aware branch-and-reduce search (Algorithm 2 of the
// paper, parallelised as in Sections 2.3 and 3).
//
// A worker is a team of threads (a warp, or a whole block for large induced
// graphs).  It pops a node (private stack first, then the shared worklist),
// stages its degree window and cover bitmap in shared memory, and then loops:
//   reduce  - degree-one, degree-two-triangle and high-degree rules in
//             synchronous rounds until a fixpoint (Section 2.2);
//   prune   - |S| >= B or |E| > (B - |S| - 1)^2 with B the Best of the
//             enclosing component (the stopping condition of Algorithms 1 and 2);
//   leaf    - |E| = 0: a new best cover of the component (Algorithm 1, 5-7);
//   split   - union-find over the live vertices finds the components
//             (Section 3.2); cliques and chordless cycles are closed at once
//             (Section 3.4); with >= 2 others the node branches on components
//             through the registry (Section 3.3);
//   branch  - on the lowest-index vertex of maximum degree: the right child
//             G - N(v) is stored (private stack or worklist), the left child
//             G - v continues in shared memory (the vertex branch of Algorithm 1).
// Completion decrements LiveNodes of the enclosing component entry; the last
// descendant adds the component's Best into its parent's Sum and, when the
// parent's LiveComps reaches zero, updates the ancestor's Best and continues
// upward (Section 3.3).
#include <climits>

#include "vc_common.cuh"

namespace vcg {

// ---------------------------------------------------------------- checks
//
// Built with -DVC_CHECKS, every shared-memory, slot, registry and stack index
// below is verified first; a bad one is skipped and recorded (status
// VC_ECAPACITY, site code 100 + n in the control block) instead of executed.
#ifdef VC_CHECKS
#define VC_GUARD(cond, site)                                            \
    if (!(cond)) {                                                      \
        set_error(P.ctl, VC_ECAPACITY, 100 + (site));                   \
        return;                                                         \
    }
#define VC_GUARD_R(cond, site, r)                                       \
    if (!(cond)) {                                                      \
        set_error(P.ctl, VC_ECAPACITY, 100 + (site));                   \
        return r;                                                       \
    }
#else
#define VC_GUARD(cond, site)
#define VC_GUARD_R(cond, site, r)
#endif

// ---------------------------------------------------------------- sizes

template <typename T>
struct Vec {
    static constexpr int kPer16 = 16 / sizeof(T);   // elements per 16-byte vector
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int align_down(int x, int a) { return x / a * a; }

// Best value broadcast to the team when the time slice is over.
constexpr int kPreempt = INT_MIN + 1;

template <typename T>
__host__ __device__ inline int deg_region_bytes(int ncap) { return align_up(ncap * (int)sizeof(T), 16); }

template <typename T>
__host__ __device__ inline int slot_bytes_for(int ncap, int wcap)
{
    return (int)sizeof(NodeHdr) + deg_region_bytes<T>(ncap) + align_up(wcap * 4, 16);
}

// A worker's node arrays: degrees, mark bytes, labels / mark list, cover
// bitmap.  They live in shared memory when they fit, else in a per-worker
// region of global memory (Section 4.1: the degree array is staged in shared
// memory if it fits); the scalars and the team's reduction scratch always
// live in shared memory.
// Capacity of a worker's list of vertices whose degree dropped to 1 or 2
// since the rules last examined them (more in one round: the next round
// examines the whole window instead).  Small arrays get one entry per
// vertex (never full); large ones a fixed 256, so that the list does not
// cost a block of occupancy (11.7k vertices: three blocks per SM fit with
// 1 KB, two with 4 KB).
__host__ __device__ inline int dirty_cap(int ncap) { return ncap <= 1024 ? ncap : 256; }

template <typename T>
__host__ __device__ inline int worker_array_bytes(int ncap, int wcap)
{
    return deg_region_bytes<T>(ncap) + align_up(ncap, 16) + ncap * 4 + align_up(wcap * 4, 16) +
           align_up(dirty_cap(ncap) * 4, 16);
}
// scalars: 16 general ints, the breakdown counters (7 x u64 at int 16), the
// leader's registry free list and time-slice end (ints 32..36); then the
// block team's reduction scratch
constexpr int kWorkerScalarInts = 64;
__host__ __device__ inline int worker_scalar_bytes(bool warp_team)
{
    return kWorkerScalarInts * 4 + (warp_team ? 0 : kRedInts * 4);
}

// shared-memory bytes of one worker (team)
template <typename T>
__host__ __device__ inline int worker_smem_bytes(int ncap, int wcap, bool arrays_global, bool warp_team)
{
    return (arrays_global ? 0 : worker_array_bytes<T>(ncap, wcap)) + worker_scalar_bytes(warp_team);
}

// ---------------------------------------------------------------- registry

// Load that bypasses L1: registry entries and node slots are written by other
// SMs and recycled, so a stale L1 line must never be read.
template <class X>
__device__ __forceinline__ X vld(const X &x) { return *(volatile const X *)&x; }

// Registry entries come from a per-worker free list first, then from a
// global stack of free chunks (entries linked through `next`, chunks linked
// through pad[0] of their first entry, which also holds the chunk's size in
// pad[1]), then from a global bump counter.  Freed entries go to the freeing
// worker's list; when it reaches 2 * kChunk, kChunk of them go back to the
// global stack as one chunk (one CAS per chunk, not per entry), and a worker
// returns whatever its list holds when it exits (so that time slices of a
// resident search lose nothing).  Only team leaders call these.
constexpr int kChunk = 32;

__device__ __forceinline__ unsigned long long cas_release_u64(unsigned long long *p, unsigned long long cmp,
                                                              unsigned long long val)
{
    unsigned long long old;
    asm volatile("atom.release.gpu.global.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "l"(p), "l"(cmp), "l"(val) : "memory");
    return old;
}

// Pop one chunk; returns its first entry or -1.
__device__ int reg_chunk_pop(const SearchParams &P)
{
    unsigned long long *head = &ctlw(P.ctl, kRegHead);
    for (int it = 0; it < 64; it++) {
        const unsigned long long h = ld_acquire_u64(head);
        const int idx = (int)(h & 0xffffffffull);
        if (idx < 0) return -1;
        const int nx = *(volatile int *)&P.reg[idx].pad[0];
        const unsigned long long nh = ((h >> 32) + 1) << 32 | (unsigned)nx;
        if (atomicCAS(head, h, nh) == h) return idx;
        __nanosleep(16 + (it << 4));
    }
    return -1;   // contended: the caller falls back to the bump counter
}

// Push a chunk of cnt entries whose first entry is idx (already linked,
// the last one's `next` is -1).
__device__ void reg_chunk_push(const SearchParams &P, int idx, int cnt)
{
    unsigned long long *head = &ctlw(P.ctl, kRegHead);
    *(volatile int *)&P.reg[idx].pad[1] = cnt;
    for (int it = 0; it < (1 << 22); it++) {
        const unsigned long long h = ld_acquire_u64(head);
        *(volatile int *)&P.reg[idx].pad[0] = (int)(h & 0xffffffffull);
        const unsigned long long nh = ((h >> 32) + 1) << 32 | (unsigned)idx;
        if (cas_release_u64(head, h, nh) == h) return;
        __nanosleep(16 + ((it & 63) << 4));
    }
    set_error(P.ctl, VC_ETIMEOUT, 1);
}

__device__ bool reg_lock(const SearchParams &P, int e)
{
    int *l = &P.reg[e].lock;
    for (int it = 0; it < (1 << 24); it++) {
        if (atomicCAS(l, 0, 1) == 0) {
            __threadfence();
            return true;
        }
        if (aborted(P.ctl)) return false;
        __nanosleep(64);
    }
    set_error(P.ctl, VC_ETIMEOUT, 2);
    return false;
}

__device__ void reg_unlock(const SearchParams &P, int e)
{
    __threadfence();
    atomicExch(&P.reg[e].lock, 0);
}

__device__ inline uint32_t *reg_words(const SearchParams &P, int e)
{
    return P.reg_words + (size_t)e * P.wcap;
}

// The query finished (its induced graph's entry completed, or PVC found a
// cover <= k).  Counted once.
__device__ void query_done(const SearchParams &P, int q)
{
    if (atomicExch(&P.queries[q].done, 1) == 0) atomicAdd(&ctlw(P.ctl, kRemaining), (unsigned long long)-1ll);
}

__device__ inline bool query_is_done(const SearchParams &P, int q)
{
    return *(volatile int *)&P.queries[q].done != 0;
}

// ---------------------------------------------------------------- worker

// GA: the node arrays are in global memory (SearchParams::wglobal).  A
// compile-time choice, so that in the shared-memory form every array access
// is a shared-memory access rather than a generic one.
template <typename T, int WT, bool GA = false>
struct Worker {
    const SearchParams &P;
    Team<WT> tm;
    int wid;

    // shared-memory arrays of this worker
    T *d;             // degrees of vertices [wlo, wlo + ncap)
    uint8_t *mark;    // per vertex: bit 0 marked for the cover, bit 1 on the dirty list
    int *lab;         // union-find labels / mark list
    uint32_t *cov;    // cover bitmap of the context window
    int *dl;          // dirty list (dirty_cap(ncap) entries)
    int *sc;          // scalars (16 ints)
    // breakdown: cycles per activity [kPhases], last mark [kPhases] (scalars 16..29)
    __device__ __forceinline__ unsigned long long *ph() const { return (unsigned long long *)(sc + 16); }

    const int *csr_s;   // staged CSR in shared memory (single-query launches) or null

    // node state (uniform across the team)
    int q, np;
    const int *rp, *col;
    int S, comp, lo, hi, clo, chi, wlo, whi, depth;
    int gen;          // generation of the node's query slot
    int dpar, danc, dlb;   // dynamic component bound of the context (dpar < 0: none)
    int cntbuf;       // double-buffer index of the mark counter
    int dc;           // double-buffer index of the dirty-list counter (scalars 2, 3)
    bool full;        // the next rule round examines every vertex of the window
    bool stop;        // the search was aborted (seen by process())
    int qk;           // the node's query: k (< 0: minimum cover)

    // leader only: loads issued ahead for the next node (prefetch())
    bool pf_ok, pf_dyn;
    unsigned pf_ab;
    unsigned long long pf_pk;
    int pf_bv, pf_av;

    // private stack depth
    int top;

    // the leader's private registry free list and time-slice end live in
    // shared memory (scalars 32..36), as does the deepest stack seen
    __device__ __forceinline__ int &lf_head() const { return sc[32]; }
    __device__ __forceinline__ int &lf_count() const { return sc[33]; }
    __device__ __forceinline__ unsigned long long &t_end() const { return *(unsigned long long *)(sc + 34); }
    __device__ __forceinline__ int &max_top() const { return sc[36]; }
    int nflush;              // nodes since the counters were last flushed
    int qnodes;              // nodes of query qcur not yet added to its counter
    int qcur;
    long long bytes_local;   // this thread's share of the algorithmic bytes
    bool preempted;          // the slice ended: the node was stored, stop

    __device__ Worker(const SearchParams &p, Team<WT> t, int w, char *smem, const int *csr)
        : P(p), tm(t), wid(w), csr_s(csr)
    {
        const int ncap = P.ncap, wcap = P.wcap;
        char *a = GA ? P.wglobal + (size_t)wid * (size_t)P.wglobal_stride : smem;
        d = (T *)a;                a += deg_region_bytes<T>(ncap);
        mark = (uint8_t *)a;       a += align_up(ncap, 16);
        lab = (int *)a;            a += ncap * 4;
        cov = (uint32_t *)a;       a += align_up(wcap * 4, 16);
        dl = (int *)a;             a += align_up(dirty_cap(ncap) * 4, 16);
        char *s = GA ? smem : a;
        sc = (int *)s;             s += kWorkerScalarInts * 4;
        if constexpr (WT == 0) {
            tm.red = (int *)s;
            tm.rb = 0;
        }
        top = P.stack_top ? P.stack_top[wid] : 0;
        gen = 0;
        dpar = -1;
        danc = -1;
        dlb = 0;
        preempted = false;
        stop = false;
        qk = -1;
        pf_ok = false;
        pf_dyn = false;
        pf_ab = 0;
        pf_pk = 0;
        pf_bv = pf_av = 0;
        nflush = 0;
        bytes_local = 0;
        qnodes = 0;
        qcur = -1;

        cntbuf = 0;
        dc = 0;
        full = true;
        if (tm.leader()) {
            sc[0] = 0;
            sc[1] = 0;
            sc[2] = 0;
            sc[3] = 0;
            lf_head() = -1;
            lf_count() = 0;
            t_end() = 0;
            max_top() = 0;
        }
        tm.sync();
    }

    // ------------------------------------------------------------ accessors

    __device__ __forceinline__ int dg(int u) const
    {
        return (u >= wlo && u <= whi) ? (int)d[u - wlo] : 0;
    }

    __device__ __forceinline__ bool marked(int u) const
    {
        return u >= wlo && u <= whi && (mark[u - wlo] & 1) != 0;
    }

    // Decrement u's degree; returns the new degree.
    __device__ __forceinline__ int dec(int u)
    {
        VC_GUARD_R(u >= wlo && u <= whi && u - wlo < P.ncap, 1, 0)
        const int off = u - wlo;
        if constexpr (sizeof(T) == 1) {
            unsigned *w = (unsigned *)((char *)d + (off & ~3));
            const int sh = 8 * (off & 3);
            return (int)((atomicSub(w, 1u << sh) >> sh) & 0xffu) - 1;
        } else if constexpr (sizeof(T) == 2) {
            unsigned *w = (unsigned *)((char *)d + 2 * (off & ~1));
            const int sh = 16 * (off & 1);
            return (int)((atomicSub(w, 1u << sh) >> sh) & 0xffffu) - 1;
        } else {
            return (int)atomicSub((unsigned *)&d[off], 1u) - 1;
        }
    }

    // Degree-one and degree-two-triangle candidates.  After a round of the
    // rules reaches its fixpoint, only a vertex whose degree has dropped to
    // 1 or 2 since can start to satisfy either rule (edges are never added,
    // so a degree-two vertex with unchanged degree keeps its neighbours), so
    // each decrement that leaves 1 or 2 puts the vertex on the dirty list
    // (once: bit 1 of its mark byte), and a round examines only the list.
    // A list that overflows makes the next round examine the whole window.
    // Missing a candidate would cost nodes, never correctness: the rules
    // only shrink the graph; the high-degree rule, on which the stopping
    // condition's soundness rests, is checked for every vertex every round.
    __device__ __forceinline__ void dec_dirty(int u)
    {
        const int nd = dec(u);
        if (nd == 1 || nd == 2) {
            const int off = u - wlo;
            const unsigned bit = 2u << (8 * (off & 3));
            if (!(atomicOr((unsigned *)(mark + (off & ~3)), bit) & bit)) {
                const int pos = atomicAdd(&sc[2 + dc], 1);
                if (pos < dirty_cap(P.ncap)) dl[pos] = u;
            }
        }
    }

    // d[u] = 0 for a vertex that goes into the cover.  Sub-word entries are
    // cleared with an atomic on their 32-bit word: other threads decrement
    // the neighbouring entries of the same word with atomics meanwhile.
    __device__ __forceinline__ void zero_deg(int u)
    {
        VC_GUARD(u >= wlo && u <= whi && u - wlo < P.ncap, 6)
        const int off = u - wlo;
        if constexpr (sizeof(T) == 1) {
            atomicAnd((unsigned *)((char *)d + (off & ~3)), ~(0xffu << (8 * (off & 3))));
        } else if constexpr (sizeof(T) == 2) {
            atomicAnd((unsigned *)((char *)d + 2 * (off & ~1)), ~(0xffffu << (16 * (off & 1))));
        } else {
            d[off] = 0;   // a vertex going into the cover is never decremented
        }
    }

    // queue u for the cover in this round (deduplicated); list in lab[].
    // Mark bytes are cleared only when a node is loaded from a slot: every
    // marked vertex goes into the cover (degree 0) and stays there for the
    // rest of the node and its left descendants, so a stale mark is only
    // ever seen on a vertex whose degree is already 0.
    __device__ __forceinline__ void mark_vertex(int u)
    {
        VC_GUARD(u >= wlo && u <= whi && u - wlo < P.ncap, 2)
        const int off = u - wlo;
        unsigned *w = (unsigned *)(mark + (off & ~3));
        unsigned bit = 1u << (8 * (off & 3));
        if (!(atomicOr(w, bit) & bit)) {
            int pos = atomicAdd(&sc[cntbuf], 1);
            VC_GUARD(pos >= 0 && pos < P.ncap, 3)
            lab[pos] = u;
        }
    }

    __device__ __forceinline__ void cov_set(int v)
    {
        VC_GUARD(v >= clo && v <= chi && (v >> 5) - (clo >> 5) < P.wcap, 4)
        atomicOr(&cov[(v >> 5) - (clo >> 5)], 1u << (v & 31));
    }

    __device__ __forceinline__ bool adjacent(int a, int b) const
    {
        const int *row = col + rp[a];
        int l = 0, h = rp[a + 1] - rp[a] - 1;
        while (l <= h) {
            int mid = (l + h) >> 1;
            int x = row[mid];
            if (x == b) return true;
            if (x < b) l = mid + 1; else h = mid - 1;
        }
        return false;
    }

    // ------------------------------------------------------------ marks

    // Rows are walked by groups of kGroup lanes: item i of a list goes to
    // group i mod (team / kGroup), whose lanes take every kGroup-th entry of
    // its row.  Rows here are a handful of entries long, so one vertex's row
    // costs about one dependent step instead of one per entry.
    static constexpr int kGroup = 8;
    __device__ __forceinline__ int ngroups() const { return tm.size() / kGroup; }
    __device__ __forceinline__ int group() const { return tm.rank / kGroup; }
    __device__ __forceinline__ int glane() const { return tm.rank % kGroup; }

    // Put the live vertex u in the cover: decrement its live unmarked
    // neighbours (the group's lanes share the row) and clear its entry.
    __device__ __forceinline__ void remove_marked(int u)
    {
        for (int e = rp[u] + glane(); e < rp[u + 1]; e += kGroup) {
            const int x = col[e];
            if (dg(x) > 0 && !marked(x)) dec_dirty(x);
        }
        if (glane() == 0) {
            cov_set(u);
            zero_deg(u);
            bytes_local += 8 + 4ll * (rp[u + 1] - rp[u]);
        }
    }

    // Put every marked vertex (list lab[0..c)) in the cover: G - M, S + M.
    // A marked vertex's own entry is cleared by its group; neighbours that
    // are marked too are skipped, so each edge between M and the rest is
    // counted once.  One team barrier.
    __device__ void apply_marks(int c)
    {
        for (int i = group(); i < c; i += ngroups()) remove_marked(lab[i]);
        S += c;
        tm.sync();
    }

    // Put the single vertex v in the cover (the left child G - v of a vertex
    // branch).  One team barrier.
    __device__ void remove_vertex(int v)
    {
        for (int e = rp[v] + tm.rank; e < rp[v + 1]; e += tm.size()) {
            const int x = col[e];
            if (dg(x) > 0) dec_dirty(x);
        }
        if (tm.leader()) {
            cov_set(v);
            zero_deg(v);
            bytes_local += 8 + 4ll * (rp[v + 1] - rp[v]);
        }
        S += 1;
        tm.sync();
    }

    // Put every live neighbour of v in the cover (the right child G - N(v)).
    // The team's threads take the row in the same stripes in both passes:
    // the first marks the live neighbours and counts them, the second applies
    // them.  Two team barriers.
    __device__ void remove_neighbourhood(int v)
    {
        int cnt = 0;
        for (int e = rp[v] + tm.rank; e < rp[v + 1]; e += tm.size()) {
            const int x = col[e];
            if (dg(x) > 0) {
                VC_GUARD(x >= wlo && x <= whi && x - wlo < P.ncap, 2)
                mark[x - wlo] = 1;
                cnt++;
            }
        }
        const int c = tm.sum(cnt);
        for (int e = rp[v] + group(); e < rp[v + 1]; e += ngroups()) {
            const int x = col[e];
            // marked in the first pass exactly when it was live; only its
            // own group clears its entry, so the mark alone decides (a
            // degree test could race with the group's own lane 0)
            if (marked(x)) remove_marked(x);
        }
        if (tm.leader()) bytes_local += 8 + 4ll * (rp[v + 1] - rp[v]);
        S += c;
        tm.sync();
    }

    // Breakdown of the execution time (the paper's SM-clock instrumentation):
    // the cycles since the last mark go to activity k.
    __device__ __forceinline__ void lap(int k)
    {
        if (P.breakdown && tm.leader()) {
            const unsigned long long now = clock64();
            ph()[k] += now - ph()[kPhases];
            ph()[kPhases] = now;
        }
    }

    // ------------------------------------------------------------ reduce

    struct Stats {
        long long e2;    // sum of live degrees
        int live;        // live vertices
        int dmax;        // maximum degree
        int vmax;        // lowest-index vertex of maximum degree
        int lo, hi;      // live window
        int pruned;      // budget exhausted during reduction
    };

    // The degree-one and degree-two-triangle rules at a live vertex v of
    // degree dv (1 or 2), against the current snapshot; ties are broken
    // towards the lower vertex so that two rules never put both ends of an
    // edge (or all of a triangle) in the cover.
    __device__ __forceinline__ void low_degree_rules(int v, int dv)
    {
        if (dv == 1) {
            int u = -1;
            int e = rp[v];
            for (; e < rp[v + 1]; e++) {
                int x = col[e];
                if (dg(x) > 0) { u = x; break; }
            }
            bytes_local += 8 + 4ll * (e - rp[v] + 1);
            if (u >= 0 && !(dg(u) == 1 && u < v)) mark_vertex(u);
        } else {
            int u = -1, w = -1;
            int e = rp[v];
            for (; e < rp[v + 1]; e++) {
                int x = col[e];
                if (dg(x) > 0) {
                    if (u < 0) u = x; else { w = x; break; }
                }
            }
            if (w < 0) return;   // (only while the snapshot is inconsistent; never at a round's start)
            bytes_local += 16 + 4ll * (e - rp[v] + 1) + 4ll * (32 - __clz(max(1, rp[u + 1] - rp[u])));
            if (adjacent(u, w) && !((dg(u) == 2 && u < v) || (dg(w) == 2 && w < v))) {
                mark_vertex(u);
                mark_vertex(w);
            }
        }
    }

    // low_degree_rules for the dirty vertex v (-1: none) by a group of
    // kGroup lanes: they read its row in parallel and a ballot finds the
    // first one or two live neighbours.  Called by every lane of the warp
    // (the loop below is uniform over the warp: the ballots need it).
    __device__ void low_degree_group(int v)
    {
        int dv = 0, r0 = 0, r1 = 0;
        if (v >= 0) {
            const int off = v - wlo;
            if (glane() == 0) atomicAnd((unsigned *)(mark + (off & ~3)), ~(2u << (8 * (off & 3))));
            dv = (int)d[off];
            if (dv == 1 || dv == 2) { r0 = rp[v]; r1 = rp[v + 1]; }
            else dv = 0;
        }
        const int lane = tm.rank & 31, gbase = lane & ~(kGroup - 1);
        const int nch = dv ? (r1 - r0 + kGroup - 1) / kGroup : 0;
        const int wmax = __reduce_max_sync(kFull, nch);
        int u = -1, w = -1, found = 0, scanned = 0;
        for (int ch = 0; ch < wmax; ch++) {
            const int e = r0 + ch * kGroup + glane();
            int x = -1;
            bool live = false;
            if (found < dv && e < r1) {
                x = col[e];
                live = dg(x) > 0;
            }
            const unsigned b = (__ballot_sync(kFull, live) >> gbase) & ((1u << kGroup) - 1);
            // the first two live entries of this chunk, as lanes of the group
            const int f1 = b ? __ffs(b) - 1 : 0;
            const unsigned b2 = b & (b - 1);
            const int f2 = b2 ? __ffs(b2) - 1 : 0;
            const int x1 = __shfl_sync(kFull, x, gbase + f1);
            const int x2 = __shfl_sync(kFull, x, gbase + f2);
            if (found < dv) {
                scanned = min(r1 - r0, (ch + 1) * kGroup);
                if (b) {
                    if (found == 0) { u = x1; found = 1; if (b2 && dv == 2) { w = x2; found = 2; } }
                    else if (found == 1) { w = x1; found = 2; }
                }
            }
        }
        if (dv == 0 || glane() != 0) return;
        bytes_local += 8 + 4ll * scanned;
        if (dv == 1) {
            if (u >= 0 && !(dg(u) == 1 && u < v)) mark_vertex(u);
        } else if (w >= 0) {
            bytes_local += 8 + 4ll * (32 - __clz(max(1, rp[u + 1] - rp[u])));
            if (adjacent(u, w) && !((dg(u) == 2 && u < v) || (dg(w) == 2 && w < v))) {
                mark_vertex(u);
                mark_vertex(w);
            }
        }
    }

    // Rules of Section 2.2 in synchronous rounds until no vertex is marked.
    // Each round is one pass over the window (statistics, high-degree rule,
    // and, in a full round, the low-degree rules at every vertex), a pass
    // over the dirty list (low-degree rules at the vertices whose degree
    // dropped to 1 or 2 since the last round) and one team reduction; a
    // round that marked vertices applies them (one more barrier) and is
    // followed by another.
    __device__ Stats reduce(int B)
    {
        Stats st;
#ifdef VC_CHECKS
        if (!(lo >= wlo && hi <= whi && whi - wlo < P.ncap && chi - clo >= 0 && (chi >> 5) - (clo >> 5) < P.wcap)) {
            if (tm.leader()) set_error(P.ctl, VC_ECAPACITY, 106);
            st.pruned = 1;
            return st;
        }
#endif
        for (;;) {
            const int bud = B - S - 1;
            if (bud < 0) { st.pruned = 1; return st; }
            // The dirty list filled since the last round (its counter is
            // final: a barrier separates every push from this point); the
            // other counter takes the pushes of this round's application.
            const int nd = sc[2 + dc];
            const bool all = full || nd > dirty_cap(P.ncap);
            full = false;
            if (tm.leader()) sc[2 + (dc ^ 1)] = 0;
            dc ^= 1;
            WinStats t;
            t.e2 = 0; t.live = 0; t.dmax = 0; t.vmax = INT32_MAX; t.lo = INT32_MAX; t.hi = -1;
            for (int v = lo + tm.rank; v <= hi; v += tm.size()) {
                const int dv = (int)d[v - wlo];
                if (dv == 0) continue;
                t.live++;
                t.e2 += dv;
                if (dv > t.dmax) { t.dmax = dv; t.vmax = v; }   // ascending v: the lowest wins ties
                t.lo = min(t.lo, v);
                t.hi = v;
                if (all && dv <= 2) low_degree_rules(v, dv);
                if (dv > bud) mark_vertex(v);
            }
            if (!all) {
                for (int base = 0; base < nd; base += ngroups()) low_degree_group(base + group() < nd ? dl[base + group()] : -1);
            } else if (nd > 0) {
                // a full round: every dirty flag goes (the list is dropped)
                for (int v = lo + tm.rank; v <= hi; v += tm.size()) {
                    const int off = v - wlo;
                    if (mark[off] & 2) atomicAnd((unsigned *)(mark + (off & ~3)), ~(2u << (8 * (off & 3))));
                }
            }
            // The reduction is also the barrier after which this round's mark
            // count is final.  The other counter was last read before the
            // previous barrier, so the leader may clear it for the next round.
            const WinStats w = tm.stats(t);
            const int c = sc[cntbuf];
            if (tm.leader()) sc[cntbuf ^ 1] = 0;
            cntbuf ^= 1;
            if (c == 0) {
                st.e2 = w.e2;
                st.live = w.live;
                st.dmax = w.dmax;
                st.vmax = w.live > 0 ? w.vmax : -1;
                st.lo = w.lo;
                st.hi = w.hi;
                st.pruned = 0;
                return st;
            }
            apply_marks(c);
        }
    }

    // ------------------------------------------------------------ slots

    __device__ char *stack_slot(int i) const
    {
#ifdef VC_CHECKS
        if (i < 0 || i >= P.stack_depth) { set_error(P.ctl, VC_ECAPACITY, 107); i = 0; }
#endif
        return P.stack_slots + ((size_t)wid * P.stack_depth + i) * P.slot_bytes;
    }

    // Write the current node (or a component child) into a slot.
    //   kind 0: the current array with a pending op (right child G - N(op))
    //   kind 1: component child: only vertices whose label is `root` (rel.)
    __device__ void write_slot(char *slot, int kind, int op, int root, int clo_c, int chi_c, int comp_c,
                               int S_c, int hi_c, int dpar_c, int danc_c, int dlb_c)
    {
        constexpr int V = Vec<T>::kPer16;
        // the stored degree window: the node's live window, or (bounds off)
        // the whole array
        const int slo = P.no_bounds ? wlo : align_down(kind == 0 ? lo : clo_c, V);
        const int shi = P.no_bounds ? whi : (kind == 0 ? hi : hi_c);
        const int nvec = (align_up(shi + 1, V) - slo) / V;
        NodeHdr *h = (NodeHdr *)slot;
        if (tm.leader()) {
            h->S = S_c;
            h->comp = comp_c;
            h->lo = slo;
            h->hi = shi;
            h->clo = clo_c;
            h->chi = chi_c;
            h->op = op;
            h->q = q;
            h->cov_empty = kind == 1;
            h->depth = depth + 1;
            h->gen = gen;
            h->dpar = kind == 0 ? dpar : dpar_c;
            h->danc = kind == 0 ? danc : danc_c;
            h->dlb = kind == 0 ? dlb : dlb_c;
            // a vertex branch's right child and a component child are stored
            // from an array the rules brought to their fixpoint; a preempted
            // node is stored after a vertex removal, before the next rules
            h->fix = (kind == 1 || op >= 0) ? 1 : 0;
            h->pad = 0;
        }
        uint4 *dst = (uint4 *)(slot + sizeof(NodeHdr));
        if (tm.leader())
            bytes_local += (long long)sizeof(NodeHdr) + 16ll * nvec +
                           (kind == 0 ? 4ll * ((chi >> 5) - (clo >> 5) + 1) : 0);
        if (kind == 0) {
            const uint4 *src = (const uint4 *)(d + (slo - wlo));
            for (int i = tm.rank; i < nvec; i += tm.size()) dst[i] = src[i];
            const int w0 = clo >> 5, nw = (chi >> 5) - w0 + 1;
            uint32_t *cdst = (uint32_t *)(slot + sizeof(NodeHdr) + deg_region_bytes<T>(P.ncap));
            for (int i = tm.rank; i < nw; i += tm.size()) cdst[i] = cov[i];
        } else {
            for (int i = tm.rank; i < nvec; i += tm.size()) {
                union { uint4 v; T e[V]; } u;
                const int base = slo + i * V;
                #pragma unroll
                for (int j = 0; j < V; j++) {
                    const int v = base + j;
                    int val = 0;
                    if (v >= lo && v <= hi && lab[v - lo] == root) val = (int)d[v - wlo];
                    u.e[j] = (T)val;
                }
                dst[i] = u.v;
            }
        }
    }

    // Load a node from a slot into shared memory.  Returns false, having
    // read only the header, when the node's request is finished (PVC answer,
    // node budget) or the node is left over from an earlier request of a
    // recycled query slot: such a node must not be expanded, since its
    // pending operation refers to a graph the slot may no longer hold.
    __device__ bool read_slot(const char *slot)
    {
        constexpr int V = Vec<T>::kPer16;
        // Every thread reads the whole header: four 16-byte loads in flight
        // at once (L2 only: the slot may have been written by another SM).
        const int4 *h4 = (const int4 *)slot;
        const int4 h0 = __ldcg(h4), h1 = __ldcg(h4 + 1), h2 = __ldcg(h4 + 2), h3 = __ldcg(h4 + 3);
        S = h0.x; comp = h0.y; wlo = h0.z; whi = h0.w;      // NodeHdr field order
        clo = h1.x; chi = h1.y;
        const int op = h1.z;
        q = h1.w;
        const int cov_empty = h2.x;
        depth = h2.y; gen = h2.z; dpar = h2.w;
        danc = h3.x; dlb = h3.y;
        const int fix = h3.z;
        lo = wlo; hi = whi;
#ifdef VC_CHECKS
        if (!(wlo >= 0 && whi >= wlo && align_up(whi + 1, V) - wlo <= P.ncap && clo <= chi &&
              (chi >> 5) - (clo >> 5) < P.wcap && comp >= 0 && comp < P.reg_cap && q >= 0 && q < P.nq &&
              (dpar < 0 || (dpar < P.reg_cap && danc >= 0 && danc < P.reg_cap)))) {
            if (tm.leader()) set_error(P.ctl, VC_ECAPACITY, 108);
            whi = wlo = lo = hi = 0; clo = chi = 0; comp = 0; q = 0; dpar = -1;
        }
#endif
        // The leader checks whether the node's request is still live while
        // the team copies the payload: a stale node's copy is simply dropped
        // (its window and bitmap were sized for this search's capacities,
        // so the copy stays inside the worker's arrays either way).
        int stale = 0;
        const QueryDesc &Q = P.queries[q];
        if (tm.leader()) {
            stale = vld(Q.done) != 0 || vld(Q.gen) != gen;
            prefetch();
            sc[2] = 0;   // empty dirty list (the mark bytes are cleared below)
            sc[3] = 0;
        }
        full = fix == 0;
        const int qnp = Q.np;
        qk = Q.k;
        const int *qrp = Q.rp2, *qcol = Q.col2;
        const int nvec = (align_up(whi + 1, V) - wlo) / V;
        const uint4 *src = (const uint4 *)(slot + sizeof(NodeHdr));
        uint4 *dst = (uint4 *)d;
        for (int i = tm.rank; i < nvec; i += tm.size()) dst[i] = __ldcg(src + i);
        uint4 z = make_uint4(0, 0, 0, 0);
        uint4 *mk = (uint4 *)mark;
        const int mvec = align_up(nvec * V, 16) / 16;
        for (int i = tm.rank; i < mvec; i += tm.size()) mk[i] = z;
        const int w0 = clo >> 5, nw = (chi >> 5) - w0 + 1;
        const uint32_t *csrc = (const uint32_t *)(slot + sizeof(NodeHdr) + deg_region_bytes<T>(P.ncap));
        for (int i = tm.rank; i < nw; i += tm.size()) cov[i] = cov_empty ? 0u : __ldcg(csrc + i);
        // (the broadcast is also the barrier after the copies)
        if (tm.bcast(stale)) return false;
        if (tm.leader()) bytes_local += (long long)sizeof(NodeHdr) + 16ll * nvec + (cov_empty ? 0 : 4ll * nw);
        if (csr_s && q == P.csr_query) {
            rp = csr_s;
            col = csr_s + qnp + 1;
        } else {
            rp = qrp;
            col = qcol;
        }
        np = qnp;
        // right child of a vertex branch: G - N(op), S + N(op)
        if (op >= 0) remove_neighbourhood(op);
        return true;
    }

    // ------------------------------------------------------------ worklist

    // Reserve a worklist slot; returns the ticket or -1 when full.
    __device__ long long wl_reserve()
    {
        int ok = 0;
        long long t = -1;
        if (tm.leader()) {
            unsigned long long *cnt = &ctlw(P.ctl, kWlCount);
            if ((long long)*(volatile unsigned long long *)cnt < P.wl_cap) {
                const long long old = (long long)atomicAdd(cnt, 1ull);
                if (old < P.wl_cap) ok = 1;
                else atomicAdd(cnt, (unsigned long long)-1ll);
            }
            if (ok) {
                t = (long long)atomicAdd(&ctlw(P.ctl, kWlTail), 1ull);
                const unsigned slot = (unsigned)t & (P.wl_cap - 1);
                int it = 0;
                while (ld_acquire_u32(&P.wl_seq[slot]) != (unsigned)t) {
                    if (++it > (1 << 24) || aborted(P.ctl)) { set_error(P.ctl, VC_ETIMEOUT, 3); ok = 0; break; }
                    __nanosleep(32);
                }
                if (it) atomicAdd(&ctlw(P.ctl, kWaitIters), (unsigned long long)it);
            }
            sc[4] = ok;
            sc[5] = (int)(t & 0x7fffffff);
            sc[6] = (int)(t >> 31);
        }
        tm.sync();
        ok = sc[4];
        long long tt = ((long long)sc[6] << 31) | (unsigned)sc[5];
        tm.sync();
        return ok ? tt : -1;
    }

    __device__ void wl_publish(long long t)
    {
        __threadfence();
        tm.sync();
        if (tm.leader()) {
            const unsigned slot = (unsigned)t & (P.wl_cap - 1);
            st_release_u32(&P.wl_seq[slot], (unsigned)t + 1u);
            atomicAdd(&ctlw(P.ctl, kOffloaded), 1ull);
        }
    }

    __device__ char *wl_slot(long long t) const
    {
        return P.wl_slots + (size_t)((unsigned)t & (P.wl_cap - 1)) * P.slot_bytes;
    }

    // Try to take a node from the worklist into shared memory: 0 nothing
    // there, 1 node loaded, 2 a finished request's node taken and dropped.
    // The item counter is only decremented while it is positive (read, then
    // CAS), so idle workers polling an empty worklist never write to it.
    __device__ int wl_pop()
    {
        int ok = 0;
        if (tm.leader()) {
            unsigned long long *cnt = &ctlw(P.ctl, kWlCount);
            for (int it = 0; it < 32; it++) {
                const unsigned long long c = *(volatile unsigned long long *)cnt;
                if ((long long)c <= 0) break;
                if (atomicCAS(cnt, c, c - 1) == c) { ok = 1; break; }
            }
            if (ok) {
                const long long t = (long long)atomicAdd(&ctlw(P.ctl, kWlHead), 1ull);
                const unsigned slot = (unsigned)t & (P.wl_cap - 1);
                int it = 0;
                while (ld_acquire_u32(&P.wl_seq[slot]) != (unsigned)t + 1u) {
                    if (++it > (1 << 24) || aborted(P.ctl)) { set_error(P.ctl, VC_ETIMEOUT, 4); ok = 0; break; }
                    __nanosleep(32);
                }
                if (it) atomicAdd(&ctlw(P.ctl, kWaitIters), (unsigned long long)it);
                sc[5] = (int)(t & 0x7fffffff);
                sc[6] = (int)(t >> 31);
            }
            sc[4] = ok;
        }
        tm.sync();
        ok = sc[4];
        const long long t = ((long long)sc[6] << 31) | (unsigned)sc[5];
        tm.sync();
        if (!ok) return 0;
        const bool loaded = read_slot(wl_slot(t));
        tm.sync();
        if (tm.leader()) {
            const unsigned slot = (unsigned)t & (P.wl_cap - 1);
            st_release_u32(&P.wl_seq[slot], (unsigned)t + (unsigned)P.wl_cap);
        }
        return loaded ? 1 : 2;
    }

    // The search ran out of node slots or registry entries (leader only).
    // A single solve stops as a whole (the caller may retry with larger
    // capacities).  A resident search of served requests ends only the
    // request that needed the room: it finishes with VC_ECAPACITY, its
    // remaining nodes are dropped when taken, and the others continue.
    __device__ void capacity_error(int site)
    {
        if (P.stack_top) {
            atomicCAS(&P.queries[q].status, VC_OK, VC_ECAPACITY);
            query_done(P, q);
        } else {
            set_error(P.ctl, VC_ECAPACITY, site);
        }
    }

    // Store a child: the worklist when it is hungry (load balancing,
    // Section 2.3), else the private stack, else the worklist.  Returns false
    // on overflow (error already recorded).
    __device__ bool push_child(int kind, int op, int root, int clo_c, int chi_c, int comp_c, int S_c, int hi_c,
                               int dpar_c = -1, int danc_c = -1, int dlb_c = 0)
    {
        // The worklist's level is read at the push itself: a reading taken
        // when the node started (one node earlier) measurably starved idle
        // workers (component-heavy 8 x 48: 23% -> 45% idle).
        int to_wl = 0;
        if (P.load_balance && tm.leader())
            to_wl = (long long)*(volatile unsigned long long *)&ctlw(P.ctl, kWlCount) < P.wl_low;
        to_wl = tm.bcast(to_wl);   // uniform decision: the team must take one path
        if (!to_wl && top < P.stack_depth) {
            write_slot(stack_slot(top), kind, op, root, clo_c, chi_c, comp_c, S_c, hi_c, dpar_c, danc_c, dlb_c);
            top++;
            if (tm.leader()) max_top() = max(max_top(), top);
            tm.sync();
            return true;
        }
        long long t = wl_reserve();
        if (t < 0) {
            if (top < P.stack_depth) {
                write_slot(stack_slot(top), kind, op, root, clo_c, chi_c, comp_c, S_c, hi_c, dpar_c, danc_c, dlb_c);
                top++;
                if (tm.leader()) max_top() = max(max_top(), top);
                tm.sync();
                return true;
            }
            if (tm.leader()) capacity_error(5);
            tm.sync();
            return false;
        }
        write_slot(wl_slot(t), kind, op, root, clo_c, chi_c, comp_c, S_c, hi_c, dpar_c, danc_c, dlb_c);
        wl_publish(t);
        tm.sync();
        return true;
    }

    // ------------------------------------------------------------ registry ops

    __device__ int reg_alloc()
    {
        if (lf_head() < 0) {
            const int c = reg_chunk_pop(P);
            if (c >= 0) { lf_head() = c; lf_count() = *(volatile int *)&P.reg[c].pad[1]; }
        }
        if (lf_head() >= 0) {
            const int e = lf_head();
            lf_head() = *(volatile int *)&P.reg[e].next;
            lf_count()--;
            return e;
        }
        const int e = (int)atomicAdd(&ctlw(P.ctl, kRegBump), 1ull);
        return e < P.reg_cap ? e : -1;
    }

    __device__ void reg_free(int e)
    {
        *(volatile int *)&P.reg[e].next = lf_head();
        lf_head() = e;
        lf_count()++;
        if (lf_count() >= 2 * kChunk) {
            // detach the first kChunk entries as one chunk
            int last = lf_head();
            for (int i = 1; i < kChunk; i++) last = *(volatile int *)&P.reg[last].next;
            const int chunk = lf_head();
            lf_head() = *(volatile int *)&P.reg[last].next;
            *(volatile int *)&P.reg[last].next = -1;
            lf_count() -= kChunk;
            reg_chunk_push(P, chunk, kChunk);
        }
    }

    // A leaf with cover size S in context `comp`: Best = min(Best, S) and the
    // witness bitmap follows (under the entry's lock).
    __device__ void improve()
    {
        int go = 0;
        if (tm.leader()) {
            RegEntry &E = P.reg[comp];
            if (S < ld_relaxed(&E.val) && reg_lock(P, comp)) {
                if (S < *(volatile int *)&E.val) go = 1;
                else reg_unlock(P, comp);
            }
            sc[7] = go;
        }
        tm.sync();
        go = sc[7];
        tm.sync();
        if (!go) return;
        uint32_t *w = reg_words(P, comp);
        const int nw = (chi >> 5) - (clo >> 5) + 1;
        for (int i = tm.rank; i < nw; i += tm.size()) w[i] = cov[i];
        if (tm.leader()) bytes_local += 4ll * nw + sizeof(RegEntry);
        __threadfence();
        tm.sync();
        int oldcur = 0;
        if (tm.leader()) {
            RegEntry &E = P.reg[comp];
            oldcur = vld(E.cur);
            E.has_w = 1;
            E.cur = S;
            atomicExch(&E.val, S);
            reg_unlock(P, comp);
            if (vld(E.link) < 0 && qk >= 0) query_done(P, q);   // PVC: a cover <= k exists
        }
        oldcur = tm.bcast(oldcur);
        if (pvc()) pvc_propagate(comp, oldcur, S);
    }

    __device__ __forceinline__ bool pvc() const { return qk >= 0; }

    // Entry a's witness := the parent entry's own cover S_P (its bitmap) plus
    // every child's current cover.  Caller holds a's lock; children are
    // locked while read when they may still improve.
    __device__ void assemble(int a, int par, bool lock_children)
    {
        const RegEntry &A = P.reg[a];
        const RegEntry &Pe = P.reg[par];
        const int aw = vld(A.wlo);
        uint32_t *dst = reg_words(P, a);
        const uint32_t *sp = reg_words(P, par);
        const int pnw = vld(Pe.nw), pw = vld(Pe.wlo);
        for (int i = tm.rank; i < pnw; i += tm.size()) dst[pw - aw + i] = __ldcg(sp + i);
        __threadfence();
        tm.sync();
        int ch = vld(Pe.first);
        for (int guard = 0; ch >= 0 && guard < (1 << 20); guard++) {
            int ok = 1;
            if (lock_children && tm.leader()) ok = reg_lock(P, ch);
            ok = tm.bcast(ok);
            if (!ok) return;   // aborted
            const RegEntry &C = P.reg[ch];
            const int cw = vld(C.wlo), cnw = vld(C.nw);
            const uint32_t *src = reg_words(P, ch);
            for (int i = tm.rank; i < cnw; i += tm.size()) dst[cw - aw + i] |= __ldcg(src + i);
            if (tm.leader()) bytes_local += 8ll * cnw;
            __threadfence();
            tm.sync();
            if (lock_children && tm.leader()) reg_unlock(P, ch);
            ch = vld(C.sib);
        }
    }

    // Section 3.5: in a parameterized query every improvement of a component
    // entry (its cover shrank from oldcur to newcur) is pushed up the chain
    // at once, so the root can reach k before the components are finished.
    __device__ void pvc_propagate(int c, int oldcur, int newcur)
    {
        for (int guard = 0; guard < (1 << 20); guard++) {
            const int par = vld(P.reg[c].link);
            if (par < 0 || newcur >= oldcur) return;
            int t = 0, a = -1, go = 0;
            if (tm.leader()) {
                t = atomicAdd(&P.reg[par].tot, newcur - oldcur) + (newcur - oldcur);
                a = vld(P.reg[par].link);
                if (t < ld_relaxed(&P.reg[a].val) && reg_lock(P, a)) {
                    if (t < vld(P.reg[a].val)) go = 1;
                    else reg_unlock(P, a);
                }
                sc[8] = t; sc[9] = a; sc[10] = go;
            }
            tm.sync();
            t = sc[8]; a = sc[9]; go = sc[10];
            tm.sync();
            if (!go) return;
            assemble(a, par, true);
            int olda = 0;
            if (tm.leader()) {
                RegEntry &A = P.reg[a];
                olda = vld(A.cur);
                A.has_w = 1;
                A.cur = t;
                atomicExch(&A.val, t);
                reg_unlock(P, a);
                if (vld(A.link) < 0) query_done(P, q);   // the query's root reached k
            }
            olda = tm.bcast(olda);
            c = a;
            oldcur = olda;
            newcur = t;
        }
    }

    // One node of context c completed (Section 3.3).  The last descendant of
    // a component adds its Best into the parent's Sum; the last component of a
    // parent updates the ancestor's Best and counts as its completion.
    __device__ void complete(int c)
    {
        for (int guard = 0;; guard++) {
            if (guard > (1 << 22)) {      // the registry chain is acyclic; never expected
                if (tm.leader()) set_error(P.ctl, VC_ETIMEOUT, 6);
                tm.sync();
                return;
            }
            int r = 0;
            if (tm.leader()) r = atom_add_acq_rel(&P.reg[c].live, -1) - 1;
            r = tm.bcast(r);
            if (r != 0) return;
            // component entry c is finished
            const RegEntry &C = P.reg[c];
            const int par = vld(C.link);
            if (par < 0) {
                if (tm.leader()) query_done(P, q);
                tm.sync();
                return;
            }
            const int bestc = vld(C.val);
            const int hw = vld(C.has_w);
            const RegEntry &Pe = P.reg[par];
            if (pvc()) {
                if (complete_pvc_child(c, par, bestc)) { c = vld(Pe.link); continue; }
                return;
            }
            if (hw) {
                const uint32_t *src = reg_words(P, c);
                const int cnw = vld(C.nw);
                uint32_t *dst = reg_words(P, par) + (vld(C.wlo) - vld(Pe.wlo));
                for (int i = tm.rank; i < cnw; i += tm.size()) atomicOr(&dst[i], __ldcg(src + i));
                if (tm.leader()) bytes_local += 8ll * cnw;
                __threadfence();
            }
            tm.sync();
            int r2 = 0;
            if (tm.leader()) {
                atomicAdd(&P.reg[par].val, bestc);
                // the child leaves the running set: its LB out, its Best in
                const int lbc = vld(C.pad[0]);
                atomicAdd((unsigned long long *)&P.reg[par].pad[0],
                          (unsigned long long)(unsigned)bestc - ((unsigned long long)(unsigned)lbc << 32));
                reg_free(c);
                r2 = atom_add_acq_rel(&P.reg[par].live, -1) - 1;
            }
            r2 = tm.bcast(r2);
            if (r2 != 0) return;
            // parent entry `par` is finished: Algorithm 2's update of its ancestor's Best
            const int anc = vld(Pe.link);
            const int sum = vld(Pe.val);
            int go = 0;
            if (tm.leader()) {
                RegEntry &A = P.reg[anc];
                if (sum < ld_relaxed(&A.val) && reg_lock(P, anc)) {
                    if (sum < *(volatile int *)&A.val) go = 1;
                    else reg_unlock(P, anc);
                }
            }
            go = tm.bcast(go);
            if (go) {
                const RegEntry &A = P.reg[anc];
                const uint32_t *src = reg_words(P, par);
                const int pnw = vld(Pe.nw);
                uint32_t *dst = reg_words(P, anc) + (vld(Pe.wlo) - vld(A.wlo));
                for (int i = tm.rank; i < pnw; i += tm.size()) dst[i] = __ldcg(src + i);
                if (tm.leader()) bytes_local += 8ll * pnw;
                __threadfence();
                tm.sync();
                if (tm.leader()) {
                    RegEntry &Aw = P.reg[anc];
                    Aw.has_w = 1;
                    atomicExch(&Aw.val, sum);
                    reg_unlock(P, anc);
                    if (vld(Aw.link) < 0 && qk >= 0) query_done(P, q);
                }
            }
            tm.sync();
            if (tm.leader()) reg_free(par);
            tm.sync();
            c = anc;
        }
    }

    // A child c of parent entry `par` finished in a parameterized query:
    // add its Best to Sum; when it was the last child, update the ancestor
    // from S_P + the children's covers (Algorithm 2's ancestor update), push that up
    // (Section 3.5), free the children and the parent, and return true so the
    // caller continues with the ancestor's LiveNodes.
    __device__ bool complete_pvc_child(int c, int par, int bestc)
    {
        int r2 = 0;
        if (tm.leader()) {
            atomicAdd(&P.reg[par].val, bestc);
            r2 = atom_add_acq_rel(&P.reg[par].live, -1) - 1;
        }
        r2 = tm.bcast(r2);
        if (r2 != 0) return false;
        const RegEntry &Pe = P.reg[par];
        const int anc = vld(Pe.link);
        const int sum = vld(Pe.val);
        int go = 0;
        if (tm.leader()) {
            RegEntry &A = P.reg[anc];
            if (sum < ld_relaxed(&A.val) && reg_lock(P, anc)) {
                if (sum < vld(A.val)) go = 1;
                else reg_unlock(P, anc);
            }
        }
        go = tm.bcast(go);
        if (go) {
            assemble(anc, par, false);
            int olda = 0;
            if (tm.leader()) {
                RegEntry &A = P.reg[anc];
                olda = vld(A.cur);
                A.has_w = 1;
                A.cur = sum;
                atomicExch(&A.val, sum);
                reg_unlock(P, anc);
                if (vld(A.link) < 0) query_done(P, q);
            }
            olda = tm.bcast(olda);
            pvc_propagate(anc, olda, sum);
        }
        tm.sync();
        if (tm.leader()) {
            int ch = vld(Pe.first);
            for (int guard = 0; ch >= 0 && guard < (1 << 20); guard++) {
                const int nx = vld(P.reg[ch].sib);
                reg_free(ch);
                ch = nx;
            }
            reg_free(par);
        }
        tm.sync();
        return true;
    }

    // ------------------------------------------------------------ components

    __device__ __forceinline__ int uf_find(int x)
    {
        int p = ((volatile int *)lab)[x];
        while (p != x) {
            int g = ((volatile int *)lab)[p];
            if (g != p) ((volatile int *)lab)[x] = g;   // path halving (benign race)
            x = p;
            p = g;
        }
        return x;
    }

    __device__ void uf_unite(int a, int b)
    {
        for (;;) {
            a = uf_find(a);
            b = uf_find(b);
            if (a == b) return;
            if (a > b) { int t = a; a = b; b = t; }
            int old = atomicCAS(&lab[b], b, a);
            if (old == b) return;
            b = old;
        }
    }

    // Connected components of the live vertices in [lo, hi] (union-find with
    // hooking to the smaller root, one pass over the live edges).  Returns
    // the number of components.  With two or more, or when need_labels is
    // set, lab[i] (i = v - lo) is afterwards the smallest relative index of
    // v's component (-1 for dead vertices); with one, the labels are left
    // unfinished (nothing reads them).
    __device__ int find_components(bool need_labels)
    {
        const int W = hi - lo + 1;
        for (int i = tm.rank; i < W; i += tm.size()) lab[i] = d[lo + i - wlo] > 0 ? i : -1;
        tm.sync();
        for (int i = tm.rank; i < W; i += tm.size()) {
            const int v = lo + i;
            if (d[v - wlo] == 0) continue;
            bytes_local += 8 + 4ll * (rp[v + 1] - rp[v]);
            for (int e = rp[v]; e < rp[v + 1]; e++) {
                const int u = col[e];
                if (u > v && u <= hi && d[u - wlo] > 0) uf_unite(i, u - lo);
            }
        }
        tm.sync();
        // the roots are final here: one per component
        int roots = 0;
        for (int i = tm.rank; i < W; i += tm.size()) roots += lab[i] == i;
        const int nc = tm.sum(roots);
        if (nc < 2 && !need_labels) return nc;
        // Final labels.  The walk to the root is read-only: with path
        // halving, a thread still passing through i could store a stale
        // ancestor into lab[i] after i's final label was written (seen with
        // block workers as vertices left outside their component).  Readers
        // of lab[i] now see its old parent or its root.
        for (int i = tm.rank; i < W; i += tm.size()) {
            if (lab[i] < 0) continue;
            int r = i;
            for (int p = ((volatile int *)lab)[r]; p != r; p = ((volatile int *)lab)[r]) r = p;
            ((volatile int *)lab)[i] = r;
        }
        tm.sync();
        return nc;
    }

    // Connected components of the live vertices in [lo, hi] by label
    // propagation, the alternative to find_components.  In each round every
    // live vertex takes the smallest label among its own and its live
    // neighbours' (pull form: the kGroup lanes of a group read the row, a
    // shuffle takes their minimum), then its label's label (pointer jumping);
    // rounds repeat until one lowers no label.  A label only falls and always
    // names a vertex of the same component, and after a round without change
    // the two ends of every live edge carry the same label, so the fixpoint
    // labels each component by its smallest relative index: the labels and
    // the count find_components leaves.  The number of rounds grows with the
    // logarithm of the components' diameter; each costs a pass over the live
    // edges and one team reduction.
    __device__ int find_components_lp()
    {
        const int W = hi - lo + 1;
        volatile int *vl = (volatile int *)lab;
        for (int i = tm.rank; i < W; i += tm.size()) lab[i] = d[lo + i - wlo] > 0 ? i : -1;
        tm.sync();
        // each round that changes a label moves the minimum one more hop at
        // least, so W + 1 rounds always reach the fixpoint
        for (int round = 0; round <= W; round++) {
            int changed = 0;
            for (int base = 0; base < W; base += ngroups()) {   // uniform over the warp
                const int i = base + group();
                int m = INT32_MAX, r0 = 0, r1 = 0;
                bool live = false;
                if (i < W) {
                    const int v = lo + i;
                    live = d[v - wlo] > 0;
                    if (live) {
                        m = vl[i];
                        r0 = rp[v];
                        r1 = rp[v + 1];
                    }
                }
                const int wmax = __reduce_max_sync(kFull, (r1 - r0 + kGroup - 1) / kGroup);
                for (int ch = 0; ch < wmax; ch++) {
                    const int e = r0 + ch * kGroup + glane();
                    if (e < r1) {
                        const int u = col[e];
                        if (u >= lo && u <= hi && d[u - wlo] > 0) m = min(m, vl[u - lo]);
                    }
                }
                for (int o = kGroup / 2; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
                if (live && glane() == 0) {
                    bytes_local += 8 + 4ll * (r1 - r0);
                    if (m < vl[i]) {
                        atomicMin(&lab[i], m);
                        changed = 1;
                    }
                }
            }
            for (int i = tm.rank; i < W; i += tm.size()) {
                const int l = vl[i];
                if (l < 0) continue;
                const int ll = vl[l];
                if (ll < l) {
                    atomicMin(&lab[i], ll);
                    changed = 1;
                }
            }
            if (tm.sum(changed) == 0) break;
        }
        int roots = 0;
        for (int i = tm.rank; i < W; i += tm.size()) roots += vl[i] == i;
        return tm.sum(roots);
    }

    // Cover of a chordless cycle component starting at vertex s: every other
    // vertex along the cycle (ceil(L/2) of them).  One thread.
    __device__ void cover_cycle(int s)
    {
        int prev = -1, cur = s, k = 0;
        for (int guard = 0; guard <= np; guard++) {
            if ((k & 1) == 0) cov_set(cur);
            int next = -1;
            for (int e = rp[cur]; e < rp[cur + 1]; e++) {
                const int x = col[e];
                if (x != prev && dg(x) > 0) { next = x; break; }
            }
            prev = cur;
            cur = next;
            k++;
            if (cur == s || cur < 0) break;
        }
    }

    // Statistics of the live vertices in [lo, hi]: degree sum, count,
    // lowest-index vertex of maximum degree, live window.  One reduction.
    __device__ WinStats window_stats()
    {
        WinStats t;
        t.e2 = 0; t.live = 0; t.dmax = 0; t.vmax = INT32_MAX; t.lo = INT32_MAX; t.hi = -1;
        for (int v = lo + tm.rank; v <= hi; v += tm.size()) {
            const int dv = (int)d[v - wlo];
            if (dv == 0) continue;
            t.live++;
            t.e2 += dv;
            if (dv > t.dmax) { t.dmax = dv; t.vmax = v; }
            t.lo = min(t.lo, v);
            t.hi = v;
        }
        return tm.stats(t);
    }

    enum { kComplete = 0, kVertexBranch = 1, kHandedOff = 2, kError = 3 };

    // Branch on >= 2 components, or close the trivial ones.  Returns
    //   kComplete      the node is finished (pruned or a leaf),
    //   kVertexBranch  one non-trivial component is left: branch on a vertex,
    //   kHandedOff     a branch on components was registered; the parent
    //                  entry now stands for this node (Section 3.3),
    //   kError         capacity exhausted (recorded in the control block).
    __device__ int handle_components(int B)
    {
        const int W = hi - lo + 1;
        int *scr = P.comp_scratch + (size_t)wid * 5 * P.ncap;
        int *csize = scr, *csum = scr + P.ncap, *cmin = scr + 2 * P.ncap, *cmax = scr + 3 * P.ncap,
            *chiv = scr + 4 * P.ncap;
        for (int i = tm.rank; i < W; i += tm.size()) {
            if (lab[i] == i) { csize[i] = 0; csum[i] = 0; cmin[i] = INT_MAX; cmax[i] = 0; chiv[i] = i; }
        }
        __threadfence();
        tm.sync();
        for (int i = tm.rank; i < W; i += tm.size()) {
            const int r = lab[i];
            if (r < 0) continue;
            const int dv = (int)d[lo + i - wlo];
            atomicAdd(&csize[r], 1);
            atomicAdd(&csum[r], dv);
            atomicMin(&cmin[r], dv);
            atomicMax(&cmax[r], dv);
            atomicMax(&chiv[r], i);
        }
        __threadfence();
        tm.sync();
        // classify: trivial (clique / cycle) components are closed here
        int s_triv = 0, lb_sum = 0, nontriv = 0;
        for (int i = tm.rank; i < W; i += tm.size()) {
            if (lab[i] != i) continue;
            const int sz = __ldcg(csize + i), mn = __ldcg(cmin + i), mx = __ldcg(cmax + i);
            const bool clique = mn == sz - 1 && mx == sz - 1;
            const bool cyc = mn == 2 && mx == 2;
            if (clique || cyc) {
                s_triv += clique ? sz - 1 : (sz + 1) / 2;
            } else {
                nontriv++;
                const int m = __ldcg(csum + i) / 2;
                lb_sum += (m + mx - 1) / mx;
            }
        }
        s_triv = tm.sum(s_triv);
        lb_sum = tm.sum(lb_sum);
        nontriv = tm.sum(nontriv);
        if (S + s_triv + lb_sum >= B) {       // even the lower bounds reach Best
            if (tm.leader()) atomicAdd(&ctlw(P.ctl, kPruned), 1ull);
            return kComplete;
        }
        if (s_triv > 0) {
            // cliques: all but the highest vertex; cycles: every other vertex
            for (int i = tm.rank; i < W; i += tm.size()) {
                const int r = lab[i];
                if (r < 0) continue;
                const int sz = __ldcg(csize + r), mn = __ldcg(cmin + r), mx = __ldcg(cmax + r);
                const bool clique = mn == sz - 1 && mx == sz - 1;
                if (clique && i != __ldcg(chiv + r)) cov_set(lo + i);
            }
            int ntriv = 0;
            for (int i = tm.rank; i < W; i += tm.size()) {
                if (lab[i] != i) continue;
                const int sz = __ldcg(csize + i), mn = __ldcg(cmin + i), mx = __ldcg(cmax + i);
                const bool clique = mn == sz - 1 && mx == sz - 1;
                const bool cyc = mn == 2 && mx == 2;
                if (cyc && !clique) cover_cycle(lo + i);
                ntriv += (clique || cyc);
            }
            tm.sync();
            for (int i = tm.rank; i < W; i += tm.size()) {
                const int r = lab[i];
                if (r < 0) continue;
                const int sz = __ldcg(csize + r), mn = __ldcg(cmin + r), mx = __ldcg(cmax + r);
                if ((mn == sz - 1 && mx == sz - 1) || (mn == 2 && mx == 2)) {
                    d[lo + i - wlo] = 0;
                    lab[i] = -1;
                }
            }
            ntriv = tm.sum(ntriv);
            S += s_triv;
            if (tm.leader()) atomicAdd(&ctlw(P.ctl, kTrivial), (unsigned long long)ntriv);
            tm.sync();
        }
        if (nontriv == 0) {                    // all edges covered: a leaf
            if (tm.leader()) atomicAdd(&ctlw(P.ctl, kLeaves), 1ull);
            improve();
            return kComplete;
        }
        if (nontriv == 1) return kVertexBranch;

        // ---- branch on components (the component branch of Algorithm 2, Section 3.3)
        // parent entry: Sum = |S| (this node's cover, trivial components
        // included), LiveComps = number of components, witness = S
        int pidx = -1;
        if (tm.leader()) {
            pidx = reg_alloc();
            if (pidx < 0) capacity_error(7);
        }
        pidx = tm.bcast(pidx);
        if (pidx < 0) return kError;
        {
            RegEntry &E = P.reg[pidx];
            if (tm.leader()) {
                E.val = S;
                E.live = nontriv;
                E.link = comp;
                E.lock = 0;
                E.has_w = 0;
                E.wlo = clo >> 5;
                E.nw = (chi >> 5) - (clo >> 5) + 1;
                E.q = q;
                E.kind = 1;
                E.first = -1;
                E.tot = S;      // + each child's cur, added as the children are registered
                // dynamic bounds: {LB of the running children, |S_P| + Best of the finished}
                *(unsigned long long *)&E.pad[0] = ((unsigned long long)(unsigned)lb_sum << 32) | (unsigned)S;
            }
            uint32_t *w = reg_words(P, pidx);
            const int nw = (chi >> 5) - (clo >> 5) + 1;
            for (int i = tm.rank; i < nw; i += tm.size()) w[i] = cov[i];
        }
        // child entries {Best_i, LiveNodes = 1, ParentIdx}, one per
        // non-trivial component in index order.  Pass 1 registers and links
        // every child (the parent's child list and running total are final
        // before any child becomes visible); pass 2 writes each child node
        // with the whole team (sequential over components, parallel within).
        // cmin[r] holds the child's entry index between the passes.
        for (int pass = 0; pass < 2; pass++) {
            for (int base = 0; base < W; base += tm.size()) {
                const int i = base + tm.rank;
                const bool isroot = i < W && lab[i] == i;
                int tot;
                const int pos = tm.excl_scan(isroot ? 1 : 0, &tot);
                for (int j = 0; j < tot; j++) {
                    // the thread holding the j-th root of this stripe broadcasts it
                    const int r = tm.max((isroot && pos == j) ? i : -1);
                    const int clo_c = lo + r, chi_c = lo + __ldcg(chiv + r);
                    const int sz = __ldcg(csize + r), mx = __ldcg(cmax + r);
                    const int m = __ldcg(csum + r) / 2;
                    const int lb = (m + mx - 1) / mx;
                    if (pass == 1) {
                        if (!push_child(1, -1, r, clo_c, chi_c, __ldcg(cmin + r), 0, chi_c, pidx, comp, lb))
                            return kError;
                        continue;
                    }
                    int bi = B - S - (lb_sum - lb);
                    if (bi > sz - 1) bi = sz - 1;
                    int cidx = -1;
                    if (tm.leader()) {
                        cidx = reg_alloc();
                        if (cidx < 0) capacity_error(8);
                    }
                    cidx = tm.bcast(cidx);
                    if (cidx < 0) return kError;
                    RegEntry &C = P.reg[cidx];
                    RegEntry &E = P.reg[pidx];
                    // a parameterized query needs every child's achievable cover
                    const int has = bi == sz - 1 || pvc();
                    const int cw0 = clo_c >> 5, cnw = (chi_c >> 5) - cw0 + 1;
                    if (tm.leader()) {
                        C.val = bi;
                        C.live = 1;
                        C.link = pidx;
                        C.lock = 0;
                        C.has_w = bi == sz - 1;
                        C.cur = sz - 1;
                        C.sib = E.first;
                        E.first = cidx;
                        E.tot += sz - 1;
                        C.wlo = cw0;
                        C.nw = cnw;
                        C.q = q;
                        C.kind = 0;
                        C.pad[0] = lb;
                        cmin[r] = cidx;
                    }
                    if (has) {
                        // every vertex of the component but its highest one
                        uint32_t *w = reg_words(P, cidx);
                        for (int x = tm.rank; x < cnw; x += tm.size()) {
                            uint32_t bits = 0;
                            for (int bb = 0; bb < 32; bb++) {
                                const int v = (cw0 + x) * 32 + bb;
                                if (v >= lo + r && v < chi_c && lab[v - lo] == r) bits |= 1u << bb;
                            }
                            w[x] = bits;
                        }
                    }
                }
            }
            __threadfence();
            tm.sync();
        }
        if (tm.leader()) {
            atomicAdd(&ctlw(P.ctl, kCompBranches), 1ull);
            int b = min(nontriv, kHistBins) - 2;
            if (b >= 0) atomicAdd(&ctlw(P.ctl, kHist + b), 1ull);
        }
        tm.sync();
        return kHandedOff;
    }

    // ------------------------------------------------------------ node

    // Process the node now in shared memory and all its left descendants.
    // The leader's loads for the next node of this context, issued at once
    // and consumed by process(): the abort flag, the context's Best and the
    // two words of the dynamic bound.  They are
    // issued early (when a node is loaded, or before the left child's
    // vertex is removed) so that their latency overlaps the team's work.
    // A stale value is safe: Best only decreases, so a stale bound prunes
    // less, and a late abort costs one more node.
    __device__ __forceinline__ void prefetch()
    {
        // (the low word of the abort flag)
        pf_ab = *(volatile unsigned *)&ctlw(P.ctl, kAbort);
        pf_bv = ld_relaxed(&P.reg[comp].val);
        pf_dyn = dpar >= 0 && !P.no_dyn_bounds;
        if (pf_dyn) {
            pf_pk = ld_relaxed_u64((const unsigned long long *)&P.reg[dpar].pad[0]);
            pf_av = ld_relaxed(&P.reg[danc].val);
        }
        pf_ok = true;
    }

    // Process the node now in shared memory and all its left descendants.
    __device__ void process()
    {
        for (int iter = 0;; iter++) {
            int B = 0;
            if (tm.leader()) {
                if (!pf_ok) prefetch();
                pf_ok = false;
                if (pf_ab) B = INT_MIN;
                else if (iter > 0 && P.quantum_ns > 0 && globaltimer() > t_end()) B = kPreempt;
                else {
                    B = pf_bv;
                    if (pf_dyn && qk < 0) {
                        // Best of the enclosing context minus what the parent
                        // and its other children already need: if this
                        // component cannot beat it, the parent's sum cannot
                        // beat the ancestor (every running sibling needs at
                        // least its LB), so no cover is lost
                        const long long bd = (long long)pf_av - (long long)(unsigned)(pf_pk & 0xffffffffull) -
                                             ((long long)(pf_pk >> 32) - dlb);
                        if (bd < B) B = bd < 0 ? 0 : (int)bd;
                    }
                }
            }
            B = tm.bcast(B);
            if (B == INT_MIN) { stop = true; return; }   // aborted (decided by the leader for the whole team)
            if (B == kPreempt) {
                // the slice is over: store this node (no pending operation) so
                // that the next slice resumes it; it stays live in its context
                push_child(0, -1, -1, clo, chi, comp, S, hi);
                if (tm.leader()) atomicAdd(&ctlw(P.ctl, kPreempts), 1ull);
                preempted = true;
                return;
            }
            nflush++;
            qnodes++;
            Stats st = reduce(B);
            lap(kPhReduce);
            if (st.pruned) {
                if (tm.leader()) atomicAdd(&ctlw(P.ctl, kPruned), 1ull);
                complete(comp);
                lap(kPhDone);
                return;
            }
            const long long bud = (long long)B - S - 1;
            if (S >= B || st.e2 / 2 > bud * bud) {      // stopping condition
                if (tm.leader()) atomicAdd(&ctlw(P.ctl, kPruned), 1ull);
                complete(comp);
                lap(kPhDone);
                return;
            }
            if (st.e2 == 0) {                            // a new best cover
                if (tm.leader()) atomicAdd(&ctlw(P.ctl, kLeaves), 1ull);
                improve();
                complete(comp);
                lap(kPhDone);
                return;
            }
            if (!P.no_bounds) {      // Section 4.3: only the non-zero window
                lo = st.lo;
                hi = st.hi;
            }
            int vmax = st.vmax;
            if (P.use_components) {
                const bool clique = (long long)st.live * (st.live - 1) == st.e2;
                const bool cycle = st.dmax == 2 && st.e2 == 2ll * st.live;
                const int ncomp = P.comp_lp ? find_components_lp() : find_components(clique || cycle);
                if (ncomp >= 2 || clique || cycle) {
                    const int r = handle_components(B);
                    lap(kPhComp);
                    if (r == kComplete) { complete(comp); lap(kPhDone); return; }
                    if (r != kVertexBranch) return;
                    // one non-trivial component is left: its window and v_max
                    const WinStats w = window_stats();
                    vmax = w.live > 0 ? w.vmax : -1;
                    if (!P.no_bounds && w.live > 0) { lo = w.lo; hi = w.hi; }
                }
                lap(kPhComp);
            }
            // ---- branch on v_max (the vertex branch of Algorithm 1)
            if (vmax < lo || vmax > hi) {                         // cannot happen with edges left
                if (tm.leader()) set_error(P.ctl, VC_ECAPACITY, 9);
                tm.sync();
                return;
            }
            // two children replace one node; the leader's increment precedes
            // its own publication of the right child (fence, then release)
            if (tm.leader()) atomicAdd(&P.reg[comp].live, 1);
            if (!push_child(0, vmax, -1, clo, chi, comp, S, hi)) return;
            if (tm.leader()) prefetch();   // for the left child, overlapping its update
            remove_vertex(vmax);
            depth++;
            lap(kPhBranch);
        }
    }

    // ------------------------------------------------------------ main loop

    // Add this worker's nodes of the current query to its counter; a query
    // over its budget stops with VC_EBUDGET (the others continue).
    __device__ void flush_query_nodes()
    {
        if (tm.leader() && qnodes > 0 && qcur >= 0) {
            QueryDesc &Q = P.queries[qcur];
            const long long tot = (long long)atomicAdd((unsigned long long *)&Q.nodes, (unsigned long long)qnodes) + qnodes;
            if (Q.budget > 0 && tot > Q.budget) {
                atomicCAS(&Q.status, VC_OK, VC_EBUDGET);
                query_done(P, qcur);
            }
        }
        qnodes = 0;
    }

    __device__ void flush_counters()
    {
        flush_query_nodes();
        const long long b = tm.lsum(bytes_local);
        bytes_local = 0;
        if (tm.leader()) {
            atomicAdd(&ctlw(P.ctl, kBytes), (unsigned long long)b);
            atomicAdd(&ctlw(P.ctl, kNodes), (unsigned long long)nflush);
            atomicAdd(&ctlw(P.ctl, kProgress), 1ull);
            atomicMax(&ctlw(P.ctl, kMaxStack), (unsigned long long)max_top());
        }
        nflush = 0;
    }

    __device__ void run()
    {
        if (P.quantum_ns > 0 && tm.leader()) t_end() = globaltimer() + (unsigned long long)P.quantum_ns;
        if (P.breakdown && tm.leader()) {
            for (int k = 0; k < kPhases; k++) ph()[k] = 0;
            ph()[kPhases] = clock64();
        }
        unsigned long long idle_since = 0, seen_progress = ~0ull;
        int backoff = 32;
        // counters are flushed every 64 nodes, more often under a small node budget
        long long flush_every = 64;
        if (P.node_budget > 0) flush_every = max(1ll, min(64ll, P.node_budget / 64));
        for (;;) {
            // process() sees an abort with its first loads; the time slice's
            // end is read from the SM's clock (no memory access)
            if (stop) break;
            if (P.quantum_ns > 0) {
                int ab = 0;
                if (tm.leader()) ab = globaltimer() > t_end();
                if (tm.bcast(ab)) break;
            }
            // 0 nothing, 1 node loaded, 2 node of a finished request (or of an
            // earlier request of a recycled slot) dropped unexpanded
            int got = 0;
            if (top > 0) {
                top--;
                got = read_slot(stack_slot(top)) ? 1 : 2;
            } else {
                got = wl_pop();
            }
            if (got == 2) {
                backoff = 32;
                idle_since = 0;
                lap(kPhPop);
                tm.sync();
                continue;
            }
            if (got == 1) {
                lap(kPhPop);
                backoff = 32;
                idle_since = 0;
                if (q != qcur) {
                    flush_query_nodes();
                    qcur = q;
                }
                const unsigned long long tp = tm.leader() ? globaltimer() : 0ull;
                process();
                if (tm.leader()) {
                    const unsigned long long dt = globaltimer() - tp;
                    if (dt > 100000ull) atomicMax(&ctlw(P.ctl, kMaxProcNs), dt);
                }
                if (preempted || stop) break;
                if (nflush >= flush_every) flush_counters();
                tm.sync();
                continue;
            }
            // idle
            int stop = 0;
            if (tm.leader()) {
                const unsigned long long rem = *(volatile unsigned long long *)&ctlw(P.ctl, kRemaining);
                if (aborted(P.ctl)) stop = 3;
                else if (rem == 0ull) stop = 2;
            }
            if (tm.leader() && !stop) {
                const unsigned long long prog = *(volatile unsigned long long *)&ctlw(P.ctl, kProgress);
                const unsigned long long now = globaltimer();
                if (prog != seen_progress || idle_since == 0) { seen_progress = prog; idle_since = now; }
                else if ((long long)(now - idle_since) > P.idle_timeout_ns) { set_error(P.ctl, VC_ETIMEOUT, 11); stop = 1; }
                __nanosleep(backoff);
            }
            backoff = min(backoff * 2, 4096);
            stop = tm.bcast(stop);
            lap(kPhIdle);
            if (stop) break;
        }
        const unsigned long long tx = tm.leader() ? globaltimer() : 0ull;
        flush_counters();
        if (tm.leader()) {
            if (lf_count() > 0) reg_chunk_push(P, lf_head(), lf_count());
            lf_head() = -1;
            lf_count() = 0;
            if (P.stack_top) P.stack_top[wid] = top;
            atomicMax(&ctlw(P.ctl, kMaxExitNs), globaltimer() - tx);
            if (P.breakdown)
                for (int k = 0; k < kPhases; k++) atomicAdd(&ctlw(P.ctl, kPhase + k), ph()[k]);
        }
    }
};

// ---------------------------------------------------------------- kernels

// Register caps keep the occupancy the planner counts on: block workers fit
// two 512-thread (four 256-thread) blocks per SM, warp workers three blocks
// of eight warps.
template <typename T, int WT, bool GA = false>
__global__ void __launch_bounds__(WT ? 256 : 1024, WT ? 3 : 1) search_kernel(const __grid_constant__ SearchParams P)
{
    extern __shared__ __align__(16) char smem_all[];
    // single-query launches keep the induced CSR (row pointers, then
    // columns) in shared memory: every row read of the search hits it
    const int *csr = nullptr;
    char *smem = smem_all;
    if (P.csr_smem > 0) {
        const QueryDesc &Q = P.queries[P.csr_query];
        int *dst = (int *)smem_all;
        const int nrp = Q.np + 1, ncol = Q.m2p;
        for (int i = threadIdx.x; i < nrp; i += blockDim.x) dst[i] = __ldg(Q.rp2 + i);
        for (int i = threadIdx.x; i < ncol; i += blockDim.x) dst[nrp + i] = __ldg(Q.col2 + i);
        __syncthreads();
        csr = dst;
        smem = smem_all + P.csr_smem;
    }
    if constexpr (WT == 1) {
        const int warp = threadIdx.x >> 5;
        const int wpb = blockDim.x >> 5;
        const int wid = blockIdx.x * wpb + warp;
        Team<1> t;
        t.rank = threadIdx.x & 31;
        static_assert(!GA, "warp workers keep their arrays in shared memory");
        char *mine = smem + (size_t)warp * align_up(worker_smem_bytes<T>(P.ncap, P.wcap, false, true), 16);
        Worker<T, 1> w(P, t, wid, mine, csr);
        w.run();
    } else {
        Team<0> t;
        t.rank = threadIdx.x;
        t.nthreads = blockDim.x;
        t.red = nullptr;
        Worker<T, 0, GA> w(P, t, blockIdx.x, smem, csr);
        w.run();
    }
}

// Registry free list over [first, cap) and each query's root entry + node.
template <typename T>
__global__ void search_init_kernel(SearchParams P, int first)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int s = tid; s < P.wl_cap; s += nth) P.wl_seq[s] = (unsigned)s;
    for (int i = tid; i < kCtlWords; i += nth) {
        unsigned long long v = 0;
        if (i == kRegHead * kCtlStride) v = 0xffffffffull;            // overflow list empty
        if (i == kRegBump * kCtlStride) v = (unsigned long long)first;  // after the root entries
        P.ctl[i] = v;
    }
}

// One block per query: its root registry entry and root node (worklist).
template <typename T>
__global__ void search_roots_kernel(SearchParams P, const int *root_slot)
{
    const int qi = blockIdx.x;
    QueryDesc &Q = P.queries[qi];
    const int slot = root_slot[qi];
    if (slot < 0) return;
    constexpr int V = Vec<T>::kPer16;
    const int np = Q.np;
    if (threadIdx.x == 0) {
        RegEntry &R = P.reg[qi];
        R.val = Q.bound - Q.forced;
        R.live = 1;
        R.link = -1;
        R.lock = 0;
        R.has_w = 0;
        R.wlo = 0;
        R.nw = (np - 1) / 32 + 1;
        R.q = qi;
        R.kind = 0;
        R.next = -1;
        Q.root_entry = qi;
        Q.done = 0;
        Q.nodes = 0;
        Q.budget = P.node_budget;
    }
    char *s = P.wl_slots + (size_t)slot * P.slot_bytes;
    NodeHdr *h = (NodeHdr *)s;
    if (threadIdx.x == 0) {
        h->S = 0; h->comp = qi; h->lo = 0; h->hi = np - 1; h->clo = 0; h->chi = np - 1;
        h->op = -1; h->q = qi; h->cov_empty = 1; h->depth = 0; h->gen = Q.gen;
        h->dpar = -1; h->danc = -1; h->dlb = 0; h->fix = 0; h->pad = 0;
    }
    T *dd = (T *)(s + sizeof(NodeHdr));
    const int lim = align_up(np, V);
    for (int v = threadIdx.x; v < lim; v += blockDim.x)
        dd[v] = v < np ? (T)(Q.rp2[v + 1] - Q.rp2[v]) : (T)0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) P.wl_seq[slot] = (unsigned)slot + 1u;
}

__global__ void search_roots_publish(SearchParams P, int nroots)
{
    ctlw(P.ctl, kWlTail) = (unsigned long long)nroots;
    ctlw(P.ctl, kWlCount) = (unsigned long long)nroots;
    ctlw(P.ctl, kRemaining) = (unsigned long long)nroots;
}

// Served requests (one block each): copy the root-reduced descriptor from the
// staging array into its slot.  A request that still needs a search gets its
// root registry entry (index = slot) and its root node in the shared
// worklist, behind the nodes of the requests admitted earlier.  The search
// kernel is not running meanwhile (the stream orders the launches), so the
// worklist tickets are taken without contention.  A request whose induced
// graph exceeds the resident node capacity or the degree type finishes with
// VC_ECAPACITY; one settled by the root phase (or rejected) is done at once.
//
// Size classes: every class has a resident search of its own (its own node
// capacity, worklist and registry) and runs this kernel over all admitted
// requests; a class places the requests whose induced graph has more than
// min_np and at most max_np vertices, class 0 also those the root phase
// settled or rejected, and the last class rejects what exceeds it.
template <typename T>
__global__ void serve_place_kernel(SearchParams P, const QueryDesc *staging, const int *slot_idx, int max_np,
                                   int lane, int min_np, int last)
{
    __shared__ long long s_t;
    __shared__ int s_ok;
    constexpr int V = Vec<T>::kPer16;
    const QueryDesc &Sg = staging[blockIdx.x];
    const bool settled = Sg.status != VC_OK || Sg.answered || Sg.np <= 0;
    const bool mine = settled ? lane == 0 : ((Sg.np > min_np && Sg.np <= max_np) || (last && Sg.np > max_np));
    if (!mine) return;   // (uniform over the block)
    const int qi = slot_idx[blockIdx.x];
    QueryDesc &Q = P.queries[qi];
    if (threadIdx.x == 0) {
        Q = staging[blockIdx.x];
        Q.lane = lane;
        int ok = Q.status == VC_OK && !Q.answered && Q.np > 0;
        const bool fits_t = sizeof(T) >= 4 || Q.maxdeg <= (int)((1u << (8 * sizeof(T))) - 1u);
        if (ok && (Q.np > max_np || !fits_t)) {
            Q.status = VC_ECAPACITY;
            ok = 0;
        }
        Q.done = ok ? 0 : 1;
        Q.nodes = 0;
        if (ok) {
            RegEntry &R = P.reg[qi];
            R.val = Q.bound - Q.forced;
            R.live = 1;
            R.link = -1;
            R.lock = 0;
            R.has_w = 0;
            R.wlo = 0;
            R.nw = (Q.np - 1) / 32 + 1;
            R.q = qi;
            R.kind = 0;
            R.next = -1;
            Q.root_entry = qi;
            Q.budget = P.node_budget;
            const long long t = (long long)atomicAdd(&ctlw(P.ctl, kWlTail), 1ull);
            const unsigned ws = (unsigned)t & (P.wl_cap - 1);
            int it = 0;
            while (ld_acquire_u32(&P.wl_seq[ws]) != (unsigned)t) {   // free once consumed
                if (++it > (1 << 20)) { set_error(P.ctl, VC_ETIMEOUT, 21); ok = 0; break; }
                __nanosleep(64);
            }
            s_t = t;
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const long long t = s_t;
    const unsigned ws = (unsigned)t & (P.wl_cap - 1);
    char *s = P.wl_slots + (size_t)ws * P.slot_bytes;
    const int np = Q.np;
    if (threadIdx.x == 0) {
        NodeHdr *h = (NodeHdr *)s;
        h->S = 0; h->comp = qi; h->lo = 0; h->hi = np - 1; h->clo = 0; h->chi = np - 1;
        h->op = -1; h->q = qi; h->cov_empty = 1; h->depth = 0; h->gen = Q.gen;
        h->dpar = -1; h->danc = -1; h->dlb = 0; h->fix = 0; h->pad = 0;
    }
    T *dd = (T *)(s + sizeof(NodeHdr));
    const int lim = align_up(np, V);
    for (int v = threadIdx.x; v < lim; v += blockDim.x)
        dd[v] = v < np ? (T)(Q.rp2[v + 1] - Q.rp2[v]) : (T)0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        st_release_u32(&P.wl_seq[ws], (unsigned)t + 1u);
        atomicAdd(&ctlw(P.ctl, kWlCount), 1ull);
        atomicAdd(&ctlw(P.ctl, kRemaining), 1ull);
    }
}

}  // namespace vcg

// ---------------------------------------------------------------- host side

#include "vc_internal.h"

namespace vcg {

template <typename T, int WT, bool GA = false>
static cudaError_t plan_one(int threads, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(search_kernel<T, WT, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<T, WT, GA>, threads, smem);
}

// The search kernel instance of a plan.
template <typename T>
static void launch_search(const SearchPlan &pl, const SearchParams &P, cudaStream_t s)
{
    if (pl.warp_team)
        search_kernel<T, 1><<<pl.blocks, pl.threads, pl.smem, s>>>(P);
    else if (pl.wglobal_bytes > 0)
        search_kernel<T, 0, true><<<pl.blocks, pl.threads, pl.smem, s>>>(P);
    else
        search_kernel<T, 0><<<pl.blocks, pl.threads, pl.smem, s>>>(P);
}

template <typename T>
static int plan_t(int team_req, int ncap, int wcap, int sms, int csr_bytes, SearchPlan *pl)
{
    const bool warp = team_req == 32;
    const int wsm = align_up(worker_smem_bytes<T>(ncap, wcap, false, warp), 16);
    const int kMaxSmem = 227 * 1024 - csr_bytes;
    pl->dtype = sizeof(T);
    pl->slot_bytes = slot_bytes_for<T>(ncap, wcap);
    pl->wglobal_bytes = 0;
    // automatic: 128-thread block workers for induced graphs up to 4,096
    // vertices, 256-thread ones above (measured faster on GB300 than warp
    // workers or 512-thread blocks); warp workers on request
    int bps = 0;
    if (warp) {
        int wpb = kMaxSmem / wsm;
        if (wpb > 8) wpb = 8;
        if (wpb < 1) return VC_ECAPACITY;
        pl->warp_team = 1;
        pl->threads = 32 * wpb;
        pl->smem = (size_t)wpb * wsm + csr_bytes;
        if (plan_one<T, 1>(pl->threads, pl->smem, &bps) != cudaSuccess) return VC_ECUDA;
    } else {
        int th = team_req >= 64 ? team_req : (ncap > 4096 ? 256 : 128);
        pl->warp_team = 0;
        pl->threads = th;
        if (wsm <= kMaxSmem) {
            pl->smem = (size_t)wsm + csr_bytes;
            if (plan_one<T, 0>(pl->threads, pl->smem, &bps) != cudaSuccess) return VC_ECUDA;
        }
        if (wsm > kMaxSmem || bps < 1) {
            // node arrays too large for shared memory: keep them in global
            // memory (no staged CSR either)
            pl->wglobal_bytes = ((long long)worker_array_bytes<T>(ncap, wcap) + 255) / 256 * 256;
            pl->csr_bytes = 0;
            pl->smem = (size_t)align_up(worker_smem_bytes<T>(ncap, wcap, true, false), 16);
            if (plan_one<T, 0, true>(pl->threads, pl->smem, &bps) != cudaSuccess) return VC_ECUDA;
        }
    }
    if (bps < 1) return VC_ECAPACITY;
    pl->blocks = bps * sms;
    pl->workers = pl->blocks * (pl->warp_team ? pl->threads / 32 : 1);
    return VC_OK;
}

int search_plan(int dtype, int team_req, int ncap, int wcap, int sms, int csr_bytes, SearchPlan *out)
{
    out->csr_bytes = csr_bytes;
    switch (dtype) {
    case 1: return plan_t<uint8_t>(team_req, ncap, wcap, sms, csr_bytes, out);
    case 2: return plan_t<uint16_t>(team_req, ncap, wcap, sms, csr_bytes, out);
    default: return plan_t<uint32_t>(team_req, ncap, wcap, sms, csr_bytes, out);
    }
}

template <typename T>
static cudaError_t run_t(const SearchPlan &pl, SearchParams &P, const int *d_root_slot, int nq, int nroots,
                         cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, unsigned ev_flags)
{
    search_init_kernel<T><<<256, 256, 0, s>>>(P, nq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    search_roots_kernel<T><<<nq, 256, 0, s>>>(P, d_root_slot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    search_roots_publish<<<1, 1, 0, s>>>(P, nroots);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev0 && (e = cudaEventRecordWithFlags(ev0, s, ev_flags)) != cudaSuccess) return e;
    launch_search<T>(pl, P, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev1 && (e = cudaEventRecordWithFlags(ev1, s, ev_flags)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T>
static cudaError_t slice_t(const SearchPlan &pl, const SearchParams &P, cudaStream_t s)
{
    launch_search<T>(pl, P, s);
    return cudaGetLastError();
}

cudaError_t search_slice_run(const SearchPlan &pl, const SearchParams &P, cudaStream_t s)
{
    switch (pl.dtype) {
    case 1: return slice_t<uint8_t>(pl, P, s);
    case 2: return slice_t<uint16_t>(pl, P, s);
    default: return slice_t<uint32_t>(pl, P, s);
    }
}

cudaError_t search_reset_run(const SearchParams &P, int first, cudaStream_t s)
{
    search_init_kernel<uint8_t><<<256, 256, 0, s>>>(P, first);
    return cudaGetLastError();
}

cudaError_t serve_place_run(const SearchPlan &pl, const SearchParams &P, const QueryDesc *d_staging,
                            const int *d_slot_idx, int na, int max_np, int lane, int min_np, int last,
                            cudaStream_t s)
{
    if (na <= 0) return cudaSuccess;
    switch (pl.dtype) {
    case 1: serve_place_kernel<uint8_t><<<na, 256, 0, s>>>(P, d_staging, d_slot_idx, max_np, lane, min_np, last); break;
    case 2: serve_place_kernel<uint16_t><<<na, 256, 0, s>>>(P, d_staging, d_slot_idx, max_np, lane, min_np, last); break;
    default: serve_place_kernel<uint32_t><<<na, 256, 0, s>>>(P, d_staging, d_slot_idx, max_np, lane, min_np, last); break;
    }
    return cudaGetLastError();
}

cudaError_t search_run(const SearchPlan &pl, SearchParams &P, const int *d_root_slot, int nq, int nroots,
                       cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, unsigned ev_flags)
{
    switch (pl.dtype) {
    case 1: return run_t<uint8_t>(pl, P, d_root_slot, nq, nroots, s, ev0, ev1, ev_flags);
    case 2: return run_t<uint16_t>(pl, P, d_root_slot, nq, nroots, s, ev0, ev1, ev_flags);
    default: return run_t<uint32_t>(pl, P, d_root_slot, nq, nroots, s, ev0, ev1, ev_flags);
    }
}

}  // namespace vcg
