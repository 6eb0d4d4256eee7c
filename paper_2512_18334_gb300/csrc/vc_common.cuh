// Shared device-side definitions of the GB300 vertex-cover solver.
//
// Layout in HBM (all device memory, owned by the library):
//   per query:   input CSR, root-phase scratch (degrees, states, frontiers),
//                induced CSR (rp2, col2) and the map back to original ids;
//   per launch:  node slots (private stacks + shared worklist), the
//                component-branch registry and its witness bitmaps.
//
// A search-tree node is a degree array over a window of the induced graph
// plus a cover bitmap (Section 4.1 "degree array"; Section 4.3 "bounds on
// non-zero entries").  Node slot = NodeHdr | degrees [lo, hi] (T each,
// 16-byte aligned) | cover words of the context window.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vc_gb300.h"

namespace vcg {

// ------------------------------------------------------------------ limits

constexpr int kMaxBlock = 1024;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kHistBins = 16;

// ------------------------------------------------------------------ queries

// One solve request: a graph and a mode (MVC, or PVC with k).  Written by the
// host (inputs, buffer pointers) and by the root-phase kernel (outputs).
struct QueryDesc {
    // input graph (device copies owned by the vc_graph handle)
    int n;
    int m2;              // row_ptr[n] = 2|E|
    const int *rp;
    const int *col;
    int k;               // -1: minimum cover; >= 0: is there a cover <= k?
    int maxdeg_in;       // maximum degree of the input graph

    // root-phase scratch (device, >= n entries each unless noted)
    int *deg;            // live degree
    int *aux;            // marks / greedy states
    int *fr0;            // frontier lists
    int *fr1;
    int *flag;           // frontier membership
    int *forced_list;    // vertices forced into the cover at the root (>= n)
    int *heavy;          // long rows handed to whole warps (>= n)
    uint8_t *st;         // 0 live, 1 forced into the cover, 2 greedy cover
    uint8_t *cover_flags;// final cover, original numbering (n bytes)

    // induced subgraph (device): rp2[np+1], col2[m2p], orig[np]
    int *rp2;
    int *col2;
    int *orig;

    // root-phase outputs
    int status;          // VC_OK or a negative status
    int forced;          // |F|
    int greedy;          // greedy cover size of the whole graph (-1: not computed)
    int bound;           // cover size the search must beat (whole graph)
    int np;              // vertices of the induced subgraph
    int m2p;             // 2 |E(induced)|
    int maxdeg;          // max degree of the induced subgraph
    int answered;        // 1: the root phase already settled the answer

    // search outputs / final answer
    int root_entry;      // registry entry of the induced graph's context
    int result;          // MVC: minimum size; PVC: size found (yes) or -1
    int yes;             // PVC answer (1 for MVC)
    int improved;        // 1: the search found a cover better than `bound`
    int cover_len;       // entries written to cover_list
    int done;            // set once when the query is finished during the search
    int rounds;          // root-phase rule rounds (diagnostics)
    int gen;             // generation of the query slot (served requests): node
                         // headers carry it; a node whose generation differs
                         // belongs to an earlier request of the slot and is dropped
    int skip_root_rules; // 1: no reduction rules at the root (ablation); the
                         // induced graph is every vertex with an edge
    int emit_complement; // 1: the output list is the complement of the cover
                         // (a maximum independent set when the cover is minimum)
    int *crown_ws;       // non-null: apply the crown reduction after the root phase
                         // (scratch of 13 * n + 1 + 2|E| ints)
    int crown_status;    // 0 nothing removed, 1 applied, -1 skipped (check failed)
    int crown_forced;    // vertices the crown reduction put in the cover
    int crown_removed;   // vertices it removed in all (cover + excluded)
    int listed;          // 1: the root phase already wrote cover_list / cover_out
                         // and cover_len (the answer is its forced set)
    long long root_cycles[4];  // clock64 cycles: phase 1, greedy, phase 2, induce
    long long nodes;     // search-tree nodes spent on this query
    long long budget;    // node budget of this query (0: none)
    int *cover_list;     // ascending original ids (device, >= n)
    int *cover_out;      // non-null: finalisation writes the same list here too
                         // (mapped host memory, >= n entries)
    int lane;            // served requests: the size class whose resident search holds it
    int best;            // a searched query that stopped early (node budget): the
                         // size of the best cover known then (forced + the search's
                         // incumbent, or the initial bound)
};

// One served request as seen after a time slice, written by the device into
// mapped host memory.
struct RetireRec {
    int slot;
    int state;             // 0: still searching; 1: finished (fields below valid)
    int status;
    int result;
    int yes;
    int cover_len;
    long long cover_off;   // offset in the cover buffer, -1: buffer full (retry)
    long long nodes;
    int np;
    int lane;              // size class of the request (its resident search)
};

// ------------------------------------------------------------------ nodes

struct NodeHdr {            // 64 bytes; the payload after it stays 16-aligned
    int32_t S;              // cover vertices chosen in this component context
    int32_t comp;           // registry entry of the enclosing component context
    int32_t lo, hi;         // degree window stored in the slot (lo % vec == 0)
    int32_t clo, chi;       // component context window (cover bitmap range)
    int32_t op;             // -1, or v: apply "G - N(v)" when the node is loaded
    int32_t q;              // query id
    int32_t cov_empty;      // 1: cover bitmap not stored (all zero)
    int32_t depth;          // search-tree depth (statistics only)
    int32_t gen;            // generation of the query slot when the node was made
    // dynamic component bound (minimum covers): the parent entry of the
    // node's component context, that parent's ancestor, and the context's
    // lower bound (dpar = -1: the context is a root entry)
    int32_t dpar, danc, dlb;
    int32_t fix;            // 1: the degree array is at a fixpoint of the degree-one
                            // and degree-two-triangle rules (pending op aside)
    int32_t pad;
};
static_assert(sizeof(NodeHdr) == 64, "node header must stay 64 bytes");

// ------------------------------------------------------------------ registry

// One entry of the component-branch registry (Section 3.3).  A "component"
// entry holds {Best, LiveNodes, ParentIdx}; a "parent" entry holds
// {Sum, LiveComps, AncestorIdx}.  The query's induced graph itself is a
// component entry whose parent is -1.
struct RegEntry {
    int32_t val;     // Best (component) or Sum (parent)
    int32_t live;    // LiveNodes (component) or LiveComps (parent)
    int32_t link;    // ParentIdx (component) or AncestorIdx (parent)
    int32_t lock;    // witness-bitmap lock (component entries)
    int32_t has_w;   // 1: the witness bitmap holds a cover of size val
    int32_t wlo;     // first bitmap word (vertex wlo*32 is bit 0 of word 0)
    int32_t nw;      // bitmap words in use
    int32_t q;       // query id
    int32_t next;    // free-list link
    int32_t kind;    // 0 component, 1 parent
    // parameterized queries (Section 3.5) keep every improvement flowing up:
    int32_t cur;     // component: size of the cover its bitmap holds
    int32_t sib;     // component: next child of the same parent (-1 ends)
    int32_t first;   // parent: first child
    int32_t tot;     // parent: |S_P| + sum of its children's cur
    // pad: while the entry is free, the chunk link and size of the free
    // stack; while in use, dynamic component bounds (minimum covers):
    //   component: pad[0] = its lower bound LB_i
    //   parent:    pad as one 64-bit word {high: sum of the LB of the children
    //              still running, low: |S_P| + Best of the children finished},
    //              updated with one atomic so that readers see a consistent pair
    int32_t pad[2];
};
static_assert(sizeof(RegEntry) == 64, "registry entry must stay 64 bytes");

// ------------------------------------------------------------------ launch

struct SearchParams {
    QueryDesc *queries;
    int nq;
    int team;                 // threads per worker
    int workers;
    int ncap;                 // degree-array capacity (elements, multiple of 16)
    int wcap;                 // cover-bitmap capacity (words)
    int slot_bytes;           // bytes per node slot
    int stack_depth;          // private slots per worker

    char *stack_slots;        // workers * stack_depth * slot_bytes
    char *wl_slots;           // wl_cap * slot_bytes
    unsigned *wl_seq;         // wl_cap
    int wl_cap;               // power of two
    int wl_low;               // offload when the worklist holds fewer items

    RegEntry *reg;            // reg_cap entries
    uint32_t *reg_words;      // reg_cap * wcap words
    int reg_cap;

    int *comp_scratch;        // workers * 5 * ncap ints (per-component statistics)

    unsigned long long *ctl;  // control block, see Ctl below
    long long node_budget;
    long long idle_timeout_ns;
    int use_components;
    int load_balance;
    int csr_smem;             // >0: the (single) query's induced CSR is staged in shared
                              // memory (this many bytes at the start of each block's region)
    int csr_query;            // the query whose CSR is staged
    long long quantum_ns;     // >0: time slice; each worker stores its node and
                              // exits once this long has passed since it started
    int *stack_top;           // non-null: per-worker private stack depth, read at
                              // start and written at exit (the stacks stay resident
                              // between slices)
    int no_bounds;            // 1: keep the whole degree array as every node's
                              // window (ablation of Section 4.3)
    int breakdown;            // 1: count SM cycles per activity (kPhase*)
    int no_dyn_bounds;        // 1: no dynamic tightening of component bounds (ablation)
    int comp_lp;              // 1: components by label propagation, 0: union-find
    char *wglobal;            // non-null: each worker's node arrays live here (they do
                              // not fit in shared memory), wglobal_stride bytes apart
    long long wglobal_stride;
};

// Control block: one unsigned long long per entry, each entry on its own
// 128-byte line (kCtlStride words apart) so that idle workers polling the
// worklist counter do not serialise with atomics on the other words.
enum Ctl : int {
    kWlCount = 0,     // items reserved in the worklist (never negative)
    kWlHead = 1,      // dequeue ticket
    kWlTail = 2,      // enqueue ticket
    kRegHead = 3,     // registry overflow free-list head {tag:32 | idx:32}
    kRemaining = 4,   // queries not finished
    kAbort = 5,       // nonzero: stop everything
    kStatus = 6,      // first error status (as unsigned of a negative int)
    kProgress = 7,    // progress ticks (for the idle timeout)
    kNodes = 8,       // statistics ...
    kCompBranches = 9,
    kLeaves = 10,
    kPruned = 11,
    kOffloaded = 12,
    kTrivial = 13,
    kMaxStack = 14,
    kErrWhere = 15,   // where the first error was raised (diagnostics)
    kRegBump = 16,    // next never-used registry entry
    kHist = 17,       // kHistBins entries
    kBytes = 33,      // algorithmic bytes moved by the search (slots, CSR rows, bitmaps)
    kWaitIters = 34,  // polls spent waiting for worklist sequence words (diagnostics)
    kPreempts = 35,   // nodes stored at the end of a time slice
    kMaxProcNs = 36,  // longest single process() call (ns, diagnostics)
    kMaxExitNs = 37,  // longest exit phase of a worker (ns, diagnostics)
    kPhase = 38,      // kPhases entries: SM cycles per activity, summed over workers
    kCtlEntries = 44
};
constexpr int kCtlStride = 16;
// activities of the execution-time breakdown
enum Phase : int {
    kPhPop = 0,       // taking a node from the private stack or the worklist
    kPhReduce = 1,    // reduction rules, prune test
    kPhComp = 2,      // finding components, registering a branch on them, closing cliques/cycles
    kPhBranch = 3,    // vertex branch: choosing v_max, storing the right child
    kPhDone = 4,      // completion and aggregation through the registry, new best covers
    kPhIdle = 5,      // waiting for work
    kPhases = 6
};
constexpr int kCtlWords = kCtlEntries * kCtlStride;

__host__ __device__ __forceinline__ unsigned long long &ctlw(unsigned long long *ctl, int e)
{
    return ctl[e * kCtlStride];
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel(int *p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Record the first error (status and a site code) and stop every worker.
__device__ __forceinline__ void set_error(unsigned long long *ctl, int status, int where = 0)
{
    if (atomicCAS(&ctlw(ctl, kStatus), 0ull, (unsigned long long)(unsigned)status) == 0ull)
        ctlw(ctl, kErrWhere) = (unsigned long long)where;
    atomicExch(&ctlw(ctl, kAbort), 1ull);
}

__device__ __forceinline__ bool aborted(unsigned long long *ctl)
{
    return *(volatile unsigned long long *)&ctlw(ctl, kAbort) != 0ull;
}

// ------------------------------------------------------------------ teams
//
// A worker is a "team" of threads that processes one search-tree node at a
// time: one warp (Team<1>) or one thread block (Team<0>, size = blockDim.x).
// Every team-wide operation below must be reached by all threads of the team
// in the same order.
//
// Block teams combine per-warp partials through shared memory with ONE
// barrier per operation: the partials go to one of two buffers, alternating
// from one operation to the next, so a buffer is rewritten only after the
// barrier of the operation in between (which every thread passes after
// reading it).  Each warp then combines the partials itself with its lanes.

// Reduction scratch of a block team: 2 buffers x kRedVals values x 32 warps.
constexpr int kRedVals = 8;
constexpr int kRedInts = 2 * kRedVals * 32;

// What one round of the reduction rules needs from the whole window.
struct WinStats {
    int e2;      // sum of live degrees (2 |E|)
    int live;    // live vertices
    int dmax;    // maximum degree (0: none live)
    int vmax;    // lowest-index vertex of maximum degree (INT_MAX: none)
    int lo, hi;  // live window (INT_MAX / -1: none)
};

__device__ __forceinline__ WinStats warp_stats(const WinStats &t)
{
    WinStats r;
    r.e2 = __reduce_add_sync(kFull, t.e2);
    r.live = __reduce_add_sync(kFull, t.live);
    r.dmax = __reduce_max_sync(kFull, t.dmax);
    r.vmax = __reduce_min_sync(kFull, t.dmax == r.dmax ? t.vmax : INT32_MAX);
    r.lo = __reduce_min_sync(kFull, t.lo);
    r.hi = __reduce_max_sync(kFull, t.hi);
    return r;
}

__device__ __forceinline__ long long warp_lsum(long long x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

template <int WARP_TEAM>
struct Team;

template <>
struct Team<1> {   // one warp per worker
    int rank;      // lane
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool leader() const { return rank == 0; }
    // Each collective starts with __syncwarp(), so that it also orders the
    // lanes' earlier shared-memory accesses (as the block barrier does for
    // block teams).
    __device__ __forceinline__ int sum(int x) { __syncwarp(); return __reduce_add_sync(kFull, x); }
    __device__ __forceinline__ int max(int x) { __syncwarp(); return __reduce_max_sync(kFull, x); }
    __device__ __forceinline__ int min(int x) { __syncwarp(); return __reduce_min_sync(kFull, x); }
    __device__ __forceinline__ long long lsum(long long x) { __syncwarp(); return warp_lsum(x); }
    __device__ __forceinline__ WinStats stats(const WinStats &t) { __syncwarp(); return warp_stats(t); }
    __device__ __forceinline__ int bcast(int x) { __syncwarp(); return __shfl_sync(kFull, x, 0); }
    __device__ __forceinline__ void bcast2(int &a, int &b)
    {
        __syncwarp();
        a = __shfl_sync(kFull, a, 0);
        b = __shfl_sync(kFull, b, 0);
    }
    // exclusive prefix of x over the team; the team total in *tot
    __device__ __forceinline__ int excl_scan(int x, int *tot)
    {
        __syncwarp();
        int inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, inc, o);
            if (rank >= o) inc += y;
        }
        *tot = __shfl_sync(kFull, inc, 31);
        return inc - x;
    }
};

template <>
struct Team<0> {   // one block per worker
    int rank;
    int nthreads;
    int *red;      // kRedInts ints of shared scratch
    int rb;        // buffer of the next operation (uniform over the team)
    __device__ __forceinline__ int size() const { return nthreads; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool leader() const { return rank == 0; }
    __device__ __forceinline__ int lane() const { return rank & 31; }
    __device__ __forceinline__ int warp() const { return rank >> 5; }
    __device__ __forceinline__ int nwarps() const { return (nthreads + 31) >> 5; }
    // the next buffer: value k of warp w at [k * 32 + w]
    __device__ __forceinline__ int *next_buf()
    {
        int *b = red + rb * (kRedVals * 32);
        rb ^= 1;
        return b;
    }
    // lane l of every warp reads value k of warp l (identity beyond the warps)
    __device__ __forceinline__ int part(const int *b, int k, int ident) const
    {
        return lane() < nwarps() ? b[k * 32 + lane()] : ident;
    }
    __device__ __forceinline__ int sum(int x)
    {
        x = __reduce_add_sync(kFull, x);
        int *b = next_buf();
        if (lane() == 0) b[warp()] = x;
        __syncthreads();
        return __reduce_add_sync(kFull, part(b, 0, 0));
    }
    __device__ __forceinline__ int max(int x)
    {
        x = __reduce_max_sync(kFull, x);
        int *b = next_buf();
        if (lane() == 0) b[warp()] = x;
        __syncthreads();
        return __reduce_max_sync(kFull, part(b, 0, INT32_MIN));
    }
    __device__ __forceinline__ int min(int x)
    {
        x = __reduce_min_sync(kFull, x);
        int *b = next_buf();
        if (lane() == 0) b[warp()] = x;
        __syncthreads();
        return __reduce_min_sync(kFull, part(b, 0, INT32_MAX));
    }
    __device__ __forceinline__ long long lsum(long long x)
    {
        x = warp_lsum(x);
        int *b = next_buf();
        if (lane() == 0) {
            b[warp()] = (int)(unsigned)(x & 0xffffffffll);
            b[32 + warp()] = (int)(x >> 32);
        }
        __syncthreads();
        long long y = 0;
        if (lane() < nwarps()) y = ((long long)b[32 + lane()] << 32) | (unsigned)b[lane()];
        return warp_lsum(y);
    }
    __device__ __forceinline__ WinStats stats(const WinStats &t)
    {
        WinStats w = warp_stats(t);
        int *b = next_buf();
        if (lane() == 0) {
            const int i = warp();
            b[i] = w.e2; b[32 + i] = w.live; b[64 + i] = w.dmax;
            b[96 + i] = w.vmax; b[128 + i] = w.lo; b[160 + i] = w.hi;
        }
        __syncthreads();
        WinStats p;
        p.e2 = part(b, 0, 0);
        p.live = part(b, 1, 0);
        p.dmax = part(b, 2, 0);
        p.vmax = part(b, 3, INT32_MAX);
        p.lo = part(b, 4, INT32_MAX);
        p.hi = part(b, 5, -1);
        return warp_stats(p);
    }
    __device__ __forceinline__ int bcast(int x)
    {
        int *b = next_buf();
        if (rank == 0) b[0] = x;
        __syncthreads();
        return b[0];
    }
    __device__ __forceinline__ void bcast2(int &x, int &y)
    {
        int *b = next_buf();
        if (rank == 0) { b[0] = x; b[1] = y; }
        __syncthreads();
        x = b[0];
        y = b[1];
    }
    __device__ __forceinline__ int excl_scan(int x, int *tot)
    {
        int inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, inc, o);
            if (lane() >= o) inc += y;
        }
        int *b = next_buf();
        if (lane() == 31) b[warp()] = inc;
        __syncthreads();
        // inclusive scan of the warp totals, by every warp
        const int y = part(b, 0, 0);
        int s = y;
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(kFull, s, o);
            if (lane() >= o) s += z;
        }
        *tot = __shfl_sync(kFull, s, 31);
        const int before = __shfl_sync(kFull, s - y, warp());   // exclusive offset of this warp
        return before + inc - x;
    }
};

}  // namespace vcg
