// C ABI of the GB300 vertex-cover solver (declared in include/vc_gb300.h).
//
// A solve is three device phases on the handle's stream:
//   1. root_kernel      one block per query: root reduction, greedy bound,
//                       induced subgraph (Section 4.2);
//   2. search_kernel    persistent workers over every query that still needs
//                       a search (Sections 2.3, 3, 4);
//   3. finalize_kernel  one block per query: cover in original ids.
// The host reads the small query descriptors between 1 and 2 to size the
// search (degree dtype, worker shape, capacities) and once at the end.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "vc_internal.h"

using namespace vcg;

namespace {

#define VC_CK(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) {                                     \
            last_cuda_error() = e_;                                  \
            return e_ == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA; \
        }                                                            \
    } while (0)


// Search workspace: node slots, worklist, registry, scratch, control block.
// A CUDA graph of one enqueue sequence, kept with the workspace whose
// buffers its nodes name.  `key` holds every value the captured launches and
// copies were built from (kernels, shapes, arguments, buffer addresses, copy
// sizes); while the key is unchanged the graph is replayed with one launch.
// The data behind the buffers is read when the graph runs, so a replay sees
// the current queries.  A key is captured the second time it comes in a row:
// capture and instantiation cost more than the launches they replace, so
// calls whose shape changes every time (one graph after another of
// different sizes) keep launching directly.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;   // capture or instantiation failed for this key: launch directly
    std::vector<unsigned char> key;   // the key of the graph, or of the last direct launch
    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        failed = false;
        key.clear();
    }
};

struct Workspace {
    DevBuf stack, wl, wl_seq, reg, reg_words, comp_scratch, ctl, root_slot, queries, qscratch, wglobal;
    HostBuf hq, hctl, hcov;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr;   // capture stream (the caller's may be the legacy default stream)
    GraphSlot search_graph;
    GraphSlot root_graph;   // phase 1: descriptor upload, root [+ crown], finalisation, read-back
    int init()
    {
        for (auto &e : ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) return VC_ECUDA;
        return VC_OK;
    }
    void release()
    {
        for (DevBuf *b : {&stack, &wl, &wl_seq, &reg, &reg_words, &comp_scratch, &ctl, &root_slot, &queries,
                          &qscratch, &wglobal})
            b->release();
        hq.release();
        hctl.release();
        hcov.release();
        for (auto &e : ev)
            if (e) { cudaEventDestroy(e); e = nullptr; }
        search_graph.release();
        root_graph.release();
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
    }
};

// Enqueue body(stream, capturing) on s through the graph in gs: replay it
// when `key` matches the captured one; on the second call in a row with a
// key, capture body on the workspace's capture stream, instantiate and
// launch; otherwise (a new key, or capture refused) run body directly on s.
// Returns 2 (replayed), 1 (captured now) or 0 (direct); *err receives the
// CUDA status of the enqueue.
template <class F>
int graph_enqueue(Workspace &ws, GraphSlot &gs, const void *key, size_t kbytes, cudaStream_t s, F body,
                  cudaError_t *err)
{
    const bool same = gs.key.size() == kbytes && memcmp(gs.key.data(), key, kbytes) == 0;
    if (same && gs.exec) {
        *err = cudaGraphLaunch(gs.exec, s);
        return 2;
    }
    if (!same) {   // first call with this key: remember it, launch directly
        gs.release();
        gs.key.assign((const unsigned char *)key, (const unsigned char *)key + kbytes);
    } else if (!gs.failed) {
        if (!ws.cap && cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ws.cap = nullptr;
        }
        cudaGraph_t g = nullptr;
        if (ws.cap && cudaStreamBeginCapture(ws.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t eb = body(ws.cap, true);
            const cudaError_t ee = cudaStreamEndCapture(ws.cap, &g);
            if (eb == cudaSuccess && ee == cudaSuccess && g && cudaGraphInstantiate(&gs.exec, g, 0) == cudaSuccess) {
                cudaGraphDestroy(g);
                *err = cudaGraphLaunch(gs.exec, s);
                return 1;
            }
            if (g) cudaGraphDestroy(g);
            gs.exec = nullptr;
        }
        cudaGetLastError();   // a refused capture leaves no sticky error
        gs.failed = true;
    }
    *err = body(s, false);
    return 0;
}

// Search workspaces are pooled per device and shared by every handle: a solve
// borrows one and gives it back after its final synchronisation, so repeated
// solves (of any graph) allocate nothing once the buffers have grown to size.
// Solves running at the same time (other host threads) get other workspaces.
std::mutex &pool_mutex()
{
    static std::mutex m;
    return m;
}

std::map<int, std::vector<Workspace *>> &pool()
{
    static std::map<int, std::vector<Workspace *>> p;
    return p;
}

struct WsLease {
    int dev;
    cudaStream_t stream;
    Workspace *ws;
    WsLease(int d, cudaStream_t s) : dev(d), stream(s), ws(nullptr)
    {
        std::lock_guard<std::mutex> lk(pool_mutex());
        auto &v = pool()[d];
        if (!v.empty()) {
            ws = v.back();
            v.pop_back();
        }
        if (!ws) ws = new Workspace();
    }
    ~WsLease()
    {
        cudaStreamSynchronize(stream);   // nothing of this solve is still in flight
        std::lock_guard<std::mutex> lk(pool_mutex());
        pool()[dev].push_back(ws);
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Graph buffers come from a per-device cache of power-of-two blocks, so that
// loading and freeing graph handles in a loop allocates nothing after the
// first round (cudaMalloc / cudaFree cost tens of microseconds each and may
// synchronise the device).  vc_trim() returns the idle blocks.
std::map<int, std::multimap<size_t, void *>> &block_cache()
{
    static std::map<int, std::multimap<size_t, void *>> c;
    return c;
}

size_t size_class(size_t b)
{
    size_t s = 256;
    while (s < b) s <<= 1;
    return s;
}

struct CachedBuf {
    void *p = nullptr;
    size_t bytes = 0;   // size class
    int dev = 0;
    int ensure(size_t want)
    {
        if (want <= bytes) return VC_OK;
        release();
        const size_t sc = size_class(want);
        cudaGetDevice(&dev);
        {
            std::lock_guard<std::mutex> lk(pool_mutex());
            auto &m = block_cache()[dev];
            auto it = m.find(sc);
            if (it != m.end()) {
                p = it->second;
                m.erase(it);
                bytes = sc;
                return VC_OK;
            }
        }
        if (cudaMalloc(&p, sc) != cudaSuccess) {
            p = nullptr;
            return VC_ENOMEM;
        }
        bytes = sc;
        return VC_OK;
    }
    void release()
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(pool_mutex());
        block_cache()[dev].emplace(bytes, p);
        p = nullptr;
        bytes = 0;
    }
    template <class X>
    X *as() const { return (X *)p; }
};

// Per-query device scratch of the root phase and the final answer.
size_t query_scratch_bytes(int n, int m2)
{
    const size_t ni = (size_t)(n > 0 ? n : 1);
    return 7 * align256(ni * 4)                   // deg aux fr0 fr1 flag forced_list heavy
           + 2 * align256(ni)                     // st cover_flags
           + align256((ni + 1) * 4)               // rp2
           + align256((size_t)(m2 > 0 ? m2 : 1) * 4)  // col2
           + 2 * align256(ni * 4);                // orig cover_list
}

void carve_query_scratch(QueryDesc &Q, char *base)
{
    const size_t ni = (size_t)(Q.n > 0 ? Q.n : 1);
    char *p = base;
    auto take = [&](size_t b) { char *r = p; p += align256(b); return r; };
    Q.deg = (int *)take(ni * 4);
    Q.aux = (int *)take(ni * 4);
    Q.fr0 = (int *)take(ni * 4);
    Q.fr1 = (int *)take(ni * 4);
    Q.flag = (int *)take(ni * 4);
    Q.forced_list = (int *)take(ni * 4);
    Q.heavy = (int *)take(ni * 4);
    Q.st = (uint8_t *)take(ni);
    Q.cover_flags = (uint8_t *)take(ni);
    Q.rp2 = (int *)take((ni + 1) * 4);
    Q.col2 = (int *)take((size_t)(Q.m2 > 0 ? Q.m2 : 1) * 4);
    Q.orig = (int *)take(ni * 4);
    Q.cover_list = (int *)take(ni * 4);
}

int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

struct vc_graph {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    int n = 0;
    int m2 = 0;
    int maxdeg = 0;
    CachedBuf rp, col, err;
};

namespace {

struct QueryRef {
    vc_graph *g;
    int k;
    int complement = 0;   // output the complement of the cover
};

struct QueryOut {
    int status, size, yes, cover_len;
};

// Everything the search phase's graph is built from (zeroed, then filled
// field by field so that padding compares equal).
struct SearchGraphKey {
    SearchParams P;
    size_t smem;
    int dtype, warp_team, threads, blocks, nq, nroots, wcap;
    const void *root_slot_d, *root_slot_h, *hctl, *hq;
    cudaEvent_t ev2, ev3;
};

// Run a set of queries in one root launch + one persistent search launch.
// covers (nullable) / cover_lens receive the covers.
// The capacities a solve's search ran with, and the search's status.
struct SearchCaps {
    int searched = 0;   // 1: a search ran
    int depth = 0, wl_cap = 0, reg_cap = 0;   // reg_cap without the per-query root entries
    int kstatus = 0;
    int err_where = 0;  // site code of the search's first error
    int workers = 0, slot_bytes = 0, wcap = 0;
    int dev = 0;
    const void *ws = nullptr;   // the workspace the solve borrowed (back in the pool now)
};

int solve_queries(vc_graph *g0, const std::vector<QueryRef> &qs, const vc_options *opt_in,
                  std::vector<QueryOut> &out, int32_t *const *covers, int32_t *cover_lens, vc_stats *stats,
                  SearchCaps *caps = nullptr)
{
    const auto t_start = std::chrono::steady_clock::now();
    vc_options opt;
    vc_options_default(&opt);
    if (opt_in) {
        opt = *opt_in;
        vc_options defaults;
        vc_options_default(&defaults);
        if (opt.idle_timeout_ms <= 0) opt.idle_timeout_ms = defaults.idle_timeout_ms;
    }
    const int nq = (int)qs.size();
    out.assign(nq, QueryOut{VC_OK, -1, 0, 0});
    if (nq == 0) return VC_OK;
    cudaStream_t s = g0->stream;
    WsLease lease(g0->device, s);
    Workspace &ws = *lease.ws;
    if (caps) {
        caps->dev = g0->device;
        caps->ws = lease.ws;
    }
    int rc;
    if ((rc = ws.init()) != VC_OK) return rc;

    // ---- query descriptors + per-query scratch
    size_t scratch = 0;
    std::vector<size_t> offs(nq), croff(nq, 0);
    for (int i = 0; i < nq; i++) {
        offs[i] = scratch;
        scratch += query_scratch_bytes(qs[i].g->n, qs[i].g->m2);
        if (opt.crown) {   // crown workspace: 13 n + 1 + 2|E| ints
            croff[i] = scratch;
            scratch += align256(((size_t)13 * std::max(qs[i].g->n, 1) + 1 + (size_t)std::max(qs[i].g->m2, 1)) * 4);
        }
    }
    if ((rc = ws.qscratch.ensure(scratch)) != VC_OK) return rc;
    if ((rc = ws.queries.ensure(sizeof(QueryDesc) * nq)) != VC_OK) return rc;
    if ((rc = ws.hq.ensure(sizeof(QueryDesc) * nq)) != VC_OK) return rc;
    // covers: finalisation writes each list straight into mapped host memory
    // (room for n entries per query), so no copy or extra synchronisation
    // follows the last kernel
    const bool want_cov = covers != nullptr;
    std::vector<size_t> coff(nq, 0);
    if (want_cov) {
        size_t total = 0;
        for (int i = 0; i < nq; i++) {
            coff[i] = total;
            total += (size_t)std::max(qs[i].g->n, 1);
        }
        if ((rc = ws.hcov.ensure(total * 4, true)) != VC_OK) return rc;
    }
    QueryDesc *hq = (QueryDesc *)ws.hq.p;
    for (int i = 0; i < nq; i++) {
        QueryDesc &Q = hq[i];
        memset(&Q, 0, sizeof(Q));
        Q.n = qs[i].g->n;
        Q.m2 = qs[i].g->m2;
        Q.rp = qs[i].g->rp.as<int>();
        Q.col = qs[i].g->col.as<int>();
        Q.k = qs[i].k;
        Q.maxdeg_in = qs[i].g->maxdeg;
        Q.skip_root_rules = opt.disable_root_rules ? 1 : 0;
        Q.emit_complement = qs[i].complement;
        Q.status = VC_OK;
        carve_query_scratch(Q, ws.qscratch.as<char>() + offs[i]);
        Q.crown_ws = opt.crown ? (int *)(ws.qscratch.as<char>() + croff[i]) : nullptr;
        Q.cover_out = want_cov && covers[i] ? ws.hcov.dev_as<int>() + coff[i] : nullptr;
    }
    QueryDesc *dq = ws.queries.as<QueryDesc>();

    // ---- phase 1: root reduction and induced subgraphs (descriptor upload,
    // root [+ crown] kernel, finalisation of the queries the root phase
    // settled, read-back): one graph launch once this shape has been seen
    int max_n_in = 0, max_deg_in = 0;
    for (int i = 0; i < nq; i++) {
        max_n_in = std::max(max_n_in, qs[i].g->n);
        max_deg_in = std::max(max_deg_in, qs[i].g->maxdeg);
    }
    auto phase1 = [&](cudaStream_t st, bool capturing) -> cudaError_t {
        const unsigned fl = capturing ? cudaEventRecordExternal : 0u;
        cudaError_t e = cudaMemcpyAsync(dq, hq, sizeof(QueryDesc) * nq, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ws.ev[0], st, fl);
        if (e == cudaSuccess) e = root_run(dq, nq, max_n_in, max_deg_in, st);
        if (e == cudaSuccess && opt.crown) e = crown_run(dq, nq, st);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ws.ev[1], st, fl);
        if (e == cudaSuccess) e = finalize_run(dq, nq, nullptr, nullptr, 0, st, 1);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hq, dq, sizeof(QueryDesc) * nq, cudaMemcpyDeviceToHost, st);
        return e;
    };
    {
        cudaError_t e = cudaSuccess;
        if (opt.cuda_graph) {
            struct {
                QueryDesc *dq, *hq;
                int nq, max_n, max_deg, crown;
                cudaEvent_t ev0, ev1;
            } key;
            memset(&key, 0, sizeof(key));
            key.dq = dq;
            key.hq = hq;
            key.nq = nq;
            key.max_n = max_n_in;
            // the root launches depend on the maximum degree only through
            // this threshold (block kernel state and cluster eligibility), so
            // graphs of one size share the captured phase
            key.max_deg = max_deg_in > 65535 ? 1 : 0;
            key.crown = opt.crown ? 1 : 0;
            key.ev0 = ws.ev[0];
            key.ev1 = ws.ev[1];
            graph_enqueue(ws, ws.root_graph, &key, sizeof(key), s, phase1, &e);
        } else {
            e = phase1(s, false);
        }
        VC_CK(e);
    }
    VC_CK(cudaStreamSynchronize(s));

    int max_np = 0, max_deg = 0, nroots = 0;
    std::vector<int> root_slot(nq, -1);
    for (int i = 0; i < nq; i++) {
        const QueryDesc &Q = hq[i];
        if (Q.status != VC_OK || Q.answered || Q.np == 0) continue;
        root_slot[i] = nroots++;
        max_np = std::max(max_np, Q.np);
        max_deg = std::max(max_deg, Q.maxdeg);
    }

    float ms_search = 0.f;
    SearchPlan pl{};
    SearchParams P;
    memset(&P, 0, sizeof(P));   // zero padding: P is compared byte by byte as part of a graph key
    int graph_state = 0;
    unsigned long long hctl_local[kCtlWords] = {};
    if (nroots > 0) {
        // ---- phase 2: size and run the persistent search
        int dtype = opt.dtype_bytes;
        const int need = max_deg <= 255 ? 1 : (max_deg <= 65535 ? 2 : 4);
        if (dtype != 1 && dtype != 2 && dtype != 4) dtype = need;
        if (dtype < need) dtype = need;
        const int ncap = (max_np + 16 + 15) / 16 * 16;
        const int wcap = max_np / 32 + 2;
        // one searched query with a small induced graph: stage its CSR in
        // shared memory (up to 48 KB, and only when it still leaves room)
        int csr_bytes = 0, csr_query = 0;
        if (nroots == 1) {
            int qi = 0;
            while (root_slot[qi] < 0) qi++;
            csr_query = qi;
            const long long b = 4ll * (hq[qi].np + 1 + hq[qi].m2p);
            if (b <= 48 * 1024) csr_bytes = (int)((b + 15) / 16 * 16);
        }
        rc = search_plan(dtype, opt.team, ncap, wcap, g0->sms, csr_bytes, &pl);
        if (rc == VC_ECAPACITY && csr_bytes > 0) rc = search_plan(dtype, opt.team, ncap, wcap, g0->sms, 0, &pl);
        if (rc != VC_OK) {
            if (rc == VC_ECUDA) last_cuda_error() = cudaGetLastError();
            return rc;
        }
        int depth = opt.stack_depth > 0 ? opt.stack_depth : std::min(max_np + 2, 4096);
        // keep the private stacks within ~24 GB of HBM
        const size_t stack_budget = (size_t)24 << 30;
        const size_t per_worker_slot = (size_t)pl.workers * pl.slot_bytes;
        if ((size_t)depth * per_worker_slot > stack_budget)
            depth = (int)std::max<size_t>(8, stack_budget / per_worker_slot);
        int wl_cap = opt.worklist_capacity > 0 ? next_pow2(opt.worklist_capacity)
                                               : next_pow2(std::max(4 * pl.workers, 1024));
        wl_cap = std::max(wl_cap, next_pow2(nroots));
        // registry entries are bump-allocated (nothing to initialise), so a
        // large capacity only costs address space: up to ~8 GB or 4M entries
        int reg_cap = opt.registry_capacity;
        if (reg_cap <= 0) {
            const size_t per_entry = sizeof(RegEntry) + (size_t)wcap * 4;
            reg_cap = (int)std::min<size_t>((size_t)4 << 20, ((size_t)8 << 30) / per_entry);
            reg_cap = std::max(reg_cap, 64 * pl.workers);
        }
        if (caps) {
            caps->searched = 1;
            caps->depth = depth;
            caps->wl_cap = wl_cap;
            caps->reg_cap = reg_cap;
            caps->workers = pl.workers;
            caps->slot_bytes = pl.slot_bytes;
            caps->wcap = wcap;
        }
        reg_cap += nq;

        if ((rc = ws.stack.ensure((size_t)pl.workers * depth * pl.slot_bytes)) != VC_OK) return rc;
        if ((rc = ws.wl.ensure((size_t)wl_cap * pl.slot_bytes)) != VC_OK) return rc;
        if ((rc = ws.wl_seq.ensure((size_t)wl_cap * 4)) != VC_OK) return rc;
        if ((rc = ws.reg.ensure((size_t)reg_cap * sizeof(RegEntry))) != VC_OK) return rc;
        if ((rc = ws.reg_words.ensure((size_t)reg_cap * wcap * 4)) != VC_OK) return rc;
        if ((rc = ws.comp_scratch.ensure((size_t)pl.workers * 5 * ncap * 4)) != VC_OK) return rc;
        if (pl.wglobal_bytes > 0 && (rc = ws.wglobal.ensure((size_t)pl.workers * (size_t)pl.wglobal_bytes)) != VC_OK)
            return rc;
        if ((rc = ws.ctl.ensure(kCtlWords * 8)) != VC_OK) return rc;
        if ((rc = ws.root_slot.ensure((size_t)nq * 4)) != VC_OK) return rc;
        if ((rc = ws.hctl.ensure(kCtlWords * 8 + (size_t)nq * 4)) != VC_OK) return rc;
        int *h_root_slot = (int *)((char *)ws.hctl.p + kCtlWords * 8);
        memcpy(h_root_slot, root_slot.data(), (size_t)nq * 4);
        P.queries = dq;
        P.nq = nq;
        P.team = pl.warp_team ? 32 : pl.threads;
        P.workers = pl.workers;
        P.ncap = ncap;
        P.wcap = wcap;
        P.slot_bytes = pl.slot_bytes;
        P.stack_depth = depth;
        P.stack_slots = ws.stack.as<char>();
        P.wl_slots = ws.wl.as<char>();
        P.wl_seq = ws.wl_seq.as<unsigned>();
        P.wl_cap = wl_cap;
        // default hunger threshold: four items per worker, at most half the
        // ring (component-heavy 8 x 48 with 1,216 workers: 52.0M nodes/s at
        // workers / 2, 55.5M at 4,096)
        P.wl_low = !opt.load_balance ? 0
                   : (opt.offload_below > 0 ? opt.offload_below : std::max(8, std::min(wl_cap / 2, 4 * pl.workers)));
        P.reg = ws.reg.as<RegEntry>();
        P.reg_words = ws.reg_words.as<uint32_t>();
        P.reg_cap = reg_cap;
        P.comp_scratch = ws.comp_scratch.as<int>();
        P.ctl = ws.ctl.as<unsigned long long>();
        P.node_budget = opt.node_budget;
        P.idle_timeout_ns = (long long)opt.idle_timeout_ms * 1000000ll;
        P.use_components = opt.use_components;
        P.load_balance = opt.load_balance;
        P.csr_smem = pl.csr_bytes;
        P.csr_query = csr_query;
        P.no_bounds = opt.disable_bounds ? 1 : 0;
        P.breakdown = opt.breakdown ? 1 : 0;
        P.no_dyn_bounds = opt.disable_dyn_bounds ? 1 : 0;
        P.comp_lp = opt.label_propagation ? 1 : 0;
        P.wglobal = pl.wglobal_bytes > 0 ? ws.wglobal.as<char>() : nullptr;
        P.wglobal_stride = pl.wglobal_bytes;
        // upload of the root slots, search, finalisation and read-back: one
        // graph launch once this launch shape has been seen
        auto enqueue = [&](cudaStream_t st, bool capturing) -> cudaError_t {
            cudaError_t e = cudaMemcpyAsync(ws.root_slot.p, h_root_slot, (size_t)nq * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = search_run(pl, P, ws.root_slot.as<int>(), nq, nroots, st, ws.ev[2], ws.ev[3],
                               capturing ? cudaEventRecordExternal : 0u);
            if (e == cudaSuccess) e = finalize_run(dq, nq, P.reg, P.reg_words, wcap, st, 2);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ws.hctl.p, P.ctl, kCtlWords * 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hq, dq, sizeof(QueryDesc) * nq, cudaMemcpyDeviceToHost, st);
            return e;
        };
        cudaError_t e = cudaSuccess;
        if (opt.cuda_graph) {
            SearchGraphKey key;
            memset(&key, 0, sizeof(key));
            memcpy(&key.P, &P, sizeof(P));
            key.dtype = pl.dtype;
            key.warp_team = pl.warp_team;
            key.threads = pl.threads;
            key.blocks = pl.blocks;
            key.smem = pl.smem;
            key.nq = nq;
            key.nroots = nroots;
            key.wcap = wcap;
            key.root_slot_d = ws.root_slot.p;
            key.root_slot_h = h_root_slot;
            key.hctl = ws.hctl.p;
            key.hq = hq;
            key.ev2 = ws.ev[2];
            key.ev3 = ws.ev[3];
            graph_state = graph_enqueue(ws, ws.search_graph, &key, sizeof(key), s, enqueue, &e);
        } else {
            e = enqueue(s, false);
        }
        VC_CK(e);
        VC_CK(cudaStreamSynchronize(s));
        memcpy(hctl_local, ws.hctl.p, kCtlWords * 8);
        VC_CK(cudaEventElapsedTime(&ms_search, ws.ev[2], ws.ev[3]));
    }
    float ms_root = 0.f;
    VC_CK(cudaEventElapsedTime(&ms_root, ws.ev[0], ws.ev[1]));

    const int kstatus = (int)(int64_t)ctlw(hctl_local, kStatus);
    if (caps) {
        caps->kstatus = kstatus;
        caps->err_where = (int)ctlw(hctl_local, kErrWhere);
    }
    if (want_cov && kstatus == 0) {
        const int32_t *hc = (const int32_t *)ws.hcov.p;
        for (int i = 0; i < nq; i++)
            if (covers[i] && hq[i].status == VC_OK && hq[i].cover_len > 0)
                memcpy(covers[i], hc + coff[i], (size_t)std::min(hq[i].cover_len, std::max(hq[i].n, 1)) * 4);
    }
    for (int i = 0; i < nq; i++) {
        QueryOut &o = out[i];
        const QueryDesc &Q = hq[i];
        o.status = Q.status != VC_OK ? Q.status : (root_slot[i] >= 0 && kstatus ? kstatus : VC_OK);
        if (o.status != VC_OK) { o.size = -1; o.yes = 0; }
        o.size = Q.result;
        o.yes = Q.yes;
        o.cover_len = (o.status == VC_OK) ? Q.cover_len : 0;
        if (cover_lens) cover_lens[i] = o.cover_len;
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->nodes = (int64_t)ctlw(hctl_local, kNodes);
        stats->search_bytes = (int64_t)ctlw(hctl_local, kBytes);
        for (int k = 0; k < kPhases; k++) stats->phase_cycles[k] = (int64_t)ctlw(hctl_local, kPhase + k);
        stats->component_branches = (int64_t)ctlw(hctl_local, kCompBranches);
        stats->leaves = (int64_t)ctlw(hctl_local, kLeaves);
        stats->pruned = (int64_t)ctlw(hctl_local, kPruned);
        stats->offloaded = (int64_t)ctlw(hctl_local, kOffloaded);
        stats->trivial_components = (int64_t)ctlw(hctl_local, kTrivial);
        for (int b = 0; b < 16 && b < kHistBins; b++) stats->comp_hist[b] = (int64_t)ctlw(hctl_local, kHist + b);
        for (int i = 0; i < nq; i++) {
            stats->root_rounds += hq[i].rounds;
            for (int c = 0; c < 4; c++) stats->root_cycles[c] += hq[i].root_cycles[c];
            stats->n += hq[i].n;
            stats->n_induced += hq[i].np;
            stats->m_induced += hq[i].m2p / 2;
            stats->forced += hq[i].forced;
            stats->greedy_size += hq[i].greedy;
            stats->crown_forced += hq[i].crown_forced;
            stats->crown_removed += hq[i].crown_removed;
            stats->crown_skipped += hq[i].crown_status < 0;
        }
        stats->dtype_bytes = nroots ? pl.dtype : 0;
        stats->team = nroots ? (pl.warp_team ? 32 : pl.threads) : 0;
        stats->workers = nroots ? pl.workers : 0;
        stats->max_stack = (int32_t)ctlw(hctl_local, kMaxStack);
        stats->err_where = (int32_t)ctlw(hctl_local, kErrWhere);
        // root [+ crown] [+ init, roots, publish, search] + finalize
        stats->launches = (nroots > 0 ? 6 : 2) + (opt.crown ? 1 : 0);
        stats->cuda_graph = graph_state;
        for (int i = 0; i < nq; i++) {
            const QueryDesc &Q = hq[i];
            const int st_i = Q.status != VC_OK ? Q.status : (root_slot[i] >= 0 && kstatus ? kstatus : VC_OK);
            if (st_i == VC_OK) stats->best_found += Q.k < 0 ? Q.result : (Q.yes ? Q.result : Q.k + 1);
            else if (st_i == VC_EBUDGET && root_slot[i] >= 0) stats->best_found += Q.best;
        }
        stats->ms_root = ms_root;
        stats->ms_search = ms_search;
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    return kstatus ? kstatus : VC_OK;
}

int load_common(int32_t n, const int32_t *rp, const int32_t *col, bool device_ptrs, void *stream,
                vc_graph **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    if (n < 0 || (n > 0 && !rp)) return VC_EINVAL;
    vc_graph *g = new vc_graph();
    g->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        delete g;
        return VC_ECUDA;
    }
    int m2 = 0;
    if (n > 0) {
        if (device_ptrs) {
            if (cudaMemcpy(&m2, rp + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                delete g;
                return VC_ECUDA;
            }
        } else {
            m2 = rp[n];
        }
    }
    if (m2 < 0 || (m2 > 0 && !col) || (m2 & 1)) { delete g; return VC_EINVAL; }
    g->n = n;
    g->m2 = m2;
    int rc;
    if ((rc = g->rp.ensure((size_t)(n + 1) * 4)) != VC_OK || (rc = g->col.ensure((size_t)std::max(m2, 1) * 4)) != VC_OK ||
        (rc = g->err.ensure(16))) {
        vc_free(g);
        return rc;
    }
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t s = g->stream;
    bool ok = true;
    if (n > 0) {
        ok = ok && cudaMemcpyAsync(g->rp.p, rp, (size_t)(n + 1) * 4, kind, s) == cudaSuccess;
        if (m2 > 0) ok = ok && cudaMemcpyAsync(g->col.p, col, (size_t)m2 * 4, kind, s) == cudaSuccess;
    } else {
        ok = ok && cudaMemsetAsync(g->rp.p, 0, 4, s) == cudaSuccess;
    }
    int herr[3] = {0, 0, 0};
    if (ok && n > 0) {
        ok = validate_run(n, m2, g->rp.as<int>(), g->col.as<int>(), g->err.as<int>(), s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(herr, g->err.p, 12, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) { vc_free(g); return VC_ECUDA; }
    if (herr[0] != 0 || (long long)herr[1] * 2 != m2) { vc_free(g); return VC_EINVAL; }
    g->maxdeg = herr[2];
    *out = g;
    return VC_OK;
}

}  // namespace

extern "C" {

int vc_options_default(vc_options *opt)
{
    if (!opt) return VC_EINVAL;
    memset(opt, 0, sizeof(*opt));
    opt->use_components = 1;
    opt->load_balance = 1;
    opt->idle_timeout_ms = 60000;
    opt->cuda_graph = 1;
    opt->capacity_retries = 2;
    return VC_OK;
}

int vc_load_csr(int32_t n, const int32_t *row_ptr, const int32_t *col, void *cuda_stream, vc_graph **out)
{
    return load_common(n, row_ptr, col, false, cuda_stream, out);
}

int vc_load_csr_device(int32_t n, const int32_t *d_row_ptr, const int32_t *d_col, void *cuda_stream,
                       vc_graph **out)
{
    return load_common(n, d_row_ptr, d_col, true, cuda_stream, out);
}

namespace {

// Growth ceilings of capacity retries, in bytes: the private stacks keep the
// 24 GB clamp of solve_queries; the worklist and the registry stop at these.
constexpr size_t kRetryWorklistBytes = (size_t)8 << 30;
constexpr size_t kRetryRegistryBytes = (size_t)16 << 30;

// Drop a workspace that a retried solve grew (it is idle in the pool again
// unless another solve borrowed it meanwhile), so that its enlarged buffers
// go back to the device instead of staying cached.
void drop_workspace(int dev, const void *w)
{
    std::lock_guard<std::mutex> lk(pool_mutex());
    auto &v = pool()[dev];
    for (size_t i = 0; i < v.size(); i++) {
        if (v[i] != w) continue;
        Workspace *x = v[i];
        v.erase(v.begin() + (long)i);
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != dev) cudaSetDevice(dev);
        x->release();
        delete x;
        if (cur != dev) cudaSetDevice(cur);
        return;
    }
}

// solve_queries, repeated while the search ran out of capacity, up to
// opt.capacity_retries times.  Only the resource the kernel reported as
// exhausted grows (doubled): node slots (site 5: private stack and worklist
// both full) grow the stack depth and the worklist; registry exhaustion
// (sites 7, 8) grows the registry; another site grows all three.  Growth
// stops at the ceilings above; a retry that could grow nothing is not made.
// After a retried solve its grown workspace is freed.  stats->retries counts
// the repeats.
int solve_with_retries(vc_graph *g0, const std::vector<QueryRef> &qs, const vc_options *opt_in,
                       std::vector<QueryOut> &out, int32_t *const *covers, int32_t *cover_lens, vc_stats *stats)
{
    vc_options o;
    if (opt_in) o = *opt_in;
    else vc_options_default(&o);
    int rc = VC_OK;
    int attempt = 0;
    SearchCaps c;
    for (;; attempt++) {
        c = SearchCaps();
        rc = solve_queries(g0, qs, &o, out, covers, cover_lens, stats, &c);
        if (stats) stats->retries = attempt;
        // (solve_queries returns the search's status, so rc is VC_ECAPACITY here too)
        const bool out_of_capacity = c.searched && c.kstatus == VC_ECAPACITY;
        if (!out_of_capacity || attempt >= o.capacity_retries) break;
        const bool slots = c.err_where == 5, regs = c.err_where == 7 || c.err_where == 8;
        const bool all = !slots && !regs;
        const auto twice = [](int x) { return x > (1 << 29) ? (1 << 30) : 2 * std::max(x, 1); };
        bool grew = false;
        if (slots || all) {
            o.stack_depth = twice(c.depth);   // clamped to 24 GB by solve_queries
            grew |= (size_t)o.stack_depth * c.workers * c.slot_bytes <= ((size_t)24 << 30);
            const int w = twice(c.wl_cap);
            if ((size_t)w * c.slot_bytes <= kRetryWorklistBytes) { o.worklist_capacity = w; grew = true; }
        }
        if (regs || all) {
            const int r = twice(c.reg_cap);
            if ((size_t)r * (sizeof(RegEntry) + 4ull * c.wcap) <= kRetryRegistryBytes) {
                o.registry_capacity = r;
                grew = true;
            }
        }
        if (!grew) break;
    }
    if (attempt > 0 && c.ws) drop_workspace(c.dev, c.ws);
    return rc;
}

}  // namespace

int vc_solve_min(vc_graph *g, const vc_options *opt, int32_t *cover_size, int32_t *cover, int32_t *cover_len,
                 vc_stats *stats)
{
    if (!g || !cover_size) return VC_EINVAL;
    std::vector<QueryRef> qs{{g, -1}};
    std::vector<QueryOut> out;
    int32_t *covers[1] = {cover};
    int32_t len = 0;
    int rc = solve_with_retries(g, qs, opt, out, cover ? covers : nullptr, &len, stats);
    if (rc != VC_OK) return rc;
    if (out[0].status != VC_OK) return out[0].status;
    *cover_size = out[0].size;
    if (cover_len) *cover_len = len;
    return VC_OK;
}

int vc_autotune(int32_t count, vc_graph *const *graphs, const int32_t *ks, const vc_options *base,
                int32_t repeats, vc_options *best, double *best_ms, vc_options *tried, double *tried_ms,
                int32_t max_trials, int32_t *trials)
{
    if (count <= 0 || !graphs || !best || !best_ms) return VC_EINVAL;
    for (int i = 0; i < count; i++)
        if (!graphs[i]) return VC_EINVAL;
    if (repeats < 1) repeats = 1;
    vc_options cur;
    if (base) cur = *base;
    else vc_options_default(&cur);
    std::vector<QueryRef> qs(count);
    for (int i = 0; i < count; i++) qs[i] = QueryRef{graphs[i], ks ? ks[i] : -1};
    int ntried = 0;
    std::vector<QueryOut> out;
    // best wall time of `repeats` runs of the whole batch; < 0: failed
    auto score = [&](const vc_options &o) -> double {
        double b = -1.0;
        for (int r = 0; r < repeats; r++) {
            vc_stats st;
            const int rc = solve_queries(graphs[0], qs, &o, out, nullptr, nullptr, &st);
            if (rc != VC_OK) return -1.0;
            for (const QueryOut &q : out)
                if (q.status != VC_OK && q.status != VC_EBUDGET) return -1.0;
            if (b < 0 || st.ms_total < b) b = st.ms_total;
        }
        if (tried && ntried < max_trials) tried[ntried] = o;
        if (tried_ms && ntried < max_trials) tried_ms[ntried] = b;
        ntried++;
        return b;
    };
    double bms = score(cur);
    if (bms < 0) return VC_EINVAL;   // the starting point itself fails
    auto stage = [&](auto apply, std::initializer_list<int> values) {
        vc_options keep = cur;
        for (int v : values) {
            vc_options o = keep;
            apply(o, v);
            if (memcmp(&o, &keep, sizeof(o)) == 0) continue;
            const double t = score(o);
            if (t >= 0 && t < bms) { bms = t; cur = o; }
        }
    };
    stage([](vc_options &o, int v) { o.team = v; }, {32, 64, 128, 256, 512});
    stage([](vc_options &o, int v) { o.dtype_bytes = v; }, {1, 2, 4});
    stage([](vc_options &o, int v) { o.offload_below = v; }, {64, 256, 1024, 4096});
    stage([](vc_options &o, int v) { o.stack_depth = v; }, {32, 256});
    stage([](vc_options &o, int v) { o.worklist_capacity = v; }, {1 << 14, 1 << 16});
    *best = cur;
    *best_ms = bms;
    if (trials) *trials = ntried;
    return VC_OK;
}

int vc_solve_mis(vc_graph *g, const vc_options *opt, int32_t *set_size, int32_t *set, int32_t *set_len,
                 vc_stats *stats)
{
    if (!g || !set_size) return VC_EINVAL;
    std::vector<QueryRef> qs{{g, -1, 1}};
    std::vector<QueryOut> out;
    int32_t *sets[1] = {set};
    int32_t len = 0;
    int rc = solve_with_retries(g, qs, opt, out, set ? sets : nullptr, &len, stats);
    if (rc != VC_OK) return rc;
    if (out[0].status != VC_OK) return out[0].status;
    *set_size = g->n - out[0].size;
    if (set_len) *set_len = len;
    return VC_OK;
}

int vc_solve_k(vc_graph *g, int32_t k, const vc_options *opt, int32_t *is_yes, int32_t *cover, int32_t *cover_len,
               vc_stats *stats)
{
    if (!g || !is_yes || k < 0) return VC_EINVAL;
    std::vector<QueryRef> qs{{g, k}};
    std::vector<QueryOut> out;
    int32_t *covers[1] = {cover};
    int32_t len = 0;
    int rc = solve_with_retries(g, qs, opt, out, cover ? covers : nullptr, &len, stats);
    if (rc != VC_OK) return rc;
    if (out[0].status != VC_OK) return out[0].status;
    *is_yes = out[0].yes;
    if (cover_len) *cover_len = out[0].yes ? len : 0;
    return VC_OK;
}

int vc_solve_batch(int32_t count, vc_graph *const *graphs, const int32_t *ks, const vc_options *opt,
                   int32_t *out_size, int32_t *out_yes, int32_t *out_status, int32_t *const *covers,
                   int32_t *cover_lens, vc_stats *stats)
{
    if (count < 0 || (count > 0 && !graphs)) return VC_EINVAL;
    if (count == 0) return VC_OK;
    std::vector<QueryRef> qs(count);
    for (int i = 0; i < count; i++) {
        if (!graphs[i]) return VC_EINVAL;
        qs[i] = {graphs[i], ks && ks[i] >= 0 ? ks[i] : -1};
    }
    std::vector<QueryOut> out;
    int rc = solve_with_retries(graphs[0], qs, opt, out, covers, cover_lens, stats);
    for (int i = 0; i < count; i++) {
        if (out_size) out_size[i] = out.empty() ? -1 : out[i].size;
        if (out_yes) out_yes[i] = out.empty() ? 0 : out[i].yes;
        if (out_status) out_status[i] = out.empty() ? rc : out[i].status;
    }
    return rc;
}

void vc_free(vc_graph *g)
{
    if (!g) return;
    g->rp.release();
    g->col.release();
    g->err.release();
    delete g;
}

int vc_trim(void)
{
    std::lock_guard<std::mutex> lk(pool_mutex());
    int n = 0;
    int cur = 0;
    if (!pool().empty() || !block_cache().empty()) cudaGetDevice(&cur);
    for (auto &kv : pool()) {
        cudaSetDevice(kv.first);
        for (Workspace *w : kv.second) {
            w->release();
            delete w;
            n++;
        }
        kv.second.clear();
    }
    for (auto &kv : block_cache()) {
        cudaSetDevice(kv.first);
        for (auto &b : kv.second) cudaFree(b.second);
        kv.second.clear();
    }
    if (n || !block_cache().empty()) cudaSetDevice(cur);
    return n;
}

const char *vc_last_cuda_error(void)
{
    return cudaGetErrorString(last_cuda_error());
}

const char *vc_strerror(int status)
{
    switch (status) {
    case VC_OK: return "ok";
    case VC_EINVAL: return "invalid argument or malformed CSR graph";
    case VC_ENOMEM: return "device or pinned host allocation failed";
    case VC_ECAPACITY: return "stack, worklist, registry or shared memory capacity exceeded";
    case VC_ETIMEOUT: return "a bounded device wait expired without progress";
    case VC_ECUDA: return "CUDA runtime error";
    case VC_EBUDGET: return "search-tree node budget exhausted";
    default: return "unknown status";
    }
}

}  // extern "C"
