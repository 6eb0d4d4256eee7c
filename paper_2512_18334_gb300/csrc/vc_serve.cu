// Served requests with continuous batching (declared in include/vc_gb300.h).
//
// The search state of the persistent kernel -- node slots (private stacks and
// the shared worklist), the component-branch registry with its witness
// bitmaps, the control block and each worker's stack depth -- stays resident
// in device memory for the life of the server.  A step is
//   admit:  one host-to-device copy of the admitted requests (descriptors,
//           slot indices, packed CSRs), device validation, the root phase
//           (Section 4.2) and the placement of each root node into the live
//           worklist;
//   slice:  the search kernel for one time slice over every request in
//           flight; at the deadline each worker stores its node and exits;
//   retire: finished requests are finalised on the device, their answers and
//           covers written to mapped host memory; one stream synchronisation.
// A request's input CSR and root-phase scratch live only in the per-step
// admission buffer; what the search and the final answer read (induced CSR,
// id map, state and cover arrays) lives in the arena until it retires.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "vc_internal.h"

using namespace vcg;

namespace {

#define SV_CK(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) {                                     \
            last_cuda_error() = e_;                                  \
            return e_ == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA; \
        }                                                            \
    } while (0)

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes a request holds while in flight: st, cover flags, induced CSR,
// id map, cover list.
size_t resident_bytes(int n, int m2)
{
    const size_t ni = (size_t)(n > 0 ? n : 1);
    return 2 * a256(ni) + a256((ni + 1) * 4) + a256((size_t)std::max(m2, 1) * 4) + 2 * a256(ni * 4);
}

// Device bytes of its root-phase scratch (admission buffer only).
size_t root_scratch_bytes(int n)
{
    const size_t ni = (size_t)(n > 0 ? n : 1);
    return 7 * a256(ni * 4);
}

// Input CSR bytes in the packed upload (16-byte aligned pieces).
size_t csr_bytes(int n, int m2)
{
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    return a16((size_t)(n + 1) * 4) + a16((size_t)std::max(m2, 1) * 4);
}

// First-fit allocator over [0, cap) with coalescing (offsets and sizes are
// multiples of 256 bytes).
struct Arena {
    size_t cap = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    void init(size_t c)
    {
        cap = c;
        free_.clear();
        if (c) free_[0] = c;
    }
    long long alloc(size_t b)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < b) continue;
            const size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > b) free_[off + b] = sz - b;
            return (long long)off;
        }
        return -1;
    }
    void release(size_t off, size_t b)
    {
        auto it = free_.emplace(off, b).first;
        auto nx = std::next(it);
        if (nx != free_.end() && off + b == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Request {
    int64_t tag;
    int n, m2, k, maxdeg;
    std::vector<int32_t> csr;   // row_ptr[n + 1] then col[m2]
    double t_submit;
};

struct Slot {
    bool busy = false;
    int lane = 0;          // size class holding the request (known after its first step)
    int gen = 0;
    int64_t tag = 0;
    int n = 0;
    double t_submit = 0, t_admit = 0;
    size_t off = 0, bytes = 0;
};

struct Done {
    vc_server_result r;
    std::vector<int32_t> cover;
};

}  // namespace

// One size class: a resident search of its own, for induced graphs of more
// than the previous class's capacity and at most max_np vertices.
struct Lane {
    int max_np = 0, min_np = 0;
    SearchPlan pl{};
    SearchParams P{};
    int ncap = 0, wcap = 0;
    DevBuf stack, wl, wl_seq, reg, reg_words, comp_scratch, ctl, stack_top, wglobal;
    HostBuf m_ctl;                               // mapped: control words after a step
    unsigned long long snap[kCtlEntries] = {};   // control words after the last step
    long long base_nodes = 0, base_bytes = 0;    // counters accumulated before resets
    long long base_waits = 0, base_preempts = 0;
    bool dirty = false;                          // resident state holds work of earlier requests
    void release()
    {
        for (DevBuf *b : {&stack, &wl, &wl_seq, &reg, &reg_words, &comp_scratch, &ctl, &stack_top, &wglobal})
            b->release();
        m_ctl.release();
    }
};
constexpr int kMaxLanes = 2;

struct vc_server {
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;
    vc_server_config cfg{};
    Lane lane[kMaxLanes];
    int nlanes = 0;
    DevBuf slots, admit, arena, cover_ctr;
    HostBuf h_up;                   // pinned: the packed admission upload
    HostBuf m_rec, m_cover, m_act;  // mapped: retire records, covers, active slots
    cudaEvent_t ev[6] = {};
    std::deque<Request> queue;
    std::vector<Slot> slot;
    std::vector<int> free_slots;
    std::vector<int> active;
    Arena arena_alloc;
    std::deque<Done> ready;
    vc_server_stats st{};
    std::chrono::steady_clock::time_point t0;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    void release()
    {
        for (Lane &L : lane) L.release();
        for (DevBuf *b : {&slots, &admit, &arena, &cover_ctr}) b->release();
        for (HostBuf *b : {&h_up, &m_rec, &m_cover, &m_act}) b->release();
        for (auto &e : ev)
            if (e) { cudaEventDestroy(e); e = nullptr; }
    }
};

namespace {

// Empty a class's resident search state (worklist, counters, registry
// allocator, stack depths); registry entries [0, max_inflight) stay reserved
// as the slots' root entries.
int reset_state(vc_server *s, Lane &L)
{
    L.base_nodes += (long long)L.snap[kNodes];
    L.base_bytes += (long long)L.snap[kBytes];
    L.base_waits += (long long)L.snap[kWaitIters];
    L.base_preempts += (long long)L.snap[kPreempts];
    SV_CK(search_reset_run(L.P, s->cfg.max_inflight, s->stream));
    SV_CK(cudaMemsetAsync(L.stack_top.p, 0, L.stack_top.bytes, s->stream));
    memset(L.snap, 0, sizeof(L.snap));
    L.dirty = false;
    s->st.resets++;
    return VC_OK;
}

void finish_slot(vc_server *s, int qi, const vc_server_result &r, const int32_t *cover)
{
    Slot &sl = s->slot[qi];
    Done d;
    d.r = r;
    d.r.tag = sl.tag;
    d.r.n = sl.n;
    d.r.t_submit_ms = sl.t_submit;
    d.r.t_admit_ms = sl.t_admit;
    d.r.t_done_ms = s->now_ms();
    if (cover && r.cover_len > 0) d.cover.assign(cover, cover + r.cover_len);
    s->ready.push_back(std::move(d));
    s->arena_alloc.release(sl.off, sl.bytes);
    sl.busy = false;
    s->free_slots.push_back(qi);
    s->st.completed++;
}

int admit(vc_server *s, int *n_admitted)
{
    *n_admitted = 0;
    if (s->queue.empty() || s->free_slots.empty()) return VC_OK;
    // worklist room: one root node per admitted request, half the ring at
    // most (in every class: which class takes a request is known only after
    // its root phase)
    long long room = LLONG_MAX;
    for (int l = 0; l < s->nlanes; l++)
        room = std::min(room, (long long)s->lane[l].P.wl_cap / 2 - (long long)s->lane[l].snap[kWlCount]);
    std::vector<Request> adm;
    std::vector<int> qidx;
    std::vector<long long> aoff;
    while (!s->queue.empty() && !s->free_slots.empty() && (long long)adm.size() < room) {
        Request &r = s->queue.front();
        const size_t rb = a256(resident_bytes(r.n, r.m2));
        const long long off = s->arena_alloc.alloc(rb);
        if (off < 0) break;   // admission by device memory: wait for retirements
        const int qi = s->free_slots.back();
        s->free_slots.pop_back();
        Slot &sl = s->slot[qi];
        sl.busy = true;
        sl.lane = 0;
        sl.gen++;
        sl.tag = r.tag;
        sl.n = r.n;
        sl.t_submit = r.t_submit;
        sl.t_admit = s->now_ms();
        sl.off = (size_t)off;
        sl.bytes = rb;
        qidx.push_back(qi);
        aoff.push_back(off);
        adm.push_back(std::move(r));
        s->queue.pop_front();
    }
    const int na = (int)adm.size();
    if (na == 0) return VC_OK;

    // upload layout (same offsets on host and device): descriptors | slot
    // indices | packed CSRs; the device buffer continues with root scratch
    const size_t off_idx = a256(sizeof(QueryDesc) * na);
    const size_t off_csr = off_idx + a256(sizeof(int) * na);
    size_t up = off_csr;
    std::vector<size_t> coff(na);
    int max_n = 0, max_deg = 0;
    for (int i = 0; i < na; i++) {
        coff[i] = up;
        up += csr_bytes(adm[i].n, adm[i].m2);
        max_n = std::max(max_n, adm[i].n);
        max_deg = std::max(max_deg, adm[i].maxdeg);
    }
    up = a256(up);
    size_t dev_total = up;
    std::vector<size_t> soff(na);
    for (int i = 0; i < na; i++) {
        soff[i] = dev_total;
        dev_total += root_scratch_bytes(adm[i].n);
    }
    int rc;
    if ((rc = s->h_up.ensure(up)) != VC_OK) return rc;
    if ((rc = s->admit.ensure(dev_total)) != VC_OK) return rc;
    char *h = s->h_up.as<char>();
    char *d = s->admit.as<char>();
    char *ar = s->arena.as<char>();
    QueryDesc *hq = (QueryDesc *)h;
    int *hidx = (int *)(h + off_idx);
    for (int i = 0; i < na; i++) {
        const Request &r = adm[i];
        char *hc = h + coff[i];
        const size_t rp_b = ((size_t)(r.n + 1) * 4 + 15) & ~(size_t)15;
        memcpy(hc, r.csr.data(), (size_t)(r.n + 1) * 4);
        if (r.m2 > 0) memcpy(hc + rp_b, r.csr.data() + r.n + 1, (size_t)r.m2 * 4);
        QueryDesc &Q = hq[i];
        memset(&Q, 0, sizeof(Q));
        Q.n = r.n;
        Q.m2 = r.m2;
        Q.rp = (const int *)(d + coff[i]);
        Q.col = (const int *)(d + coff[i] + rp_b);
        Q.k = r.k;
        Q.maxdeg_in = r.maxdeg;
        Q.status = VC_OK;
        Q.gen = s->slot[qidx[i]].gen;
        const size_t ni = (size_t)(r.n > 0 ? r.n : 1);
        char *p = d + soff[i];
        auto take = [&](char *&q, size_t b) { char *x = q; q += a256(b); return x; };
        Q.deg = (int *)take(p, ni * 4);
        Q.aux = (int *)take(p, ni * 4);
        Q.fr0 = (int *)take(p, ni * 4);
        Q.fr1 = (int *)take(p, ni * 4);
        Q.flag = (int *)take(p, ni * 4);
        Q.forced_list = (int *)take(p, ni * 4);
        Q.heavy = (int *)take(p, ni * 4);
        char *a = ar + aoff[i];
        Q.st = (uint8_t *)take(a, ni);
        Q.cover_flags = (uint8_t *)take(a, ni);
        Q.rp2 = (int *)take(a, (ni + 1) * 4);
        Q.col2 = (int *)take(a, (size_t)std::max(r.m2, 1) * 4);
        Q.orig = (int *)take(a, ni * 4);
        Q.cover_list = (int *)take(a, ni * 4);
        hidx[i] = qidx[i];
    }
    cudaStream_t st = s->stream;
    SV_CK(cudaEventRecord(s->ev[0], st));
    SV_CK(cudaMemcpyAsync(d, h, up, cudaMemcpyHostToDevice, st));
    QueryDesc *dq = (QueryDesc *)d;
    SV_CK(serve_validate_run(dq, na, st));
    SV_CK(root_run(dq, na, max_n, max_deg, st));
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        SV_CK(serve_place_run(L.pl, L.P, dq, (const int *)(d + off_idx), na, L.max_np, l, L.min_np,
                              l == s->nlanes - 1 ? 1 : 0, st));
        L.dirty = true;
    }
    SV_CK(cudaEventRecord(s->ev[1], st));
    s->st.h2d_bytes += (long long)up;
    s->st.admitted += na;
    *n_admitted = na;
    return VC_OK;
}

int step(vc_server *s, int *completed)
{
    *completed = 0;
    cudaStream_t st = s->stream;
    int rc;
    s->st.steps++;
    // a class with nothing in flight is emptied before new requests come in
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        bool busy = false;
        for (int qi : s->active) busy |= s->slot[qi].lane == l;
        if (!busy && L.dirty && (rc = reset_state(s, L)) != VC_OK) return rc;
    }
    int na = 0;
    if ((rc = admit(s, &na)) != VC_OK) return rc;
    s->active.clear();
    for (int i = 0; i < s->cfg.max_inflight; i++)
        if (s->slot[i].busy) s->active.push_back(i);
    const int nact = (int)s->active.size();
    if (nact == 0) return VC_OK;
    // one time slice per class with work (each class's kernel ends at once
    // when none of its requests is unfinished)
    bool sliced = false;
    SV_CK(cudaEventRecord(s->ev[2], st));
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        if (!(na > 0 || L.snap[kRemaining] > 0)) continue;
        SV_CK(cudaMemsetAsync(&ctlw(L.P.ctl, kMaxProcNs), 0, 8, st));
        SV_CK(cudaMemsetAsync(&ctlw(L.P.ctl, kMaxExitNs), 0, 8, st));
        SV_CK(search_slice_run(L.pl, L.P, st));
        s->st.slices++;
        sliced = true;
    }
    SV_CK(cudaEventRecord(s->ev[3], st));
    memcpy(s->m_act.p, s->active.data(), sizeof(int) * nact);
    SV_CK(cudaMemsetAsync(s->cover_ctr.p, 0, sizeof(unsigned long long), st));
    SV_CK(cudaEventRecord(s->ev[4], st));
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        SV_CK(serve_retire_run(s->slots.as<QueryDesc>(), s->m_act.dev_as<int>(), nact, L.P.reg, L.P.reg_words,
                               L.wcap, s->m_rec.dev_as<RetireRec>(), s->m_cover.dev_as<int>(), s->cfg.cover_buffer,
                               s->cover_ctr.as<unsigned long long>(), L.P.ctl,
                               L.m_ctl.dev_as<unsigned long long>(), l, st));
    }
    SV_CK(cudaEventRecord(s->ev[5], st));
    SV_CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (na > 0 && cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]) == cudaSuccess) s->st.ms_admit += ms;
    if (sliced && cudaEventElapsedTime(&ms, s->ev[2], s->ev[3]) == cudaSuccess) s->st.ms_search += ms;
    if (cudaEventElapsedTime(&ms, s->ev[4], s->ev[5]) == cudaSuccess) s->st.ms_retire += ms;
    int kstatus[kMaxLanes] = {};
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        memcpy(L.snap, L.m_ctl.p, sizeof(L.snap));
        s->st.max_stack = std::max(s->st.max_stack, (int32_t)L.snap[kMaxStack]);
        s->st.d2h_bytes += (long long)sizeof(L.snap);
        kstatus[l] = (int)(int64_t)L.snap[kStatus];
    }
    s->st.d2h_bytes += (long long)sizeof(RetireRec) * nact;

    const RetireRec *rec = s->m_rec.as<RetireRec>();
    const int32_t *cov = s->m_cover.as<int32_t>();
    int done = 0;
    for (int i = 0; i < nact; i++) {
        const RetireRec &R = rec[i];
        const int qi = s->active[i];
        const int l = R.lane >= 0 && R.lane < s->nlanes ? R.lane : 0;
        s->slot[qi].lane = l;
        vc_server_result r{};
        if (R.state == 1 && R.cover_off >= 0) {
            r.status = R.status;
            r.size = R.status == VC_OK ? R.result : -1;
            r.yes = R.status == VC_OK ? R.yes : 0;
            r.n_induced = R.np;
            r.cover_len = R.cover_len;
            r.nodes = R.nodes;
            s->st.d2h_bytes += 4ll * R.cover_len;
            finish_slot(s, qi, r, cov + R.cover_off);
            done++;
        } else if (kstatus[l] != 0) {
            // the class's slice failed as a whole: each of its unfinished
            // requests ends with that status
            r.status = kstatus[l];
            r.size = -1;
            r.n_induced = R.np;
            r.nodes = R.state == 1 ? R.nodes : 0;
            finish_slot(s, qi, r, nullptr);
            done++;
        }
    }
    for (int l = 0; l < s->nlanes; l++)
        if (kstatus[l] != 0) s->lane[l].dirty = true;   // emptied before the next admission
    s->active.clear();
    for (int i = 0; i < s->cfg.max_inflight; i++)
        if (s->slot[i].busy) s->active.push_back(i);
    *completed = done;
    return VC_OK;
}

}  // namespace

extern "C" {

int vc_server_config_default(vc_server_config *cfg)
{
    if (!cfg) return VC_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    cfg->max_inflight = 1024;
    cfg->max_induced = 2048;
    cfg->dtype_bytes = 2;
    cfg->team = 128;
    cfg->quantum_us = 2000;
    cfg->use_components = 1;
    cfg->load_balance = 1;
    cfg->idle_timeout_ms = 60000;
    cfg->arena_bytes = (int64_t)2 << 30;
    cfg->cover_buffer = (int64_t)16 << 20;
    cfg->max_induced_large = 20000;
    return VC_OK;
}

int vc_server_create(const vc_server_config *cfg_in, void *cuda_stream, vc_server **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    vc_server_config cfg;
    vc_server_config_default(&cfg);
    if (cfg_in) {
        vc_server_config d = cfg;
        cfg = *cfg_in;
        if (cfg.max_inflight <= 0) cfg.max_inflight = d.max_inflight;
        if (cfg.max_induced <= 0) cfg.max_induced = d.max_induced;
        if (cfg.dtype_bytes == 0) cfg.dtype_bytes = d.dtype_bytes;
        if (cfg.team == 0) cfg.team = d.team;
        if (cfg.quantum_us <= 0) cfg.quantum_us = d.quantum_us;
        if (cfg.idle_timeout_ms <= 0) cfg.idle_timeout_ms = d.idle_timeout_ms;
        if (cfg.arena_bytes <= 0) cfg.arena_bytes = d.arena_bytes;
        if (cfg.cover_buffer <= 0) cfg.cover_buffer = d.cover_buffer;
        if (cfg.max_induced_large < 0) cfg.max_induced_large = 0;
    }
    if (cfg.dtype_bytes != 1 && cfg.dtype_bytes != 2 && cfg.dtype_bytes != 4) return VC_EINVAL;
    if (cfg.max_inflight > (1 << 20) || cfg.max_induced > (1 << 24) || cfg.max_induced_large > (1 << 24) ||
        cfg.node_budget < 0)
        return VC_EINVAL;
    if (cfg.team != 32 && cfg.team < 64) return VC_EINVAL;

    vc_server *s = new vc_server();
    s->cfg = cfg;
    s->stream = (cudaStream_t)cuda_stream;
    s->t0 = std::chrono::steady_clock::now();
    auto fail = [&](int rc) { s->release(); delete s; return rc; };
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        return fail(VC_ECUDA);
    for (auto &e : s->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(VC_ECUDA);

    // size classes: induced graphs of up to max_induced vertices, then (when
    // max_induced_large is larger) up to max_induced_large
    const int caps[kMaxLanes] = {cfg.max_induced, cfg.max_induced_large};
    s->nlanes = cfg.max_induced_large > cfg.max_induced ? 2 : 1;
    int rc;
    for (int l = 0; l < s->nlanes; l++) {
        Lane &L = s->lane[l];
        L.ncap = (caps[l] + 16 + 15) / 16 * 16;
        L.wcap = caps[l] / 32 + 2;
        L.min_np = l == 0 ? 0 : s->lane[l - 1].max_np;
        L.max_np = L.ncap;
        // the large class uses the default worker shape for its size (the
        // configured team is for the small class)
        rc = search_plan(cfg.dtype_bytes, l == 0 ? cfg.team : 0, L.ncap, L.wcap, s->sms, 0, &L.pl);
        if (rc != VC_OK) return fail(rc);
        const SearchPlan &pl = L.pl;
        int depth = cfg.stack_depth > 0 ? cfg.stack_depth : std::min(L.ncap + 2, l == 0 ? 1024 : 2048);
        const size_t per_level = (size_t)pl.workers * pl.slot_bytes;
        const size_t stack_budget = (size_t)8 << 30;
        if (cfg.stack_depth <= 0 && (size_t)depth * per_level > stack_budget)
            depth = (int)std::max<size_t>(16, stack_budget / per_level);
        int wl_cap = 1;
        const int wl_want = cfg.worklist_capacity > 0
                                ? cfg.worklist_capacity
                                : std::max(std::max(4 * pl.workers, 1024), (l == 0 ? 4 : 16) * cfg.max_inflight);
        while (wl_cap < wl_want) wl_cap <<= 1;
        int reg_cap = cfg.registry_capacity;
        if (reg_cap <= 0) {
            const size_t per_entry = sizeof(RegEntry) + (size_t)L.wcap * 4;
            reg_cap = (int)std::min<size_t>((size_t)4 << 20, (((size_t)4 << 30) >> l) / per_entry);
            reg_cap = std::max(reg_cap, 64 * pl.workers);
        }
        reg_cap += cfg.max_inflight;
        if ((rc = L.stack.ensure((size_t)pl.workers * depth * pl.slot_bytes)) != VC_OK ||
            (rc = L.wl.ensure((size_t)wl_cap * pl.slot_bytes)) != VC_OK ||
            (rc = L.wl_seq.ensure((size_t)wl_cap * 4)) != VC_OK ||
            (rc = L.reg.ensure((size_t)reg_cap * sizeof(RegEntry))) != VC_OK ||
            (rc = L.reg_words.ensure((size_t)reg_cap * L.wcap * 4)) != VC_OK ||
            (rc = L.comp_scratch.ensure((size_t)pl.workers * 5 * L.ncap * 4)) != VC_OK ||
            (rc = L.ctl.ensure(kCtlWords * 8)) != VC_OK ||
            (rc = L.stack_top.ensure((size_t)pl.workers * 4)) != VC_OK ||
            (rc = L.m_ctl.ensure(kCtlEntries * 8, true)) != VC_OK ||
            (pl.wglobal_bytes > 0 && (rc = L.wglobal.ensure((size_t)pl.workers * (size_t)pl.wglobal_bytes)) != VC_OK))
            return fail(rc);
        SearchParams &P = L.P;
        P.queries = nullptr;   // set below, once the slot array exists
        P.nq = cfg.max_inflight;
        P.team = pl.warp_team ? 32 : pl.threads;
        P.workers = pl.workers;
        P.ncap = L.ncap;
        P.wcap = L.wcap;
        P.slot_bytes = pl.slot_bytes;
        P.stack_depth = depth;
        P.stack_slots = L.stack.as<char>();
        P.wl_slots = L.wl.as<char>();
        P.wl_seq = L.wl_seq.as<unsigned>();
        P.wl_cap = wl_cap;
        P.wl_low = cfg.load_balance ? std::max(8, std::min(wl_cap / 2, 4 * pl.workers)) : 0;
        P.reg = L.reg.as<RegEntry>();
        P.reg_words = L.reg_words.as<uint32_t>();
        P.reg_cap = reg_cap;
        P.comp_scratch = L.comp_scratch.as<int>();
        P.ctl = L.ctl.as<unsigned long long>();
        P.node_budget = cfg.node_budget;
        P.idle_timeout_ns = (long long)cfg.idle_timeout_ms * 1000000ll;
        P.use_components = cfg.use_components;
        P.load_balance = cfg.load_balance;
        P.csr_smem = 0;
        P.csr_query = 0;
        P.quantum_ns = (long long)cfg.quantum_us * 1000ll;
        P.stack_top = L.stack_top.as<int>();
        P.no_bounds = 0;
        P.breakdown = 0;
        P.no_dyn_bounds = 0;
        P.comp_lp = 0;
        P.wglobal = pl.wglobal_bytes > 0 ? L.wglobal.as<char>() : nullptr;
        P.wglobal_stride = pl.wglobal_bytes;
        for (DevBuf *b : {&L.stack, &L.wl, &L.wl_seq, &L.reg, &L.reg_words, &L.comp_scratch, &L.ctl, &L.stack_top,
                          &L.wglobal})
            s->st.device_bytes += (int64_t)b->bytes;
    }
    if ((rc = s->slots.ensure(sizeof(QueryDesc) * cfg.max_inflight)) != VC_OK ||
        (rc = s->arena.ensure((size_t)cfg.arena_bytes)) != VC_OK ||
        (rc = s->cover_ctr.ensure(256)) != VC_OK ||
        (rc = s->m_rec.ensure(sizeof(RetireRec) * cfg.max_inflight, true)) != VC_OK ||
        (rc = s->m_cover.ensure((size_t)cfg.cover_buffer * 4, true)) != VC_OK ||
        (rc = s->m_act.ensure(sizeof(int) * cfg.max_inflight, true)) != VC_OK)
        return fail(rc);
    s->arena_alloc.init((size_t)cfg.arena_bytes);
    for (int l = 0; l < s->nlanes; l++) s->lane[l].P.queries = s->slots.as<QueryDesc>();

    s->slot.assign(cfg.max_inflight, Slot{});
    for (int i = cfg.max_inflight - 1; i >= 0; i--) s->free_slots.push_back(i);
    if (cudaMemsetAsync(s->slots.p, 0, s->slots.bytes, s->stream) != cudaSuccess) return fail(VC_ECUDA);
    for (int l = 0; l < s->nlanes; l++)
        if ((rc = reset_state(s, s->lane[l])) != VC_OK) return fail(rc);
    s->st.resets = 0;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(VC_ECUDA);

    const Lane &L0 = s->lane[0];
    s->st.workers = L0.pl.workers;
    s->st.team = L0.P.team;
    s->st.dtype_bytes = L0.pl.dtype;
    s->st.max_induced = s->nlanes > 1 ? cfg.max_induced_large : cfg.max_induced;
    s->st.slot_bytes = L0.pl.slot_bytes;
    for (DevBuf *b : {&s->slots, &s->arena, &s->cover_ctr}) s->st.device_bytes += (int64_t)b->bytes;
    *out = s;
    return VC_OK;
}

int vc_server_submit(vc_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k, int64_t tag)
{
    if (!s || n < 0 || !row_ptr) return VC_EINVAL;
    const int m2 = row_ptr[n];
    if (m2 < 0 || (m2 & 1) || (m2 > 0 && !col) || (n == 0 && m2 != 0)) return VC_EINVAL;
    if (a256(resident_bytes(n, m2)) > (size_t)s->cfg.arena_bytes) return VC_ECAPACITY;
    Request r;
    r.tag = tag;
    r.n = n;
    r.m2 = m2;
    r.k = k < 0 ? -1 : k;
    r.maxdeg = 0;
    for (int v = 0; v < n; v++) r.maxdeg = std::max(r.maxdeg, row_ptr[v + 1] - row_ptr[v]);
    r.csr.resize((size_t)n + 1 + m2);
    memcpy(r.csr.data(), row_ptr, (size_t)(n + 1) * 4);
    if (m2 > 0) memcpy(r.csr.data() + n + 1, col, (size_t)m2 * 4);
    r.t_submit = s->now_ms();
    s->queue.push_back(std::move(r));
    s->st.submitted++;
    return VC_OK;
}

int vc_server_step(vc_server *s, int32_t *completed)
{
    if (!s) return VC_EINVAL;
    int c = 0;
    const int rc = step(s, &c);
    if (completed) *completed = c;
    return rc;
}

int vc_server_counts(const vc_server *s, int32_t *queued, int32_t *inflight, int32_t *ready)
{
    if (!s) return VC_EINVAL;
    if (queued) *queued = (int32_t)s->queue.size();
    if (inflight) *inflight = (int32_t)s->active.size();
    if (ready) *ready = (int32_t)s->ready.size();
    return VC_OK;
}

int vc_server_poll(vc_server *s, int32_t max_results, vc_server_result *out, int32_t *count, int32_t *cover_buf,
                   int64_t cover_cap)
{
    if (!s || !count || (max_results > 0 && !out) || cover_cap < 0 || (cover_cap > 0 && !cover_buf))
        return VC_EINVAL;
    int c = 0;
    int64_t used = 0;
    while (c < max_results && !s->ready.empty()) {
        Done &d = s->ready.front();
        const int64_t len = (int64_t)d.cover.size();
        if (used + len > cover_cap) break;
        out[c] = d.r;
        out[c].cover_off = len > 0 ? used : -1;
        if (len > 0) memcpy(cover_buf + used, d.cover.data(), (size_t)len * 4);
        used += len;
        c++;
        s->ready.pop_front();
    }
    *count = c;
    return VC_OK;
}

int vc_server_get_stats(const vc_server *s, vc_server_stats *st)
{
    if (!s || !st) return VC_EINVAL;
    *st = s->st;
    st->nodes = st->search_bytes = st->wait_polls = st->preemptions = st->max_node_ns = st->max_exit_ns = 0;
    for (int l = 0; l < s->nlanes; l++) {
        const Lane &L = s->lane[l];
        st->nodes += L.base_nodes + (long long)L.snap[kNodes];
        st->search_bytes += L.base_bytes + (long long)L.snap[kBytes];
        st->wait_polls += L.base_waits + (long long)L.snap[kWaitIters];
        st->preemptions += L.base_preempts + (long long)L.snap[kPreempts];
        st->max_node_ns = std::max(st->max_node_ns, (int64_t)L.snap[kMaxProcNs]);
        st->max_exit_ns = std::max(st->max_exit_ns, (int64_t)L.snap[kMaxExitNs]);
    }
    return VC_OK;
}

void vc_server_free(vc_server *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    s->release();
    delete s;
}

}  // extern "C"
