// Host-side launch wrappers shared by the .cu files of the library.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "vc_common.cuh"

namespace vcg {

// The CUDA error behind the last VC_ECUDA / VC_ENOMEM on this host thread.
inline cudaError_t &last_cuda_error()
{
    static thread_local cudaError_t e = cudaSuccess;
    return e;
}

// Growable device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t want)
    {
        if (want <= bytes) return VC_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (cudaMalloc(&p, want) != cudaSuccess) return VC_ENOMEM;
        bytes = want;
        return VC_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class X>
    X *as() const { return (X *)p; }
};

// Growable pinned host buffer; `mapped` ones are also addressable by the
// device (dev = the device pointer of the same memory).
struct HostBuf {
    void *p = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    int ensure(size_t want, bool mapped = false)
    {
        if (want <= bytes && (!mapped || dev)) return VC_OK;
        release();
        if (cudaHostAlloc(&p, want, mapped ? cudaHostAllocMapped : cudaHostAllocDefault) != cudaSuccess) {
            p = nullptr;
            return VC_ENOMEM;
        }
        if (mapped && cudaHostGetDevicePointer(&dev, p, 0) != cudaSuccess) {
            release();
            return VC_ECUDA;
        }
        bytes = want;
        return VC_OK;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        dev = nullptr;
        bytes = 0;
    }
    template <class X>
    X *as() const { return (X *)p; }
    template <class X>
    X *dev_as() const { return (X *)dev; }
};

// ---- root phase (vc_root.cu)
cudaError_t validate_run(int n, int m2, const int *rp, const int *col, int *d_err, cudaStream_t s);
// max_n / max_deg: the largest input graph and degree among the queries
cudaError_t root_run(QueryDesc *d_q, int nq, int max_n, int max_deg, cudaStream_t s);
// Answers and ascending cover lists (also into Q.cover_out when set).
// mode 0: every query; 1: only the queries the root phase settled (reg may be
// null); 2: only the searched ones.
cudaError_t finalize_run(QueryDesc *d_q, int nq, const RegEntry *reg, const uint32_t *reg_words, int wcap,
                         cudaStream_t s, int mode = 0);
// Crown (Nemhauser-Trotter) reduction of each query's induced graph, for the
// queries whose descriptor has a crown workspace (after root_run).
cudaError_t crown_run(QueryDesc *d_q, int nq, cudaStream_t s);

// ---- search (vc_search.cu)
struct SearchPlan {
    int dtype;          // bytes per degree entry
    int warp_team;      // 1: one warp per worker, 0: one block per worker
    int threads;        // threads per block
    int blocks;         // persistent blocks
    int workers;        // workers = blocks * (warp_team ? threads / 32 : 1)
    size_t smem;        // dynamic shared memory per block
    int slot_bytes;     // bytes per node slot
    int csr_bytes;      // shared memory reserved for a staged CSR (0: none)
    long long wglobal_bytes;  // > 0: bytes of global memory per worker for its node
                              // arrays (they do not fit in shared memory)
};

// Choose the worker shape for induced graphs of up to ncap vertices.
// Returns VC_OK or VC_ECAPACITY (does not fit in shared memory).
// csr_bytes > 0 reserves that much shared memory per block for a staged CSR.
int search_plan(int dtype, int team_req, int ncap, int wcap, int sms, int csr_bytes, SearchPlan *out);

// Initialise the registry / worklist, place each root node (root_slot[q] >= 0
// for searched queries) and run the persistent kernel; ev0 / ev1 (nullable)
// are recorded around it with ev_flags (cudaEventRecordExternal while the
// stream is being captured into a graph).
cudaError_t search_run(const SearchPlan &pl, SearchParams &P, const int *d_root_slot, int nq, int nroots,
                       cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, unsigned ev_flags = 0);

// ---- served requests (resident search state, vc_search.cu)
// Launch only the persistent search kernel (one time slice when
// P.quantum_ns > 0, resuming from P.stack_top).
cudaError_t search_slice_run(const SearchPlan &pl, const SearchParams &P, cudaStream_t s);
// Empty worklist, counters and registry allocator; registry entries below
// `first` are reserved (one root entry per query slot).
cudaError_t search_reset_run(const SearchParams &P, int first, cudaStream_t s);
// Place na root-reduced descriptors (device staging array) into their slots
// and push the root nodes of those that need a search.
// (lane: the size class placing; it takes the requests with min_np < np <=
// max_np, lane 0 also the settled ones, the last lane also the larger ones)
cudaError_t serve_place_run(const SearchPlan &pl, const SearchParams &P, const QueryDesc *d_staging,
                            const int *d_slot_idx, int na, int max_np, int lane, int min_np, int last,
                            cudaStream_t s);

// ---- served requests (vc_root.cu)
// Validate na staged CSR graphs (one block each); a malformed one gets
// status VC_EINVAL, which the root phase and the placement respect.
cudaError_t serve_validate_run(QueryDesc *d_staging, int na, cudaStream_t s);

// For each active slot: if its request is finished, finalise the answer and
// cover (as finalize_run) and copy the cover to cover_out at an offset taken
// from *cover_ctr (device counter, zeroed by the caller).  Block 0 also
// copies the control block's first words to ctl_out (mapped).  Only the
// slots of size class `lane` are handled (reg / reg_words / wcap / ctl are
// that class's); the others keep their records for their own class.
cudaError_t serve_retire_run(QueryDesc *d_slots, const int *active, int nactive, const RegEntry *reg,
                             const uint32_t *reg_words, int wcap, RetireRec *rec, int *cover_out,
                             long long cover_cap, unsigned long long *cover_ctr,
                             const unsigned long long *ctl, unsigned long long *ctl_out, int lane,
                             cudaStream_t s);

}  // namespace vcg
