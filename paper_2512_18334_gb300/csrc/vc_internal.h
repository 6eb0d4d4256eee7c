// Host-side launch wrappers shared by the .cu files of the library.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "vc_common.cuh"

namespace vcg {

// ---- root phase (vc_root.cu)
cudaError_t validate_run(int n, int m2, const int *rp, const int *col, int *d_err, cudaStream_t s);
// max_n / max_deg: the largest input graph and degree among the queries
cudaError_t root_run(QueryDesc *d_q, int nq, int max_n, int max_deg, cudaStream_t s);
cudaError_t finalize_run(QueryDesc *d_q, int nq, const RegEntry *reg, const uint32_t *reg_words, int wcap,
                         cudaStream_t s);

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
};

// Choose the worker shape for induced graphs of up to ncap vertices.
// Returns VC_OK or VC_ECAPACITY (does not fit in shared memory).
// csr_bytes > 0 reserves that much shared memory per block for a staged CSR.
int search_plan(int dtype, int team_req, int ncap, int wcap, int sms, int csr_bytes, SearchPlan *out);

// Initialise the registry / worklist, place each root node (root_slot[q] >= 0
// for searched queries) and run the persistent kernel.
cudaError_t search_run(const SearchPlan &pl, SearchParams &P, const int *d_root_slot, int nq, int nroots,
                       cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1);

}  // namespace vcg
