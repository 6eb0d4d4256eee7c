/*
 * Exact vertex cover on one GB300 (sm_103a): C ABI.
 *
 * The solver is the component-aware parallel branch-and-reduce of
 * "Faster Vertex Cover Algorithms on GPUs with Component-Aware Parallel
 * Branching" (arXiv 2512.18334):
 *   - the graph is reduced at the root and an induced subgraph is built on
 *     the device (Section 4.2),
 *   - persistent workers pop search-tree nodes (degree arrays of the induced
 *     subgraph, Section 4.1) from a private stack or a shared worklist
 *     (Section 2.3), apply the degree-one, degree-two-triangle and high-degree
 *     rules (Section 2.2), prune with the stopping condition (Algorithm 1),
 *     find connected components (Section 3.2) and branch on them
 *     (Algorithm 2, Section 3.3) through a component-branch registry whose
 *     last descendant aggregates the result (Section 3.3); cliques and
 *     chordless cycles are closed directly (Section 3.4).
 *
 * Input graphs are simple and undirected, in CSR form:
 *   row_ptr  int32[n + 1], row_ptr[0] = 0, non-decreasing
 *   col      int32[row_ptr[n]], each row sorted strictly ascending,
 *            symmetric (v in row u iff u in row v), no self-loops.
 * Anything else is rejected with VC_EINVAL (checked on the device).
 *
 * Cover outputs are vertex ids of the caller's numbering, sorted ascending,
 * in caller-owned host arrays of capacity n.  Every function returns VC_OK
 * (0) or a negative status; vc_strerror() names it.
 *
 * Threading: a vc_graph handle owns device memory and a CUDA stream binding;
 * it is not thread-safe.  Use one handle per host thread / stream.
 */
#ifndef VC_GB300_H
#define VC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VC_OK 0
#define VC_EINVAL (-1)     /* malformed CSR, bad argument                        */
#define VC_ENOMEM (-2)     /* a device or pinned-host allocation failed          */
#define VC_ECAPACITY (-3)  /* stack, worklist or registry full after retries     */
#define VC_ETIMEOUT (-4)   /* a bounded device wait expired (no progress)        */
#define VC_ECUDA (-5)      /* a CUDA runtime call failed                         */
#define VC_EBUDGET (-6)    /* node budget exhausted before the search finished   */

typedef struct vc_graph vc_graph;

/* Solver options.  Start from vc_options_default().  For team, dtype_bytes,
 * stack_depth, worklist_capacity, registry_capacity, idle_timeout_ms and
 * node_budget, 0 means automatic / the default; use_components and
 * load_balance are 1 in the defaults (0 switches them off); the ablation
 * switches are 0 (off) in the defaults. */
typedef struct vc_options {
    int32_t use_components;   /* 1: branch on components (Algorithm 2); 0: Algorithm 1 */
    int32_t team;             /* threads per worker: 0 auto (128-thread blocks up to
                                 4,096 induced vertices, 256 above), 32 (one warp
                                 per worker) or 64..1024 (one block per worker) */
    int32_t dtype_bytes;      /* degree-array entry size: 0 auto, 1, 2 or 4 (Section 4.4) */
    int32_t stack_depth;      /* private stack slots per worker, 0 auto             */
    int32_t worklist_capacity;/* shared worklist slots, 0 auto                      */
    int32_t registry_capacity;/* component-branch registry entries, 0 auto          */
    int32_t load_balance;     /* 1: offload to the shared worklist; 0: only the
                                 root is shared, workers keep what they create      */
    int32_t idle_timeout_ms;  /* abort with VC_ETIMEOUT after this long without
                                 any worker making progress; 0 = 60000              */
    int64_t node_budget;      /* 0 = unlimited; else a query that needs more search-tree
                                 nodes stops with VC_EBUDGET (per query in a batch) */
    /* Ablations of the paper's optimisations (answers do not change): */
    int32_t disable_bounds;   /* 1: every node keeps the whole degree array as its
                                 window instead of the non-zero bounds (Section 4.3) */
    int32_t disable_root_rules; /* 1: no reduction at the root (Section 4.2): the
                                 search starts from every vertex that has an edge */
    int32_t breakdown;        /* 1: count SM cycles per activity (vc_stats.phase_cycles) */
    int32_t offload_below;    /* load balancing: a new right child goes to the shared
                                 worklist while it holds fewer items than this;
                                 0 = four per worker, at most half the worklist */
    int32_t disable_dyn_bounds; /* 1: a component's bound stays the one fixed when it
                                 was registered (no dynamic tightening from the
                                 enclosing Best and the finished siblings) */
    int32_t crown;            /* 1: crown reduction at the root (Section 4.2), applied
                                 as the Nemhauser-Trotter LP reduction on the device
                                 after the other root rules; answers do not change */
    int32_t cuda_graph;       /* 1 (default): the root phase (descriptor upload,
                                 root [and crown] kernel, finalisation of settled
                                 queries, read-back) and the search phase (root-
                                 slot upload, registry and worklist set-up, root
                                 placement, the persistent search, finalisation,
                                 read-back) are each captured into a CUDA graph
                                 the second time a launch shape comes in a row,
                                 kept with the workspace and replayed with one
                                 launch; 0: their kernels are launched one by one */
    int32_t capacity_retries; /* when the search runs out of capacity, solve again
                                 up to this many times (default 2; 0: report
                                 VC_ECAPACITY at once), doubling only what ran out:
                                 the stack depth and worklist capacity when both
                                 were full, the registry capacity when it was
                                 exhausted.  Growth stops at 24 GB of private
                                 stacks, 8 GB of worklist and 16 GB of registry
                                 (worst case about 48 GB for one solve); a solve
                                 that retried frees its grown buffers before it
                                 returns.  vc_autotune does not retry */
    int32_t label_propagation;/* how a node's graph is split into connected
                                 components (Section 3.2): 0 (default) union-find,
                                 one pass over the live edges; 1 label propagation,
                                 every live vertex pulling the smallest label of its
                                 live neighbours (rows walked by 8-lane groups of a
                                 warp) and then its label's label, in rounds until
                                 one changes nothing.  Answers do not change */
} vc_options;

/* What a solve did.  All counters are totals over the launch. */
typedef struct vc_stats {
    int64_t nodes;              /* search-tree nodes processed                      */
    int64_t component_branches; /* nodes that branched on >= 2 components           */
    int64_t leaves;             /* nodes whose graph had no edges left              */
    int64_t pruned;             /* nodes cut by the stopping condition              */
    int64_t offloaded;          /* nodes pushed to the shared worklist              */
    int64_t trivial_components; /* components closed by the clique / cycle rules    */
    int64_t comp_hist[16];      /* branches on c components, c = 2..16 (16 = >=16)  */
    int32_t n;                  /* vertices of the input graph                      */
    int32_t n_induced;          /* vertices of the induced subgraph searched        */
    int32_t m_induced;          /* edges of the induced subgraph                    */
    int32_t forced;             /* vertices put in the cover by the root reduction  */
    int32_t greedy_size;        /* initial upper bound (whole graph)                */
    int32_t dtype_bytes;        /* degree-array entry size used                     */
    int32_t team;               /* threads per worker used                          */
    int32_t workers;            /* persistent workers launched                      */
    int32_t max_stack;          /* deepest private stack seen                       */
    int32_t err_where;          /* diagnostic site code of the first device error   */
    int32_t launches;           /* kernels this call launched                       */
    int32_t root_rounds;        /* synchronous rule rounds in the root phase        */
    double ms_root;             /* root reduction + induced subgraph (device)       */
    double ms_search;           /* persistent search kernel (device)                */
    double ms_total;            /* whole call, host wall clock                      */
    int64_t root_cycles[4];     /* SM cycles in the root phase: rules without a
                                   bound, greedy bound, rules with the bound, induce */
    int64_t search_bytes;       /* algorithmic bytes the search moved: node slots
                                   read and written, CSR rows read, witness bitmaps */
    int64_t phase_cycles[6];    /* with opt.breakdown: SM cycles summed over workers,
                                   per activity: take a node from the stack or the
                                   worklist, reduction rules, components (finding,
                                   registering, closing cliques and cycles), vertex
                                   branch, completion through the registry, idle */
    int32_t crown_forced;       /* with opt.crown: vertices it put in the cover     */
    int32_t crown_removed;      /* ... and vertices it removed in all               */
    int32_t crown_skipped;      /* queries where its matching check failed (nothing
                                   was removed)                                     */
    int32_t cuda_graph;         /* search phase: 0 launched kernel by kernel (or no
                                   search), 1 captured into a graph by this call,
                                   2 replayed from the graph of an earlier call     */
    int32_t retries;            /* solves repeated with larger capacities
                                   (opt.capacity_retries); the other fields describe
                                   the last attempt                                 */
    int32_t best_found;         /* summed over the queries: the size of the best
                                   cover known when each stopped -- the answer when
                                   solved (k + 1 for a PVC no), and for a search
                                   that ran out of its node budget the forced
                                   vertices plus the best cover the search had found
                                   (or the initial bound): an upper bound on the
                                   minimum that a caller can set beside a lower
                                   bound of its own                                  */
} vc_stats;

/* Fill *opt with the defaults. */
int vc_options_default(vc_options *opt);

/* Copy a CSR graph from HOST memory to the device and return a handle.
 * `cuda_stream` is a cudaStream_t (NULL = the legacy default stream); every
 * later call on the handle runs on it.  The caller keeps ownership of its
 * arrays.  The graph is validated here (VC_EINVAL on a malformed CSR).
 * Cost: one host-to-device copy of (n + 1 + row_ptr[n]) int32 values. */
int vc_load_csr(int32_t n, const int32_t *row_ptr, const int32_t *col,
                void *cuda_stream, vc_graph **out);

/* As vc_load_csr, but row_ptr / col are DEVICE pointers (already resident in
 * HBM); they are copied device-to-device so the caller may free them. */
int vc_load_csr_device(int32_t n, const int32_t *d_row_ptr, const int32_t *d_col,
                       void *cuda_stream, vc_graph **out);

/* Minimum vertex cover (MVC, Section 2.1).  Writes the minimum size to
 * *cover_size and, when `cover` is non-NULL, a minimum cover (ascending
 * original ids, capacity n) and its length to *cover_len.  `opt` and `stats`
 * may be NULL. */
int vc_solve_min(vc_graph *g, const vc_options *opt, int32_t *cover_size,
                 int32_t *cover, int32_t *cover_len, vc_stats *stats);

/* Parameterized vertex cover (PVC, Section 2.1): is there a cover of size at
 * most k?  *is_yes = 1 with a cover of size <= k (when `cover` is non-NULL),
 * or *is_yes = 0 and *cover_len = 0.  k < 0 is VC_EINVAL; k = 0 is "yes iff
 * the graph has no edge". */
int vc_solve_k(vc_graph *g, int32_t k, const vc_options *opt, int32_t *is_yes,
               int32_t *cover, int32_t *cover_len, vc_stats *stats);

/* Many queries in one root launch and one persistent search launch (a
 * build extension; the paper solves one graph per launch).  Query i is graph
 * graphs[i] with ks == NULL or ks[i] < 0 meaning "minimum cover" and
 * ks[i] >= 0 meaning "is there a cover of size <= ks[i]?".  A graph may
 * appear in several queries (e.g. at two values of k).  Per query:
 *   out_size[i]    minimum size (MVC), size of the cover found (PVC yes) or -1
 *   out_yes[i]     PVC answer (1 for MVC)
 *   out_status[i]  VC_OK or the status that stopped it
 *   covers[i]      (nullable array, nullable entries) host array of capacity
 *                  n_i receiving the cover, ascending original ids
 *   cover_lens[i]  (nullable) its length
 * The launch runs on graphs[0]'s stream with graphs[0]'s workspace.
 * `stats` (nullable) sums over the batch. */
int vc_solve_batch(int32_t count, vc_graph *const *graphs, const int32_t *ks,
                   const vc_options *opt, int32_t *out_size, int32_t *out_yes,
                   int32_t *out_status, int32_t *const *covers, int32_t *cover_lens,
                   vc_stats *stats);

/* Root reduction and induced-subgraph build WITHOUT ANY ALLOCATION.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- for instance a process whose device memory is
 * owned by another allocator (a framework's caching pool that reserved the
 * GPU), or a latency-critical loop that must not call cudaMalloc / cudaFree,
 * which can synchronise the whole device.  It runs the same root phase as
 * vc_solve_min (degree-one and degree-two-triangle rules, greedy bound,
 * high-degree rule, induced subgraph; Section 4.2) on one graph and stops
 * there.
 *
 * Scratch: one file-scope device array of 2 MiB (vertex limit
 * n <= 65536).  Every GPU that loads this library holds it until the
 * process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and sets a kernel attribute; make that
 * first call before any stream capture.  With CUDA's lazy module loading
 * (the default) that first call may also load the library's device code,
 * which allocates the 2 MiB array and the code itself and synchronises: make
 * it outside any region that must not allocate (a warm-up call at start-up).
 * Calls after it on the same device allocate nothing.  All calls share the array and it
 * keeps the last call's contents, so calls whose work overlaps on the GPU
 * (on different streams, or from different host threads) race: serialise
 * them.  Larger graphs are rejected with VC_ECAPACITY; nothing is allocated
 * by this function or by the kernels it launches.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *   d_row_ptr int32[n + 1], d_col int32[m2]   the graph (m2 = row_ptr[n],
 *                                              passed by value); checked on
 *                                              the device like vc_load_csr
 *   k                          < 0: minimum cover; >= 0: bound for "<= k"
 *   d_forced                   int32[n]: vertices forced into the cover
 *   d_induced_row_ptr          int32[n + 1], d_induced_col int32[m2],
 *   d_induced_orig             int32[n]: the induced subgraph (sorted rows,
 *                              vertices relabelled 0..n'-1 in increasing
 *                              original id; orig[i] = original id)
 *   d_info                     int32[8]: status (VC_OK / VC_EINVAL), forced
 *                              count, n', 2|E'|, greedy cover size (-1 if not
 *                              computed), answered (1: the root phase
 *                              settled the answer), the answer when
 *                              answered (minimum size; PVC: size or -1),
 *                              max degree of the induced subgraph.
 * Witness: d_forced plus any cover of the induced subgraph is a cover.  When
 * the root phase settles the answer through the greedy bound (answered = 1
 * and the answer exceeds the forced count), the greedy cover that reaches it
 * is NOT exported: no witness is returned for that answer.
 * Asynchronous on `cuda_stream`: d_info is valid once the stream reaches
 * the end of the call.  Returns VC_OK, VC_EINVAL (bad arguments),
 * VC_ECAPACITY (n > 65536) or VC_ECUDA (launch failure). */
int vc_root_reduce_static(int32_t n, int32_t m2, const int32_t *d_row_ptr, const int32_t *d_col,
                          int32_t k, int32_t *d_forced, int32_t *d_induced_row_ptr,
                          int32_t *d_induced_col, int32_t *d_induced_orig, int32_t *d_info,
                          void *cuda_stream);

/* Autotuner for a batch of queries (same arguments as vc_solve_batch).
 * Starting from *base (NULL = defaults), it tunes by coordinate descent, on
 * the given queries themselves: the worker size (team), the degree type
 * (the dtype threshold: the smallest type that fits, or a wider one), the
 * worklist hunger threshold (offload_below), the stack depth and the
 * worklist capacity.  Each candidate runs `repeats` times (>= 1) and scores
 * the best wall time of a whole vc_solve_batch; candidates that fail are
 * skipped.  Writes the best options to *best and its time to *best_ms; up to
 * max_trials tried candidates and their times (-1: failed) to tried /
 * tried_ms (nullable), and their number to *trials. */
int vc_autotune(int32_t count, vc_graph *const *graphs, const int32_t *ks, const vc_options *base,
                int32_t repeats, vc_options *best, double *best_ms, vc_options *tried, double *tried_ms,
                int32_t max_trials, int32_t *trials);

/* Exact maximum independent set: the complement of a minimum vertex cover
 * (the paper notes that its techniques carry over; related work, "Independent
 * set").  Writes the
 * maximum size n - OPT to *set_size and, when `set` is non-NULL, an
 * independent set of that size (ascending original ids, capacity n) and its
 * length to *set_len.  Same options, statistics and errors as vc_solve_min. */
int vc_solve_mis(vc_graph *g, const vc_options *opt, int32_t *set_size, int32_t *set,
                 int32_t *set_len, vc_stats *stats);

/* Release the handle.  NULL is a no-op.  Its graph buffers go back to a
 * per-device cache that later vc_load_csr calls reuse; the search workspaces
 * (node slots, worklist, registry) are not owned by handles either: they are
 * kept per device, shared by every handle and reused by later solves.
 * vc_trim() frees what is idle in both. */
void vc_free(vc_graph *g);

/* Free the idle search workspaces and cached graph buffers on every device
 * (nothing in use by a live handle or a running solve).  Returns the number
 * of search workspaces freed. */
int vc_trim(void);

/* ------------------------------------------------------------------ serving
 *
 * A request server with continuous batching (a build extension: the paper
 * solves one graph per launch).  Requests -- a graph and a mode (minimum
 * cover, or "is there a cover of size <= k?") -- are queued on the host by
 * vc_server_submit().  Each vc_server_step():
 *   1. admits queued requests in submission order while a query slot is free
 *      and the device arena has room for the request's resident arrays
 *      (induced subgraph, id map, cover arrays: about 4 n + 4 * 2|E| + 14 n
 *      bytes): admission by device memory.  The admitted graphs are copied
 *      to the device in one transfer, validated like vc_load_csr,
 *      root-reduced (Section 4.2), and their root nodes are pushed into the
 *      shared worklist, which still holds the nodes of the requests admitted
 *      earlier;
 *   2. runs the persistent search (Sections 2.3, 3) for one time slice over
 *      every request in flight, old and new together.  At the end of the
 *      slice each worker stores the node it holds and exits; node slots,
 *      worklist, registry and private stacks stay resident in device memory
 *      and the next slice resumes from them;
 *   3. retires the requests that finished: answers and covers are finalised
 *      on the device and written to mapped host memory, and their slots and
 *      arena space are freed.
 * The answer of a request does not depend on what else is in flight; it is
 * the answer vc_solve_min / vc_solve_k give for the same graph.  Requests
 * are served in size classes by the size of their induced subgraph (after
 * the root reduction): up to max_induced vertices, and up to
 * max_induced_large; each class has a resident search of its own (node
 * slots sized for it), and every step runs one time slice of each class
 * that has work.  An induced subgraph above the largest class finishes with
 * VC_ECAPACITY.
 *
 * Threading: a server is not thread-safe; one host thread drives it.
 */
typedef struct vc_server vc_server;

typedef struct vc_server_config {
    int32_t max_inflight;      /* query slots resident on the device (default 1024) */
    int32_t max_induced;       /* vertex capacity of a search node (default 2048) */
    int32_t dtype_bytes;       /* degree entry size 1, 2 or 4 (0: 2) */
    int32_t team;              /* as vc_options.team (0: 128-thread block workers) */
    int32_t stack_depth;       /* private stack slots per worker (0: auto) */
    int32_t worklist_capacity; /* shared worklist slots (0: auto) */
    int32_t registry_capacity; /* registry entries (0: auto) */
    int32_t quantum_us;        /* search time slice per step (default 2000) */
    int32_t use_components;    /* default 1 */
    int32_t load_balance;      /* default 1 */
    int32_t idle_timeout_ms;   /* default 60000 */
    int32_t max_induced_large; /* a second size class: induced graphs larger than
                                  max_induced and up to this many vertices go to a
                                  resident search of their own, sized for them
                                  (default 20000; 0 or <= max_induced: none) */
    int64_t arena_bytes;       /* device memory for admitted requests (default 2 GiB) */
    int64_t node_budget;       /* per request (0: none); VC_EBUDGET when exceeded */
    int64_t cover_buffer;      /* int32 entries of the mapped cover buffer (default 16M) */
} vc_server_config;

typedef struct vc_server_result {
    int64_t tag;               /* the caller's tag from vc_server_submit */
    int32_t status;            /* VC_OK, or the status that ended the request */
    int32_t size;              /* MVC: minimum size; PVC: size of the cover found, or -1 */
    int32_t yes;               /* PVC answer (1 for MVC) */
    int32_t n;                 /* vertices of the request's graph */
    int32_t n_induced;         /* vertices left after the root reduction */
    int32_t cover_len;         /* entries of the cover (0 when status != VC_OK or PVC no) */
    int64_t cover_off;         /* offset of the cover in vc_server_poll's cover_buf */
    int64_t nodes;             /* search-tree nodes spent on the request */
    double t_submit_ms;        /* server clock: milliseconds since vc_server_create */
    double t_admit_ms;
    double t_done_ms;
} vc_server_result;

typedef struct vc_server_stats {
    int64_t steps;             /* vc_server_step calls */
    int64_t slices;            /* search kernel launches */
    int64_t submitted, admitted, completed;
    int64_t nodes;             /* search-tree nodes, all requests */
    int64_t search_bytes;      /* algorithmic bytes moved by the search */
    int64_t h2d_bytes;         /* graphs copied to the device */
    int64_t d2h_bytes;         /* records and covers written to host memory */
    int64_t resets;            /* times the resident search state was emptied */
    double ms_admit;           /* device time: validation, root phase, placement */
    double ms_search;          /* device time of the search slices */
    double ms_retire;          /* device time of finalisation */
    int32_t workers, team, dtype_bytes, max_induced;   /* (of the small class; max_induced:
                                                           the largest class's capacity) */
    int32_t slot_bytes, max_stack;
    int64_t device_bytes;      /* device memory held by the server */
    int64_t wait_polls;        /* polls of worklist sequence words (contention) */
    int64_t preemptions;       /* nodes stored at the end of a time slice */
    int64_t max_node_ns;       /* longest single node (with its left descendants) in the last slice */
    int64_t max_exit_ns;       /* longest worker exit phase in the last slice */
} vc_server_stats;

/* Fill *cfg with the defaults. */
int vc_server_config_default(vc_server_config *cfg);

/* Create a server on the current device; every launch runs on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  Allocates the resident
 * search state (node slots, worklist, registry), the arena and the mapped
 * host buffers up front.  VC_EINVAL (bad config), VC_ECAPACITY (max_induced
 * does not fit a worker in shared memory), VC_ENOMEM, VC_ECUDA. */
int vc_server_create(const vc_server_config *cfg, void *cuda_stream, vc_server **out);

/* Queue a request.  row_ptr / col are HOST arrays in the CSR form above;
 * they are copied, so the caller may reuse them on return.  k < 0: minimum
 * cover; k >= 0: is there a cover of size <= k.  The graph is validated on
 * the device at admission (a malformed one finishes with VC_EINVAL).
 * Returns VC_EINVAL (n < 0, null arrays, row_ptr[n] odd or negative) or
 * VC_ECAPACITY (the request alone is larger than the arena). */
int vc_server_submit(vc_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k,
                     int64_t tag);

/* One scheduling iteration (admit, one search slice per size class with
 * work, retire); blocks until the device finished it.  *completed (nullable)
 * receives the number of requests retired by this step.  A request whose
 * search runs out of node slots or registry entries finishes alone with
 * VC_ECAPACITY; the others continue.  A bounded wait that expires
 * (VC_ETIMEOUT) ends every request in flight in that size class and empties
 * its resident state.  The server stays usable and the step returns VC_OK.
 * VC_ECUDA / VC_ENOMEM are returned as such. */
int vc_server_step(vc_server *s, int32_t *completed);

/* Counts of queued (not yet admitted), in-flight and retired-but-not-polled
 * requests (each pointer nullable). */
int vc_server_counts(const vc_server *s, int32_t *queued, int32_t *inflight, int32_t *ready);

/* Take up to max_results retired requests in completion order.  Their
 * covers are packed into cover_buf (host, capacity cover_cap int32
 * entries; nullable when cover_cap is 0) at each result's cover_off; a
 * result whose cover does not fit stays for the next poll.  *count receives
 * the number taken. */
int vc_server_poll(vc_server *s, int32_t max_results, vc_server_result *out, int32_t *count,
                   int32_t *cover_buf, int64_t cover_cap);

/* Cumulative statistics. */
int vc_server_get_stats(const vc_server *s, vc_server_stats *st);

/* Release the server and all its memory.  NULL is a no-op. */
void vc_server_free(vc_server *s);

/* ------------------------------------------------------------------ measurement
 *
 * The L2 read bandwidth of the current device: the ceiling of the search
 * kernel's roofline, since its working set (node slots, registry, induced
 * CSR) stays in L2 (Section 5 reports throughput; the bandwidth ceiling is
 * this library's).  Allocates a device buffer of `bytes` (>= 1 MiB; keep it
 * well inside L2), reads it once to warm L2, then times `trials` launches
 * of a read kernel (16-byte loads that bypass L1, one pass per rep, `reps`
 * passes per launch) with CUDA events on `cuda_stream`, and writes the best
 * rate in GB/s (10^9 bytes) to *gbs.  Frees the buffer before returning.
 * VC_EINVAL (bad sizes, null gbs), VC_ENOMEM, VC_ECUDA. */
int vc_measure_l2_read(int64_t bytes, int32_t reps, int32_t trials, void *cuda_stream, double *gbs);

/* Name of the CUDA error behind the last VC_ECUDA / VC_ENOMEM returned on
 * this host thread ("no error" if none). */
const char *vc_last_cuda_error(void);

/* Static string naming a status code. */
const char *vc_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* VC_GB300_H */
