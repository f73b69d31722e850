/*
 * dfl.h -- C ABI of the GB300 Dynamic Frontier Louvain library (libdfl.so).
 *
 * The library keeps one dynamic graph and its community state on the GPU
 * and updates the communities after each batch of edge deletions and
 * insertions, as in "DF Louvain: Fast Incrementally Expanding Approach for
 * Community Detection on Dynamic Graphs" (arXiv 2404.19634):
 *   - the batch is applied to a slack CSR graph kept on the device,
 *   - vertex weighted degrees K_i and community totals Sigma_c are updated
 *     incrementally (Alg. 7),
 *   - the initially affected vertices are marked (Alg. 1 DF, Alg. 2 ND,
 *     Alg. 3 DS),
 *   - Louvain runs from the previous membership (Alg. 4): local-moving with
 *     frontier expansion (Alg. 5), aggregation into a super-vertex graph
 *     (Alg. 6), later passes on the super-vertex graph.
 *
 * Conventions for every call:
 *   - Return DFL_OK (0) on success or a negative DFL_ERR_* code.  On error
 *     the handle's state is unchanged (batches are validated before any
 *     mutation) and dfl_last_error() describes the cause.  After
 *     DFL_ERR_CUDA the handle should be destroyed.
 *   - Vertex ids are uint32 in [0, n); edge weights are uint32 > 0; the sum
 *     of all arc weights, 2m, must stay below 2^32 (DFL_ERR_OVERFLOW).
 *     K, Sigma and 2m are reported as int64.
 *   - `mem_kind` says where a caller buffer lives: DFL_MEM_HOST (pageable or
 *     pinned host memory) or DFL_MEM_DEVICE (device memory of the handle's
 *     GPU).  Input buffers are only read during the call and are copied;
 *     output buffers are owned and sized by the caller.
 *   - All device work runs on the handle's CUDA stream, in stream order.
 *     Calls that hand results to the caller (host values, caller buffers)
 *     return after that work is complete.  dfl_static, dfl_apply_batch,
 *     dfl_update, dfl_louvain_from and the group forms return once their
 *     host-side decisions are made (the batch validated, convergence
 *     decided); device work they queued last
 *     may still be running on the stream, ordered before the handle's next
 *     call -- a caller reading device state directly must order its work
 *     after the handle's stream.  A handle must not be used from two threads
 *     at once.
 *   - The computation is deterministic: the same inputs give the same
 *     membership, K, Sigma and modularity on every run.
 *
 * Local-moving schedule (the paper's own is asynchronous; this library fixes
 * a deterministic one): each iteration visits the frontier in `substeps`
 * hash classes (class of vertex i = top bits of i * 0x9E3779B1 mod 2^32);
 * the vertices of one class decide together against the state left by the
 * previous class, then their moves are applied at once.  A vertex moves to
 * the neighbour community with the largest 2m*K_{i->c} - K_i*Sigma_c (ties to
 * the smallest id) if that beats staying (delta-modularity > 0, Eq. 2), except
 * that a singleton never moves into a singleton community with a larger id.
 * The per-iteration tolerance test on the summed delta-modularity is exact.
 */
#ifndef DFL_H
#define DFL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle: graph, K, Sigma, 2m, membership and work buffers, all owned
 * by the library and released by dfl_destroy. */
typedef struct dfl_handle dfl_handle;

/* One undirected edge of a batch, given once (the library adds both arcs).
 * For a deletion, w = 0 removes the whole edge and w > 0 removes that much
 * weight; for an insertion, w > 0 is added to the edge (created if absent). */
typedef struct {
  uint32_t u, v, w;
} dfl_edge;

enum { DFL_ND = 0, DFL_DS = 1, DFL_DF = 2 };
enum { DFL_MEM_HOST = 0, DFL_MEM_DEVICE = 1 };

enum {
  DFL_OK = 0,
  DFL_ERR_INVALID = -1,   /* bad argument: vertex id >= n, self-loop, zero insert
                             weight, an edge deleted twice in one call, a
                             non-symmetric / unsorted / duplicated input CSR */
  DFL_ERR_NOT_FOUND = -2, /* deletion of an absent edge, or of more weight than present */
  DFL_ERR_OVERFLOW = -3,  /* an edge weight would exceed 2^32-1, or 2m would reach 2^32 */
  DFL_ERR_NOMEM = -4,     /* device or pinned host allocation failed */
  DFL_ERR_CUDA = -5,      /* a CUDA runtime call failed */
  DFL_ERR_TIMEOUT = -6,   /* a bounded device wait gave up (DFL_FLAG_PERSISTENT) */
  DFL_ERR_STATE = -7      /* call out of order, e.g. dfl_update before dfl_static */
};

/* Option flags. */
enum {
  DFL_FLAG_PROFILE = 1u, /* time every kernel class with CUDA events (dfl_profile) */
  DFL_FLAG_TRACE = 2u,   /* reserved */
  DFL_FLAG_NO_GRAPH = 4u, /* launch every kernel from the host (overrides DFL_FLAG_GRAPH) */
  DFL_FLAG_SERIAL_BINS = 8u, /* run the degree bins of a sub-step one after another on the handle's
                                stream instead of concurrently (for measuring each bin alone) */
  DFL_FLAG_PERSISTENT = 16u,  /* run each local-moving iteration as one cooperative launch whose
                                 blocks meet at bounded grid barriers between sub-steps; a barrier
                                 that waits about a second gives up and the call returns
                                 DFL_ERR_TIMEOUT (the handle should then be destroyed).  On a
                                 device without cooperative launch, or where fewer than 4 blocks
                                 of the kernel fit at once, the per-bin kernels run instead (same
                                 results) */
  DFL_FLAG_GRAPH = 32u,       /* always replay each first-pass local-moving iteration as a
                                 captured CUDA graph (needs a handle stream other than the legacy
                                 default stream).  Without this flag or DFL_FLAG_NO_GRAPH, replay
                                 is used except for group handles and for DF/DS updates of fewer
                                 than 256 batch edges, which launch from the host with the list
                                 lengths read (empty bins skipped, grids fit to the work) */
  DFL_FLAG_PROFILE_MOVE = 64u, /* time only the decide phase of each sub-step (two CUDA events per
                                 sub-step, the DFL_PROF_MOVE class of dfl_profile): the cheap
                                 subset of DFL_FLAG_PROFILE */
  DFL_FLAG_RECOMPUTE_AUX = 128u, /* the ablation of Section 4.2: every dfl_update / dfl_group_update
                                 first recomputes K from the graph and Sigma (and 2m) from K and
                                 the memberships, as a dynamic method without auxiliary
                                 information must.  Results are identical; the extra time is
                                 what reusing K^{t-1} and Sigma^{t-1} saves.  (The batch apply
                                 still updates K and Sigma incrementally, fused into its kernels.) */
  DFL_FLAG_TEST_UNREACHABLE_BARRIER = 256u /* test hook, no counterpart in the paper: with
                                 DFL_FLAG_PERSISTENT, every grid barrier of the iteration kernel
                                 waits for one more block than the grid has (a wait nothing
                                 completes) and gives up after a few milliseconds instead of
                                 about a second; every block then returns, and the call returns
                                 DFL_ERR_TIMEOUT.  For testing the timeout path without a fault */
};

/* Algorithm options; defaults from Section 5.1.2 of the paper. */
typedef struct {
  uint32_t max_iterations; /* MAX_ITERATIONS per pass, default 20 */
  uint32_t max_passes;     /* MAX_PASSES, default 10 */
  uint64_t tau_num;        /* iteration tolerance tau = tau_num / tau_den, default 1/100 */
  uint64_t tau_den;
  uint64_t tolerance_drop; /* tau is divided by this after every pass, default 10 */
  double tau_agg;          /* aggregation tolerance: passes stop when communities exceed tau_agg
                              of the current graph's vertices (Alg. 4); default 0.8, 1.0
                              disables the test */
  uint32_t substeps;       /* synchronous sub-steps per iteration: 1, 2, 4 (default) or 8 */
  uint32_t flags;          /* DFL_FLAG_* */
} dfl_options;

/* Statistics of the last dfl_static / dfl_update. */
typedef struct {
  uint32_t passes;             /* Louvain passes executed */
  uint32_t iterations[16];     /* local-moving iterations of each pass (first 16) */
  uint64_t affected_initial;   /* vertices in the initial frontier */
  uint64_t affected_ever;      /* vertices processed at least once in the first pass */
  uint64_t kernel_launches;    /* kernels launched by this handle since creation */
  uint64_t num_arcs;           /* arcs of the current graph G^t (2 per edge) */
  uint64_t arc_pool;           /* arc slots allocated for the slack CSR */
  uint32_t max_degree;         /* largest vertex degree of G^t (upper bound) */
  uint32_t num_communities;    /* distinct labels of the last first-pass membership */
  uint64_t graph_captures;     /* local-moving iteration graphs captured since creation */
  double graph_capture_ms;     /* host time spent capturing and instantiating them */
} dfl_stats_t;

/* Per kernel class timing and algorithmic traffic (DFL_FLAG_PROFILE). */
enum {
  DFL_PROF_APPLY = 0,   /* batch apply, K/Sigma update */
  DFL_PROF_MARK = 1,    /* initial frontier marking */
  DFL_PROF_MOVE = 2,    /* local-moving decide phase of each sub-step: wall time from the
                           first to the end of the last (concurrent) decide kernel */
  DFL_PROF_COMMIT = 3,  /* local-moving move-apply kernels */
  DFL_PROF_AGG = 4,     /* renumbering and aggregation */
  DFL_PROF_OTHER = 5,
  DFL_PROF_BIN0 = 6,    /* decide kernels by degree bin (<= 32, <= 256, <= 4096, larger); */
  DFL_PROF_BIN1 = 7,    /* these run concurrently inside the DFL_PROF_MOVE wall time */
  DFL_PROF_BIN2 = 8,
  DFL_PROF_BIN3 = 9,
  DFL_PROF_CLASSES = 10
};
typedef struct {
  uint64_t launches[DFL_PROF_CLASSES];
  double ms[DFL_PROF_CLASSES];         /* summed kernel durations (CUDA events) */
  uint64_t bytes[DFL_PROF_CLASSES];    /* algorithmic bytes: for the decide phase, per
                                          processed vertex 24 + 12*deg + 12*candidates, plus
                                          16 + 4*deg per mover */
} dfl_profile_t;

/* Fill *opt with the defaults above. */
void dfl_default_options(dfl_options* opt);

/* Create a handle from a symmetric CSR graph (Section 3: undirected, both
 * arcs of every edge present with equal weights).  offsets[n+1] (uint64),
 * indices[nnz], weights[nnz]; rows must be sorted by neighbour id with no
 * duplicates and no self-loops; nnz = offsets[n].  The graph is copied into
 * a slack CSR on the device; communities are not computed (call dfl_static).
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream); opt may
 * be NULL for defaults.  n must be below 2^31. */
int dfl_create(dfl_handle** out, uint32_t n, const uint64_t* offsets, const uint32_t* indices,
               const uint32_t* weights, uint64_t nnz, int mem_kind, const dfl_options* opt,
               void* cuda_stream);

/* Release every device and host resource of the handle (NULL is a no-op).
 * Resource lifetime of this library; the paper has no counterpart. */
void dfl_destroy(dfl_handle* h);

/* Replace the options (Section 5.1.2's parameters and the flags above) or
 * the stream (the stream change is stream-ordered: the caller must make the
 * new stream wait for the old one if needed; streams have no counterpart in
 * the paper). */
int dfl_set_options(dfl_handle* h, const dfl_options* opt);
int dfl_set_stream(dfl_handle* h, void* cuda_stream);

/* Static Louvain (the paper's "Static" baseline, GVE-Louvain): K from
 * scratch, every vertex its own community, every vertex affected.  Clears
 * the pending batch.  If it fails part-way (DFL_ERR_NOMEM, DFL_ERR_TIMEOUT)
 * the handle keeps its graph and K but has no communities until a later
 * dfl_static or dfl_set_membership succeeds (the same holds for
 * dfl_update). */
int dfl_static(dfl_handle* h);

/* Apply a batch update (Section 3.4): deletions first, then insertions,
 * each edge given once.  Updates the graph, K, Sigma (with the current
 * membership C^{t-1}, Alg. 7) and 2m immediately, and appends the batch to
 * the pending list consumed by the next dfl_update.  Several calls may
 * precede one dfl_update.  Requires dfl_static first (DFL_ERR_STATE).
 * Errors (nothing is changed): DFL_ERR_INVALID, DFL_ERR_NOT_FOUND,
 * DFL_ERR_OVERFLOW; if several apply, INVALID is reported before NOT_FOUND
 * before OVERFLOW. */
int dfl_apply_batch(dfl_handle* h, const dfl_edge* del, uint64_t n_del, const dfl_edge* ins,
                    uint64_t n_ins, int mem_kind);

/* Update the communities for the pending batch with DFL_ND (Alg. 2),
 * DFL_DS (Alg. 3) or DFL_DF (Alg. 1); runs Louvain (Alg. 4-6) from the
 * current membership and clears the pending list. */
int dfl_update(dfl_handle* h, int mode);

/* One step of a dynamic method (Section 4.2's f(G^{t-1}, Delta^{t-}, Delta^{t+},
 * C^{t-1}, K^{t-1}, Sigma^{t-1})): dfl_apply_batch of (del, ins) followed by
 * dfl_update(mode), with the same results, arguments and errors as those two
 * calls.  With DFL_DF the update is queued on the stream behind the apply
 * before the host has read the apply's validation; the update's first
 * control read settles both, so the step makes one host wait fewer, and
 * none between the apply's validation and its writes.  If the batch is
 * invalid (DFL_ERR_INVALID, DFL_ERR_NOT_FOUND, DFL_ERR_OVERFLOW) nothing
 * changes: graph, K, Sigma, 2m, membership and any earlier pending batches
 * stay as they were (the queued update marks no vertex).  Other modes, and
 * DFL_FLAG_RECOMPUTE_AUX, run the two calls one after the other.  Errors of
 * the update part leave the handle as a failed dfl_update does. */
int dfl_step(dfl_handle* h, const dfl_edge* del, uint64_t n_del, const dfl_edge* ins, uint64_t n_ins,
             int mem_kind, int mode);

/* Membership C^t (n uint32 labels in [0, n)): the community of every
 * vertex that Alg. 1 (DF), Alg. 2 (ND) and Alg. 3 (DS) return, obtained by
 * Alg. 4's final dendrogram lookup (the last pass's labels, not renumbered);
 * after dfl_static, the result of static Louvain.  out: n entries in memory
 * of kind mem_kind, owned by the caller.  DFL_ERR_STATE before dfl_static. */
int dfl_membership(const dfl_handle* h, uint32_t* out, int mem_kind);

/* Modularity of the current membership (Eq. 1): Q = (2m*sum_c sigma_c -
 * sum_c Sigma_c^2) / (2m)^2, computed exactly in integers and converted once
 * to double (0 when 2m = 0).  parts (optional, may be NULL) receives the
 * numerator and denominator as {num_hi, num_lo, den_hi, den_lo}. */
int dfl_modularity(dfl_handle* h, double* q, int64_t* parts);

/* The auxiliary information of Section 4.2 that Alg. 1 returns beside C^t:
 * K^t (n weighted degrees, Alg. 7's incremental update of K^{t-1}), Sigma^t
 * (n community totals, indexed by community label, for the membership
 * dfl_membership reports) and 2m (the sum of K).  Any pointer may be NULL;
 * K and Sigma are caller buffers of n int64 in memory of kind mem_kind,
 * two_m is a host value. */
int dfl_weights(dfl_handle* h, int64_t* K, int64_t* Sigma, int64_t* two_m, int mem_kind);

/* Number of arcs of G^t, and G^t as a compact CSR with sorted rows
 * (offsets n+1, indices and weights num_arcs). */
/* Rewrite the arc pool densely.  Rows that outgrow their slot move to the
 * end of the pool and leave the old slot behind, so a long stream of
 * batches only ever grows it; this gives every row a fresh slot of slack
 * capacity for its live arcs (tombstones dropped; the live part of the
 * sorted prefix kept in order, then the live tail).  The graph, membership,
 * K, Sigma and pending batches are unchanged, and so is every later result.
 * before / after (optional, out): arc slots of the pool before and after.
 * Allocates the new pool before freeing the old (DFL_ERR_NOMEM leaves the
 * handle unchanged); synchronizes the stream.  Works on group handles. */
int dfl_compact(dfl_handle* h, uint64_t* before, uint64_t* after);

/* G^t after the batches applied so far (Section 3.4: G^{t-1} with
 * Delta^{t-} removed and Delta^{t+} added): the arc count, and the graph as
 * a compact CSR with rows sorted by neighbour (offsets n+1, indices and
 * weights num_arcs entries, caller buffers in memory of kind mem_kind). */
int dfl_num_arcs(dfl_handle* h, uint64_t* num_arcs);
int dfl_graph(dfl_handle* h, uint64_t* offsets, uint32_t* indices, uint32_t* weights,
              int mem_kind);

/* Statistics of the last dfl_static / dfl_update (dfl_stats_t above): the
 * passes of Alg. 4, the iterations l_i of Alg. 5 in each pass, the size of
 * the initial frontier (Alg. 1-3's initially affected vertices) and the
 * vertices processed at least once in the first pass (the affected-vertex
 * counts compared in Section 5.2.3).  *s is a host struct. */
int dfl_stats(dfl_handle* h, dfl_stats_t* s);

/* Timings and algorithmic bytes per kernel class accumulated since the last
 * reset (only with DFL_FLAG_PROFILE).  Synchronizes the stream. */
int dfl_profile(dfl_handle* h, dfl_profile_t* p, int reset);

/* First-pass trace of the last Louvain run: for each iteration
 * {vertices processed, vertices moved, S_hi, S_lo} where S is the sum of the
 * movers' numerators 2m^2 * dQ (Eq. 2).  Returns the iteration count in
 * *len; writes at most cap iterations. */
int dfl_trace(dfl_handle* h, uint64_t* out, uint32_t cap, uint32_t* len);

/* Message of the last error on this handle ("" if none; "no handle" for
 * NULL).  The string is owned by the handle and valid until its next call.
 * Error reporting of this library; the paper has no counterpart. */
const char* dfl_last_error(const dfl_handle* h);

/* ---- Inspection entry points used by the parity tests ------------------ */

/* Replace the membership; K, Sigma, community sizes and 2m are recomputed
 * from the graph and the pending batch is cleared.  With dfl_graph,
 * dfl_membership and dfl_get_tuning this makes a checkpoint: between
 * updates those three record everything later updates depend on, and
 * dfl_create, dfl_set_tuning and dfl_set_membership restore it exactly. */
int dfl_set_membership(dfl_handle* h, const uint32_t* C, int mem_kind);

/* Initial frontier and affected range (one byte per vertex) that `mode`
 * would use for the pending batch, without running Louvain. */
int dfl_mark(dfl_handle* h, int mode, uint8_t* F, uint8_t* R, int mem_kind);

/* Run Louvain from the current membership with an explicit initial
 * frontier F0 and first-pass range R0 (one byte per vertex). */
int dfl_louvain_from(dfl_handle* h, const uint8_t* F0, const uint8_t* R0, int mem_kind);

/* One local-moving iteration (all sub-steps) on G^t: F (in: frontier, out:
 * next frontier), R range, moved (out: 1 for movers), dq = {S_hi, S_lo}. */
int dfl_move_iteration(dfl_handle* h, uint8_t* F, const uint8_t* R, uint8_t* moved,
                       int64_t* dq, int mem_kind);

/* Aggregate G^t with the current membership renumbered by ascending label
 * (Alg. 6) and export the super-vertex graph as CSR with rows sorted by
 * neighbour.  With offsets == NULL only *nv and *na are written. */
int dfl_aggregate(dfl_handle* h, uint32_t* nv, uint64_t* na, uint64_t* offsets,
                  uint32_t* indices, uint64_t* weights);

/* ---- Kernel tuning ------------------------------------------------------ */

/* Launch-shape choices of the local-moving step.  They change which kernel
 * decides a vertex and where its community table lives, never the result:
 * any valid tuning gives the same membership, K, Sigma and modularity.
 *   degree <= bin_warp:       W = bin_warp rounded up to a power of two (>= 4)
 *                             lanes per vertex, 32/W vertices per warp,
 *                             communities grouped in registers
 *   degree <= bin_warp_hash:  one warp (registers up to 32 arcs, else an
 *                             open-addressing table in shared memory)
 *   degree <= bin_block:      one block of block_threads, shared-memory table
 *                             (global-memory slice when it overflows)
 *   larger:                   split into 1024-arc chunks, one block each,
 *                             summed in a global table of the vertex; its
 *                             last chunk block (or, for many distinct
 *                             communities, a block per 2048 of them) decides
 * Valid ranges: bin_warp <= 32, bin_warp <= bin_warp_hash <= 256,
 * bin_warp_hash <= bin_block, block_threads in {128, 256, 512}.
 * Defaults: 8, 256, 4096, 256. */
typedef struct {
  uint32_t bin_warp;
  uint32_t bin_warp_hash;
  uint32_t bin_block;
  uint32_t block_threads;
} dfl_tuning;

int dfl_get_tuning(const dfl_handle* h, dfl_tuning* t);
int dfl_set_tuning(dfl_handle* h, const dfl_tuning* t); /* DFL_ERR_INVALID if out of range */

/* Autotuner: marks the initial frontier that dfl_update(mode) would use for
 * the pending batch (every vertex for DFL_ND), then times one local-moving
 * iteration's decide phase over it (CUDA events, median of `reps`) for
 * candidate tunings by coordinate descent over block_threads, bin_block,
 * bin_warp_hash and bin_warp, starting from the current tuning.  Decisions
 * are computed but not applied, so the graph, membership and pending batch
 * are unchanged; the fastest tuning is set on the handle and written to
 * *chosen (may be NULL).  *ms (may be NULL) receives its median time. */
int dfl_autotune(dfl_handle* h, int mode, uint32_t reps, dfl_tuning* chosen, double* ms);

/* ---- Groups: many independent graphs in one handle --------------------- */

/* A group holds G independent graphs in one handle, laid out as their
 * disjoint union (graph g's vertices are a contiguous range), so that every
 * step of an update -- batch apply, marking, each local-moving sub-step,
 * aggregation -- is one launch over all graphs.  Each graph keeps its own
 * 2m, tolerance test, iteration and pass counts and aggregation decision
 * (Alg. 4-5 per graph): every graph gets exactly the membership, K, Sigma
 * and modularity that a handle of its own would, with labels in [0, n_g).
 * A graph that converges stops being processed while the others continue.
 * Each graph's 2m must stay below 2^32; the group's total need not.
 *
 * dfl_group_create: G graphs, graph g given as symmetric CSR (the
 * dfl_create rules) offsets[g] (n[g]+1 entries), indices[g], weights[g],
 * all in HOST memory.  The sum of n[g] must be below 2^31.  The returned
 * handle works with dfl_destroy, dfl_set_options, dfl_set_stream,
 * dfl_profile, dfl_get/set_tuning, dfl_autotune and dfl_membership (labels
 * of the union, graph g's in [start_g, start_g + n_g)); dfl_static,
 * dfl_apply_batch, dfl_update and dfl_modularity return DFL_ERR_STATE on it. */
int dfl_group_create(dfl_handle** out, uint32_t num_graphs, const uint32_t* n,
                     const uint64_t* const* offsets, const uint32_t* const* indices,
                     const uint32_t* const* weights, const dfl_options* opt, void* cuda_stream);

/* Static Louvain of every graph of the group. */
int dfl_group_static(dfl_handle* h);

/* One batch per graph: graph g's deletions are del[del_off[g] .. del_off[g+1])
 * and its insertions ins[ins_off[g] .. ins_off[g+1]), with vertex ids local
 * to graph g (del_off and ins_off have num_graphs + 1 entries, in HOST
 * memory; del and ins in memory of kind mem_kind).  The batches are applied
 * together (dfl_apply_batch rules per graph); on any error nothing changes.
 * DFL_ERR_OVERFLOW also if a graph's 2m plus twice its inserted weight would
 * reach 2^32. */
int dfl_group_apply_batch(dfl_handle* h, const dfl_edge* del, const uint64_t* del_off,
                          const dfl_edge* ins, const uint64_t* ins_off, int mem_kind);

/* Update every graph for its pending batch (mode as in dfl_update). */
int dfl_group_update(dfl_handle* h, int mode);

/* Membership of graph g (n_g labels in [0, n_g)). */
int dfl_group_membership(dfl_handle* h, uint32_t g, uint32_t* out, int mem_kind);

/* Modularity of graph g (as dfl_modularity). */
int dfl_group_modularity(dfl_handle* h, uint32_t g, double* q, int64_t* parts);

/* Statistics of graph g for the last dfl_group_static / dfl_group_update
 * (passes, iterations, num_communities; the launch, arc and capture
 * counters are the group's). */
int dfl_group_stats(dfl_handle* h, uint32_t g, dfl_stats_t* s);

/* ---- Test hooks (host-side fault injection; no counterpart in the paper) -- */

/* Make device allocations fail, process-wide: after `after` more successful
 * allocations every further device allocation of the library fails as if
 * the GPU were out of memory (the call returns DFL_ERR_NOMEM); `after` < 0
 * lifts it.  Nothing is allocated for the failed requests.  What an
 * allocation failure leaves (also for a real out-of-memory): dfl_create
 * returns no handle; dfl_apply_batch and dfl_group_apply_batch leave the
 * graph, K, Sigma, 2m and the pending batches unchanged; dfl_static,
 * dfl_update and their group forms keep the graph and K but no communities
 * (calls that need them return DFL_ERR_STATE) until dfl_static, or
 * dfl_set_membership, succeeds.  It applies to every handle of the process. */
int dfl_test_fail_allocations(int64_t after);

/* ---- Allocation-free entry point --------------------------------------- */

/* Largest vertex count accepted by dfl_modularity_csr_noalloc. */
#define DFL_NOALLOC_MAX_VERTICES (1u << 20)

/* Modularity Q of a caller-supplied graph and membership, computed without
 * allocating any memory (no cudaMalloc, cudaFree or allocating library call).
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run it -- e.g. a service whose
 * device memory is owned by another allocator or fixed at start-up, or a
 * latency-critical path where cudaMalloc/cudaFree would block or synchronize
 * the device.  It computes the same Q, numerator and denominator as
 * dfl_modularity does for a handle holding that graph and membership.
 *   n: vertices, at most DFL_NOALLOC_MAX_VERTICES (else DFL_ERR_INVALID)
 *   offsets[n+1] (uint64), indices[nnz], weights[nnz]: symmetric CSR in DEVICE
 *   memory (both arcs of every edge); offsets must be non-decreasing and
 *   offsets[n] = nnz, the length of indices and weights (decreasing offsets
 *   give DFL_ERR_INVALID; offsets beyond the arrays cannot be detected and
 *   make the call read out of bounds); membership[n]: DEVICE memory, labels < n
 *   q: HOST output; parts: optional HOST output {num_hi, num_lo, den_hi, den_lo}
 *   cuda_stream: cudaStream_t the work is ordered on; returns when it is done.
 * Errors: DFL_ERR_INVALID (n too large, a label or neighbour id >= n,
 * decreasing offsets, null pointer), DFL_ERR_OVERFLOW (2m >= 2^32),
 * DFL_ERR_CUDA.
 * Its scratch (8 MiB of per-community totals plus a few counters) is a fixed
 * array in the library's device memory, held by every GPU that loads the
 * library until the process exits, and shared by all calls: each call clears
 * it first, but calls whose GPU work overlaps race and must be serialized.
 * The first call on a device also looks up that array's device address with
 * the device current and remembers it for the life of the process, by device
 * ordinal: after a cudaDeviceReset of that device the remembered address is
 * stale and the entry point must not be called.  Under CUDA's lazy module
 * loading that first call also loads the library's device code, which
 * allocates the fixed array and may synchronize the device: make it once,
 * outside any stream capture and any latency-critical path, before relying
 * on the call allocating nothing. */
int dfl_modularity_csr_noalloc(uint32_t n, const uint64_t* offsets, const uint32_t* indices,
                               const uint32_t* weights, const uint32_t* membership, double* q,
                               int64_t* parts, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DFL_H */
