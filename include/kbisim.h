/*
 * kbisim.h -- C ABI of the GB300 k-bisimulation library (libkbisim.so).
 *
 * The library computes k-partition identifiers (Definition 2 of "External
 * memory bisimulation reduction of big graphs"): for a directed graph
 * <N, E, lambda_N, lambda_E> (Section 2.1) and k >= 0, identifiers
 * pId_0..pId_k with pId_i(u) == pId_i(v) iff u and v are i-bisimilar
 * (Definition 1).  Level 0 groups nodes by label (Algorithm 1, k = 0 branch);
 * level i > 0 groups nodes by the signature
 *     sig_i(u) = (pId_{i-1}(u), { (lambda_E(u,v), pId_{i-1}(v)) : (u,v) in E })
 * (Definition 3 and Proposition 2; using pId_{i-1}(u) rather than pId_0(u) as
 * the first component gives the same partition by Proposition 1).  Rounds stop
 * early once a level has as many blocks as the one before it (Section 3,
 * "Early stopping condition"); later levels are then equal to it.
 *
 * Numbering is canonical: on every level the blocks are numbered 0, 1, 2, ...
 * in the order of their smallest node id.  The paper allows any numbering
 * (Section 3, "Numbering schemes of partition identifier and S"); this one is
 * unique, so results can be compared bit for bit.
 *
 * Edges form a multiset of (source, label, target) triples.  Repeated triples
 * and several labels on one node pair are allowed; signatures are sets, so
 * repeats never change a partition.  Self-loops are allowed.
 *
 * All work runs in CUDA kernels on the device and stream given at creation;
 * every host call that returns results waits for that stream.  There is no
 * CPU fallback: without a usable GPU, kbisim_create fails with
 * KBISIM_ERR_CUDA.
 *
 * Conventions shared by every entry point:
 *  - Return value: KBISIM_OK (0) or one of the KBISIM_ERR_* codes below.
 *    No C++ exception crosses this boundary.  kbisim_last_error() gives a
 *    message for the last failure on a handle.
 *  - A failed kbisim_refine or kbisim_extend leaves the previous result of
 *    the handle readable and unchanged: new levels are computed into spare
 *    buffers and replace the old ones only when the call succeeds.  For
 *    kbisim_load, kbisim_build, kbisim_build_many and kbisim_update see their
 *    own comments (they replace the graph).  After KBISIM_ERR_CUDA the handle
 *    should be destroyed.
 *  - Test hooks (host-side fault injection; read from the environment at the
 *    start of each call that computes, and applied to that call only):
 *    KBISIM_FAULT_ALLOC=N makes the call's (N+1)-th device allocation fail
 *    with KBISIM_ERR_OUT_OF_MEMORY; KBISIM_FAULT_TIMEOUT_ROUND=r makes round r
 *    report KBISIM_ERR_TIMEOUT; KBISIM_FAULT_CORRUPT_DST=1 (checked mode only)
 *    sets one stored edge target to num_nodes before each round, which the
 *    checked-mode index check reports as KBISIM_ERR_CHECKED (the value is put
 *    back before the call returns); KBISIM_FAULT_STORE_ROOM=W builds the
 *    signature stores of incremental maintenance with W words of room beyond
 *    their signatures (default 4M), so that the next updates grow them.
 *  - Inputs are borrowed for the duration of the call only; the library
 *    copies what it keeps.  Results live in the handle and stay valid until
 *    the next call that loads, refines, extends or updates the handle, or
 *    until kbisim_destroy.
 *  - A handle is not thread safe: use one handle per host thread.
 */
#ifndef KBISIM_H_
#define KBISIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KBISIM_OK 0
#define KBISIM_ERR_INVALID_ARG 1   /* bad pointer, size, id or label */
#define KBISIM_ERR_OUT_OF_MEMORY 2 /* a device allocation failed */
#define KBISIM_ERR_BUDGET 3        /* the call would exceed options.hbm_budget_bytes */
#define KBISIM_ERR_CUDA 4          /* a CUDA runtime call or kernel failed */
#define KBISIM_ERR_TIMEOUT 5       /* a bounded loop gave up (table probe, hub bucket growth, collision repair) */
#define KBISIM_ERR_CHECKED 6       /* a device bounds check fired (options.checked) */
#define KBISIM_ERR_STATE 7         /* the call needs a loaded graph or computed levels */

/* Identifier of a deleted node on every level; deleted nodes are not counted. */
#define KBISIM_DELETED 0xFFFFFFFFu

/* Largest k accepted by the entry points. */
#define KBISIM_MAX_K 1024u

typedef struct kbisim_handle kbisim_handle;

typedef struct {
  /* CUDA stream (a cudaStream_t) all work is ordered on; NULL = the legacy
   * default stream of the device. */
  void *stream;
  /* CUDA device ordinal the handle uses. */
  int device;
  /* Upper bound on the device bytes the handle may hold; 0 = no bound.
   * A handle keeps its scratch between calls (so that steady-state calls
   * neither allocate nor free: cudaFree waits for the whole device).  When an
   * allocation would pass the budget, the handle first releases the scratch
   * no running step uses (staging, batch temporaries, spare levels, the
   * signature stores of maintenance, stale copy-out buffers); a call that
   * still does not fit fails with KBISIM_ERR_BUDGET before allocating. */
  uint64_t hbm_budget_bytes;
  /* 1 (default) = stop refining once a level has as many blocks as the level
   * before it; 0 = always compute k rounds.  Results are identical. */
  int early_stop;
  /* Seed of the 64-bit signature hash.  The hash only orders work: equal
   * signatures are always found by exact comparison, so results do not
   * depend on it. */
  uint64_t hash_seed;
  /* Number of signature-hash bits kept (1..64, default 64).  Values below 64
   * exist to test the exact collision handling: they make unequal
   * signatures collide on purpose.  Results do not change, only speed. */
  uint32_t hash_bits;
  /* 1 = checked mode: before a kernel indexes with a device array, a check
   * kernel verifies every index in it (edge offsets and targets, the previous
   * level's identifiers, block heads, identifiers) and the call stops with
   * KBISIM_ERR_CHECKED, without launching the kernel, if one is out of range.
   * Results are identical; each check costs one pass over the array. */
  int checked;
  /* 1 = record CUDA events around every kernel and keep per-kernel totals
   * (see kbisim_kernel_times). */
  int collect_timing;
  /* 1 (default) = kbisim_update maintains the levels incrementally (Section
   * 4, Algorithm 3): only nodes whose signature may have changed are signed
   * again, level by level, against per-level signature stores kept in the
   * handle; 0 = kbisim_update recomputes every level.  Results are identical.
   * The stores are made at the first update after a build (a cost of about
   * one signature pass per level) and take, per maintained level, about 24
   * bytes per distinct element of the stored signatures (up to one per edge:
   * the element pool keeps room for three times the stored elements, for the
   * signatures later updates add) and about 84 bytes per node (labels, and a
   * table twice as large as the number of labels).  The handle times both paths (host clock, per
   * maintained level, building the stores not included: they serve every
   * later update; the handle's first frontier update, which allocates that
   * path's scratch, is not timed): after one timed update on each, it takes
   * the frontier path only while that measured cheaper, and otherwise
   * recomputes for the next 16 updates (reason KBISIM_MAINT_COST) before
   * trying the frontier path again.
   * 2 = the frontier path whenever it applies, without timing. */
  int maintain;
  /* Key words a hub bucket holds at most (out-degree > 4096: the hub's keys
   * are split into buckets by key bits, each deduplicated by one CTA in
   * shared memory): 2048, 4096 or 8192; 0 (default) = tuned once per handle, in the
   * first full round from level 2 on, by timing the hub pass twice with 4096
   * and twice with 2048, alternating, and comparing the second passes (2048 is
   * kept only when more than 5% faster; kbisim_hub_bucket_keys reports the
   * choice).  Results do not depend on it. */
  uint32_t hub_bucket_keys;
} kbisim_options;

/* Fill *opt with the defaults (stream NULL, device 0, no budget, early stop
 * on, a fixed seed, 64 hash bits, unchecked, no timing, incremental
 * maintenance). */
void kbisim_default_options(kbisim_options *opt);

/* A graph <N, E, lambda_N, lambda_E> (Section 2.1).
 * Node ids are 0..num_nodes-1 and must be < 2^32 - 1.
 * Edges are given either in CSR form grouped by source (offsets != NULL:
 * offsets[u]..offsets[u+1] index dst/edge_label for the out-edges of u,
 * offsets[0] == 0, non-decreasing, offsets[num_nodes] == num_edges) or as
 * an unordered COO list (offsets == NULL: src[e], dst[e], edge_label[e]).
 * Edge labels have edge_label_bytes = 1, 2 or 4 bytes each (unsigned).
 * With on_device = 1 every pointer is a device pointer on the handle's device;
 * with 0 they are host pointers (pinned host memory copies faster). */
typedef struct {
  uint64_t num_nodes;
  uint64_t num_edges;
  const uint32_t *node_label; /* [num_nodes] */
  const uint64_t *offsets;    /* [num_nodes + 1] or NULL */
  const uint32_t *src;        /* [num_edges], used when offsets == NULL */
  const uint32_t *dst;        /* [num_edges] */
  const void *edge_label;     /* [num_edges] */
  uint32_t edge_label_bytes;  /* 1, 2 or 4 */
  int on_device;
} kbisim_graph;

/* Result of a call that computes levels.  block_count points into the
 * handle ([k_requested + 1] entries, host memory) and follows the handle's
 * result lifetime.  rounds_run is the number of signature rounds computed;
 * with early stop it can be below k_requested, and levels after it repeat
 * level rounds_run. */
typedef struct {
  uint32_t k_requested;
  uint32_t rounds_run;
  const uint64_t *block_count;
} kbisim_result;

/* Per-kernel device time collected when options.collect_timing = 1.
 * Indices are the KBISIM_KERNEL_* values; total_ms is the time between CUDA
 * events recorded around each group of launches of a class, launches the
 * number of this library's kernels launched in that class (counted whether or
 * not timing is on; clears done with cudaMemsetAsync are not counted). */
enum {
  KBISIM_KERNEL_LABEL_GROUP = 0, /* level 0 grouping by node label */
  KBISIM_KERNEL_SIG_SMALL,       /* signatures of out-degree <= 64 */
  KBISIM_KERNEL_SIG_MEDIUM,      /* signatures of out-degree 65..4096 */
  KBISIM_KERNEL_SIG_HUB,         /* signatures of larger out-degree (all hub kernels) */
  KBISIM_KERNEL_GROUP,           /* hash-table grouping of equal signatures */
  KBISIM_KERNEL_VERIFY,          /* exact signature comparison, marking block heads */
  KBISIM_KERNEL_RENUMBER,        /* canonical renumbering (scan of head counts + ranks) */
  KBISIM_KERNEL_OTHER,           /* clears, collision repair, copies */
  KBISIM_KERNEL_COUNT
};

typedef struct {
  double total_ms[KBISIM_KERNEL_COUNT];
  uint64_t launches[KBISIM_KERNEL_COUNT];
} kbisim_kernel_times;

/* Create a handle on options->device (NULL options = defaults).
 * Errors: INVALID_ARG (h == NULL or bad options), CUDA (no device). */
int kbisim_create(kbisim_handle **h, const kbisim_options *opt);

/* Release everything the handle holds.  NULL is ignored. */
void kbisim_destroy(kbisim_handle *h);

/* Message for the last failed call on h (never NULL; "" if none). */
const char *kbisim_last_error(const kbisim_handle *h);

/* Copy a graph into the handle (building the CSR-by-source edge table when
 * COO is given) and drop any previous graph and levels (also when the load
 * fails after validation: then the handle holds no graph).  Validates ids
 * (INVALID_ARG if a node id >= num_nodes or num_nodes >= 2^32 - 1).  A handle
 * without an HBM budget keeps its device buffers (including the staging of
 * host inputs) for the next load, so reloading graphs of similar size
 * allocates nothing; with a budget they are released and allocated again. */
int kbisim_load(kbisim_handle *h, const kbisim_graph *g);

/* Compute levels 0..k of the loaded graph (Algorithm 1, Build_Bisim).
 * Errors: STATE (no graph), INVALID_ARG (k > KBISIM_MAX_K or out == NULL),
 * OUT_OF_MEMORY, BUDGET, TIMEOUT, CHECKED, CUDA. */
int kbisim_refine(kbisim_handle *h, uint32_t k, kbisim_result *out);

/* kbisim_load followed by kbisim_refine.  If the refinement fails, the new
 * graph stays loaded without levels (KBISIM_ERR_STATE on read). */
int kbisim_build(kbisim_handle *h, const kbisim_graph *g, uint32_t k, kbisim_result *out);

/* Change k (Section 4, "Change k"): a larger k runs the missing rounds from
 * the kept levels; a smaller k only truncates.  Errors as kbisim_refine. */
int kbisim_extend(kbisim_handle *h, uint32_t k_new, kbisim_result *out);

/* A maintenance batch (Section 4: Add_Nodes, Add_Edges, deletions).  Applied
 * in this order: node additions (ids num_nodes, num_nodes+1, ... in batch
 * order, isolated, with the given labels); edge insertions (one copy of each
 * triple; endpoints must exist and not be deleted); edge deletions (one copy
 * of each listed triple; triples that are not present are ignored and
 * counted); node deletions (every incident edge is removed, then the node
 * is marked deleted).  Pointers are host or device memory per on_device. */
typedef struct {
  const uint32_t *add_node_label; uint64_t n_add_nodes;
  const uint32_t *ins_src, *ins_dst, *ins_label; uint64_t n_ins;
  const uint32_t *del_src, *del_dst, *del_label; uint64_t n_del;
  const uint32_t *del_nodes; uint64_t n_del_nodes;
  int on_device;
} kbisim_batch;

/* Apply a batch to the loaded graph and bring levels 0..k up to date, so
 * that the result equals a build of the updated graph (Theorem 2: the
 * maintained partition is the k-bisimulation of the new graph).  With
 * options.maintain the levels are maintained incrementally (Algorithm 3): the
 * frontier of level 1 is the sources of the batch's edges and the new nodes;
 * a node is signed again at level j only if it is such a source, or its own
 * level-(j-1) label changed, or a child's did; its signature is looked up in
 * the level's signature store, which keeps labels of unchanged signatures.
 * The update switches back to a full recomputation (Section 4, "When to
 * switch back to Algorithm 1") when a level's frontier holds more than a
 * quarter of the nodes (and more than 4096; later batches of at least that
 * many edges at the same k then recompute at once), when a store runs out of room, when the batch deletes
 * nodes, or when k exceeds the levels the stores hold; kbisim_update_info
 * tells which path the last update took.  *missing_deletes (may be NULL)
 * receives the number of edge deletions that named no edge.
 * Errors: STATE, INVALID_ARG (bad id, or an edge on a deleted node), and the
 * errors of kbisim_refine.  A batch that is rejected (INVALID_ARG), or whose
 * staging or matching fails (OUT_OF_MEMORY, BUDGET, TIMEOUT), leaves the graph
 * and levels unchanged.  Once the updated graph has been stored the old levels
 * no longer describe it: a failure of that step leaves no graph, and a failure
 * of the recomputation leaves the updated graph loaded without levels
 * (KBISIM_ERR_STATE on read; kbisim_refine computes them). */
int kbisim_update(kbisim_handle *h, const kbisim_batch *b, uint32_t k, kbisim_result *out,
                  uint64_t *missing_deletes);

/* How the last kbisim_update ran.  incremental = 1: the frontier path, with
 * frontier_nodes nodes signed over `levels` levels; 0: every level was
 * recomputed, for the reason in `reason` (KBISIM_MAINT_*).  The paper has no
 * counterpart: this reports which of its two paths (Algorithm 3 or a rebuild)
 * ran. */
#define KBISIM_MAINT_OFF 1        /* options.maintain = 0 */
#define KBISIM_MAINT_NO_STORE 2   /* no stores yet (first update after a build), or k above them */
#define KBISIM_MAINT_FRONTIER 3   /* a level's frontier held more than a quarter of the nodes (and > 4096) */
#define KBISIM_MAINT_CAPACITY 4   /* a signature store ran out of room */
#define KBISIM_MAINT_DELETES 5    /* the batch deletes nodes */
#define KBISIM_MAINT_COST 6       /* recomputation measured cheaper on this handle (options.maintain = 1) */
typedef struct {
  int incremental;
  int reason;
  uint64_t frontier_nodes;
  uint64_t levels;
  /* 1 = the batch was applied to the edge table in place (edge insertions and
   * deletions that keep every node in its out-degree class: node ids keep
   * their internal order); 0 = the updated graph was laid out again. */
  int in_place;
} kbisim_update_info;
int kbisim_get_update_info(const kbisim_handle *h, kbisim_update_info *out);

/* Batched build: many independent graphs refined together, one sequence of
 * kernel launches per round for all of them.  The paper has no counterpart
 * (it builds one graph at a time); each graph's result is that of
 * kbisim_build on the graph alone.  `g` holds the graphs as one graph whose
 * node ids are grouped by graph: graph j owns ids graph_start[j] ..
 * graph_start[j+1] - 1 (graph_start: host memory, num_graphs + 1 entries,
 * graph_start[0] = 0, non-decreasing, graph_start[num_graphs] =
 * g->num_nodes; empty graphs are allowed), and every edge joins two nodes of
 * one graph.  Graph j is refined to k[j] levels (host memory, num_graphs
 * entries), with the handle's early-stop setting applied to graph j's own
 * block counts.  Identifiers of graph j are canonical within graph j (blocks
 * ranked by their smallest node id, counted from graph_start[j]).  The batch
 * replaces any graph and levels held by the handle (kbisim_pids then returns
 * levels of the union of the graphs).  Errors: INVALID_ARG (num_graphs == 0,
 * bad graph_start, k[j] > KBISIM_MAX_K, an edge between two graphs), and the
 * errors of kbisim_build. */
int kbisim_build_many(kbisim_handle *h, const kbisim_graph *g, const uint64_t *graph_start,
                      uint32_t num_graphs, const uint32_t *k);

/* Level `level` (0..k[graph]) of graph `graph` of the last kbisim_build_many,
 * into dst[graph_start[graph+1] - graph_start[graph]] (host memory when
 * dst_on_device = 0).  Errors: STATE (no batched result), INVALID_ARG. */
int kbisim_many_pids(kbisim_handle *h, uint32_t graph, uint32_t level, uint32_t *dst, int dst_on_device);

/* Rounds computed for graph `graph` (its own early stop) into *rounds_run,
 * and its block counts of levels 0..k[graph] into counts (host memory,
 * k[graph] + 1 entries); either may be NULL.  Errors: STATE, INVALID_ARG. */
int kbisim_many_info(kbisim_handle *h, uint32_t graph, uint32_t *rounds_run, uint64_t *counts);

/* Copy level `level` (0..k of the last result) into dst[num_nodes]
 * (host memory when dst_on_device = 0).  A handle without an HBM budget keeps
 * an original-order copy of each level it has returned (until the levels
 * change); a handle with a budget allocates nothing here.
 * Errors: STATE, INVALID_ARG, OUT_OF_MEMORY. */
int kbisim_pids(kbisim_handle *h, uint32_t level, uint32_t *dst, int dst_on_device);

/* Device pointer to level `level` ([num_nodes] uint32), owned by the handle;
 * NULL if there is no such level.  Valid until the handle's results change. */
const uint32_t *kbisim_pids_device(kbisim_handle *h, uint32_t level);

/* Number of nodes of the loaded graph (including deleted ones). */
uint64_t kbisim_num_nodes(const kbisim_handle *h);

/* Number of edges of the loaded graph. */
uint64_t kbisim_num_edges(const kbisim_handle *h);

/* Device bytes the handle holds now (graph, levels, scratch, spares); the
 * quantity options.hbm_budget_bytes bounds.  0 for NULL. */
uint64_t kbisim_device_bytes(const kbisim_handle *h);

/* Hub bucket size in use (options.hub_bucket_keys, or the tuned choice; 4096
 * before tuning).  0 for NULL. */
uint32_t kbisim_hub_bucket_keys(const kbisim_handle *h);

/* Change the handle's HBM budget (options.hbm_budget_bytes; 0 = none) for
 * later calls.  A budget below what the handle holds now is allowed: calls
 * that would allocate fail with KBISIM_ERR_BUDGET until memory is released.
 * The paper has no counterpart (a serving loop sets it when it admits work). */
int kbisim_set_hbm_budget(kbisim_handle *h, uint64_t bytes);

/* Per-kernel device times summed since the last kbisim_reset_times(). */
int kbisim_get_kernel_times(const kbisim_handle *h, kbisim_kernel_times *out);
void kbisim_reset_times(kbisim_handle *h);

/* Statistics of the last refine, per computed round r (1-based):
 * number of distinct (label, child) keys over all nodes, largest signature
 * size, nodes whose 64-bit hash matched an unequal signature, and nodes on
 * the hub path.  Errors: STATE, INVALID_ARG (round out of range). */
typedef struct {
  uint64_t blocks;
  uint64_t unique_keys;
  uint64_t max_signature;
  uint64_t collided_nodes;
  uint64_t hub_nodes;
} kbisim_round_stats;
int kbisim_get_round_stats(const kbisim_handle *h, uint32_t round, kbisim_round_stats *out);

/* Level 0 (the label partition) for callers that cannot allocate device
 * memory -- e.g. a serving loop whose device memory is fully reserved up front
 * by another allocator, or code that must not risk the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  The paper has no counterpart:
 * it is a packaging of the level-0 step of kbisim_refine.
 * node_label [num_nodes] and pid0 [num_nodes] are device pointers on the
 * current device; block_count (device pointer, may be NULL) receives the
 * number of blocks.  pid0 equals kbisim_pids(h, 0, ...) of a handle holding a
 * graph with these labels.  Work is queued on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and the call returns without waiting.
 * Scratch lives in a fixed static device array of about 5 MB that every GPU
 * loading the library holds until exit; hence num_nodes <= 262144, and larger
 * inputs fail with KBISIM_ERR_INVALID_ARG.  No device memory is allocated or
 * freed.  All calls share the scratch array: calls that may overlap on the GPU
 * (other streams, unordered threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address;
 * make it before any stream capture.  Errors: INVALID_ARG, CUDA. */
int kbisim_label_partition_noalloc(const uint32_t *node_label, uint64_t num_nodes, uint32_t *pid0,
                                   uint32_t *block_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KBISIM_H_ */
