// Internal declarations of libkbisim: device helpers, the device graph store
// and the per-round driver.  Not part of the public ABI (see include/kbisim.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kbisim.h"

namespace kb {

// ---------------------------------------------------------------------------
// Constants
// ---------------------------------------------------------------------------
constexpr uint64_t kEmpty64 = 0xFFFFFFFFFFFFFFFFull;  // empty hash slot
constexpr uint32_t kNone32 = 0xFFFFFFFFu;
constexpr uint32_t kDead = KBISIM_DELETED;

// Degree classes of the signature kernels.
constexpr int kSmallMax = 64;      // out-degree <= 64: one thread per node, keys in registers
constexpr int kWarpMax = 256;      // class bounds above kSmallMax (65..256, 257..1024, 1025..4096):
constexpr int kWarp2Max = 1024;    //   node ordering only; all three run as CTA chunks of whole
constexpr int kBlockMax = 4096;    //   nodes (at most kChunkEdges edges per chunk)
constexpr int kChunkThreads = 512; // threads of the chunk kernels for out-degree > kWarp2Max and hubs
constexpr int kSmallChunkThreads = 128;  // threads of the chunk kernel for out-degree kSmallMax+1..kWarp2Max
constexpr int kChunkItems = 8;     // edges per thread
constexpr int kChunkEdges = kChunkThreads * kChunkItems;  // 4096 = kBlockMax
constexpr int kChunkMaxNodes = 64; // nodes per medium chunk (each has > kSmallMax edges)
constexpr int kHubChunk = kChunkEdges;  // hub edges per chunk CTA
constexpr int kSmallClasses = 8;        // out-degree 0, 1, 2, 3-4, 5-8, 9-16, 17-32, 33-64
constexpr int kClassWarp = kSmallClasses, kClassWarp2 = kSmallClasses + 1, kClassBlock = kSmallClasses + 2,
              kClassHub = kSmallClasses + 3, kClassDead = kSmallClasses + 4;
constexpr int kNumClasses = kSmallClasses + 5;  // including deleted nodes (last)
static_assert(kChunkEdges >= kBlockMax, "a medium node must fit one chunk");
static_assert(kChunkEdges / (kSmallMax + 1) < kChunkMaxNodes, "chunk node table too small");
static_assert(kSmallChunkThreads * kChunkItems >= kWarp2Max, "a node of out-degree <= kWarp2Max must fit one small chunk");

// Degree class of a node of out-degree d: 0, 1, 2, 3-4, 5-8, 9-16, 17-32,
// 33-64, then 65..kWarpMax, ..kWarp2Max, ..kBlockMax, hubs.
__host__ __device__ __forceinline__ int degree_class_of(uint64_t d) {
  if (d == 0) return 0;
  if (d <= (uint64_t)kSmallMax) {
    int c = 1;
    while ((1ull << (c - 1)) < d) ++c;
    return c;
  }
  if (d <= (uint64_t)kWarpMax) return kClassWarp;
  if (d <= (uint64_t)kWarp2Max) return kClassWarp2;
  if (d <= (uint64_t)kBlockMax) return kClassBlock;
  return kClassHub;
}

// Device error flags (bit set in Store::d_err).
enum : uint32_t {
  kErrChecked = 1u,       // an index check failed
  kErrProbe = 2u,         // a hash probe sequence ran past its bound
  kErrHubOverflow = 4u,   // a hub bucket received more key words than its capacity
  kErrHubSet = 16u,       // a hub bucket held more distinct keys than its shared set
  kErrBadInput = 8u,      // input validation failed (ids, offsets)
};

// ---------------------------------------------------------------------------
// Mixing functions.  mix64 is the output function of SplitMix64 (Steele, Lea
// and Flood, OOPSLA 2014, with Vigna's constants); mix32 is the 32-bit
// finalizer of MurmurHash3 (Appleby).  Both are bijections: xor-shifts and
// multiplications by odd constants are invertible.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// A signature element (edge label, child identifier) as one word of type K.
// The pair is packed one-to-one -- (label << pbits) | pid with 32-bit words
// when label and pid fit, (label << 32) | pid with 64-bit words otherwise --
// and then passed through a bijective mix, so equal words <=> equal elements.
// A node's signature set is stored as its distinct words in arbitrary order
// (sets are compared as sets); the mix spreads the words uniformly, which the
// hash sets and the hub buckets rely on for balance.  The 32-bit mix is a
// multiplication by an odd constant (every input bit reaches the high bits,
// which pick set regions and hub buckets) followed by folding the high half
// into the low half (which pick home slots in power-of-two sets).
template <typename K>
struct KeyOps;

template <>
struct KeyOps<uint32_t> {
  static constexpr uint32_t kEmpty = 0xFFFFFFFFu;
  static constexpr int kBits = 32;
  __device__ __forceinline__ static uint32_t make(uint32_t label, uint32_t pid, int pbits) {
    const uint32_t x = ((label << pbits) | pid) * 0x9e3779b1u;
    return x ^ (x >> 16);
  }
};

template <>
struct KeyOps<uint64_t> {
  static constexpr uint64_t kEmpty = 0xFFFFFFFFFFFFFFFFull;
  static constexpr int kBits = 64;
  __device__ __forceinline__ static uint64_t make(uint32_t label, uint32_t pid, int) {
    return mix64(((uint64_t)label << 32) | (uint64_t)pid);
  }
};

// Per-element hash term.  A set's term sum adds the two 32-bit halves of the
// terms separately (each modulo 2^32), so kernels can accumulate it with
// 32-bit adds in any order.  64-bit words: the SplitMix64 output function of
// (key + seed).  32-bit words, which are already the output of a mixing
// bijection of (label, identifier): the low half is the word plus half of the
// seed, the high half the word times (word xor the other half of the seed,
// made odd), so the two halves of a set's sum are its first moment and a
// quadratic one.  Three integer operations instead of two 32-bit mixes; the
// hash only routes nodes to candidate groups, and equality is always decided
// by exact comparison.
template <typename K>
__host__ __device__ __forceinline__ uint64_t elem_term(K key, uint64_t seed) {
  return mix64((uint64_t)key + seed);
}
__host__ __device__ __forceinline__ uint64_t elem_term(uint32_t key, uint64_t seed) {
  return ((uint64_t)(key * ((key ^ (uint32_t)(seed >> 32)) | 1u)) << 32) | (key + (uint32_t)seed);
}

// Sum of two packed term sums, half by half.
__host__ __device__ __forceinline__ uint64_t term_add(uint64_t acc, uint64_t t) {
  return (uint64_t)((uint32_t)acc + (uint32_t)t) | ((uint64_t)((uint32_t)(acc >> 32) + (uint32_t)(t >> 32)) << 32);
}

// Hash of a node's signature from its parts.  Never returns kEmpty64.
__host__ __device__ __forceinline__ uint64_t node_hash(uint64_t term_sum, uint32_t first,
                                                       uint64_t count, uint64_t seed,
                                                       uint64_t mask) {
  uint64_t h = mix64(term_sum + (uint64_t)first * 0xc2b2ae3d27d4eb4full + count * 0x165667b19e3779f9ull + seed);
  h &= mask;
  return h == kEmpty64 ? kEmpty64 - 1 : h;
}

// ---------------------------------------------------------------------------
// Device buffers
// ---------------------------------------------------------------------------
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

struct KernelTimer;  // per-kernel CUDA event timing (kbisim_round.cu)

// Batched build state (kbisim_many.cu): graph j of the batch owns original
// ids start[j] .. start[j+1]-1 of the loaded union.
struct ManyState {
  bool valid = false;
  uint32_t G = 0;
  std::vector<uint64_t> start;                 // [G+1]
  std::vector<uint32_t> k;                     // [G]
  std::vector<uint32_t> rounds;                // [G] per-graph rounds (own early stop)
  std::vector<std::vector<uint64_t>> counts;   // [level][G] per-graph block counts
  uint32_t levels = 0;                         // union levels renumbered per graph
  std::vector<Buf> lvl;                        // per level: uint32 [n] per-graph ids, original order
  Buf dstart;                                  // uint64 [G+1]
  Buf gid, gidp;                               // uint32 [n] graph of each original / internal node
  Buf tkey, tmin, slot;                        // (graph, union block) -> smallest original id
  Buf hbits, hword, cnt;                       // head bitmap, per-word prefix, per-graph prefix
  Buf live, live_mask;                         // uint8 [G] graph still refined; bitmap over internal ids
  uint64_t live_graphs = 0;                    // graphs refined in the next round
};

}  // namespace kb

#include "kbisim_maint_state.cuh"  // MaintLevel, MaintState

namespace kb {

struct Store;
struct Status;
using LevelHook = Status (*)(Store&, uint32_t);

// The device graph store plus all scratch a round needs.  One per handle.
//
// Node ids are relabelled once per graph: internal id p orders the alive
// nodes by (degree class, original id), deleted nodes last.  The edge table
// is a CSR by source over internal ids (targets relabelled too), so every
// degree class is a contiguous range of nodes whose edges are contiguous.
// Levels are stored by internal id; copy-out restores original order.
struct Store {
  // configuration
  int device = 0;
  int sms = 1;                 // multiprocessors of the device (grid sizes)
  cudaStream_t stream = nullptr;
  uint64_t budget = 0;
  bool early_stop = true;
  uint64_t seed = 0;
  uint64_t hash_mask = ~0ull;
  bool checked = false;
  bool timing = false;

  // graph in internal ids
  uint64_t n = 0, m = 0;       // all nodes / edges
  uint64_t n_alive = 0;        // internal ids [0, n_alive) are alive
  bool has_graph = false;
  bool label8 = true;          // edge labels stored as uint8 (else uint32)
  uint32_t label_bits = 1;     // bits needed for the largest edge label
  Buf offsets;                 // uint64 [n+1]
  Buf dst;                     // uint32 [m] internal target ids
  Buf elabel;                  // uint8 or uint32 [m]
  Buf nlabel;                  // uint32 [n]
  Buf p2o;                     // uint32 [n] internal -> original id
  Buf o2p;                     // uint32 [n] original -> internal id
  bool any_dead = false;       // some node was deleted by a maintenance batch
  Buf alive_o;                 // uint8 [n] alive flags in original order (when any_dead)

  // degree classes (internal id ranges)
  uint64_t class_start[kNumClasses + 1] = {0};
  uint64_t n_hub = 0;
  Buf mid_chunks;              // uint2 (first node, node count): runs of whole nodes, three lists
  uint64_t n_mid_chunks[3] = {0, 0, 0};  // out-degree 33..64, 65..1024, 1025..4096
  Buf hub_bits;                // uint32 [n_hub]  log2(bucket count)
  Buf hub_bbase;               // uint64 [n_hub+1] first bucket of each hub
  Buf hub_cap;                 // uint32 [n_hub]  key words a bucket of this hub can hold
  Buf hub_tbase;               // uint64 [n_hub]  start of the hub's buckets in hub_tmp
  Buf hub_chunks;              // uint4 [n_chunks] (hub index, begin lo, begin hi, length)
  Buf hub_cstart;              // uint32 [n_hub + 1] first chunk of each hub
  uint64_t n_hub_chunks = 0;
  uint64_t hub_tmp_words = 0;  // key words of all hub buckets
  uint64_t n_hub_buckets = 0;
  uint64_t hub_edges = 0;
  std::vector<uint32_t> h_hub_xbits;  // per hub: more buckets, after a bucket's set filled
  std::vector<uint32_t> h_hub_shift;  // per hub: larger buckets, after a bucket's capacity was exceeded
  std::vector<uint8_t> h_hub_force;   // per hub: deduplicating chunk pass, after a scatter overflowed
  std::vector<uint64_t> h_hub_deg;

  // levels (all kept: history for extend / maintenance), internal order
  std::vector<Buf> level;
  std::vector<Buf> spare_level;  // a refinement computes into these; the levels it replaces
  Buf spare_alone;               //   come back here if it fails (and are its spares next time)
  std::vector<Buf> out_level;  // original-order copies made on demand
  std::vector<bool> out_valid;
  std::vector<uint64_t> counts;
  uint32_t computed = 0;       // highest computed level (valid if has_levels)
  bool has_levels = false;
  bool stable = false;         // computed level equals the one before it
  uint32_t k_requested = 0;
  uint32_t rounds_run = 0;
  std::vector<kbisim_round_stats> stats;  // index r-1 for round r

  // round scratch
  Buf sigkey;                  // key words [m]: distinct keys per node (any order) at its CSR offset
  Buf ucnt;                    // uint32 [n]
  Buf hash;                    // uint64 [n]
  Buf table;                   // 64-bit slots (hash fingerprint, smallest original id)
  uint64_t tcap = 0;
  Buf slot;                    // uint32 [n]
  Buf rep;                     // uint32 [n] internal id of the block head
  Buf ulist[2];                // uint32 [n] unresolved nodes (ping-pong)
  Buf hbits;                   // uint32 [(n+31)/32] head bitmap over original ids
  Buf member;                  // uint8 [n] block head has other members (this level)
  Buf alone;                   // uint8 [n] node is alone in its block at the last computed level
  Buf hword;                   // uint64 [(n+31)/32] heads before each bitmap word
  uint64_t n_alone = 0;        // nodes alone in their block at the last computed level
  Buf bsum;                    // uint64 scan block sums
  Buf long_pairs;              // uint32 [2n] (node, candidate) pairs with long signatures
  Buf hub_cursor;              // uint32 [buckets] key words appended to each bucket
  Buf bucket_hub;              // uint32 [buckets] hub of each bucket
  Buf hub_acc;                 // per hub: keys written, term sum (uint64), buckets done (uint32)
  Buf hub_mode;                // uint8 [hubs]: chunk pass of each hub this round (1 = no chunk set)
  Buf hub_force;               // uint8 [hubs]: copy of h_hub_force
  Buf hub_err;                 // uint32 [hubs]: overflow flags of the last hub pass
  Buf hub_retry;               // bitmap over internal ids: the hubs a repeated hub pass runs
  Buf hub_tmp;                 // key words [hub_tmp_words]: fixed-capacity hub buckets
  static constexpr int kStageBufsN = 9;
  Buf stage[kStageBufsN];      // staging of host inputs and COO grouping (kbisim_load)
  Buf rl_tcnt, rl_hot, rl_ost; // relabelling temporaries
  static constexpr int kUpdBufsN = 24;
  Buf upd[kUpdBufsN];          // temporaries of a maintenance batch (kbisim_update)
  static constexpr int kInplaceBufsN = 15;
  Buf inplace[kInplaceBufsN];  // a batch applied in place: claims, degrees, the other edge table
  Buf d_err;                   // uint32 error flags
  Buf d_scalars;               // uint64 [16] small device counters
  Buf h_scalars;               // pinned host mirror of d_scalars

  ManyState many;               // batched build (kbisim_build_many)
  MaintState mt;                // incremental maintenance (kbisim_update with options.maintain)
  int maintain = 1;            // options.maintain: 0 off, 1 timed choice, 2 always when it applies
  double maint_frontier_max = 0.25;  // switch back to a rebuild above this fraction of the nodes
  LevelHook level_hook = nullptr;  // called after each computed level (batched build)
  const uint32_t* round_mask = nullptr;  // nodes signed in the next round (NULL = all); the
                                         // others keep their block (batched build work list)

  // Host-side fault injection for tests (read from the environment at every
  // mutating call, see read_fault_hooks): allocations that succeed before one
  // fails (-1 = off), the round that reports a timeout (0 = off), and, in
  // checked mode only, one edge target set out of range before each round;
  // and the pool words of room a signature store is built with beyond its
  // signatures' words (smaller: the next updates grow the store).
  long fault_alloc = -1;
  uint32_t fault_timeout_round = 0;
  bool fault_corrupt_dst = false;
  uint64_t store_room = 4u << 20;

  // hub bucket size (key words at most per bucket: 2048, 4096 or 8192) and its
  // tuning: 1 = the next full round from level 2 on times both sizes and
  // keeps the faster, 2 = chosen (tuned, or fixed by options.hub_bucket_keys)
  uint32_t hub_ucap = 4096;
  int hub_tune = 1;
  bool tune_now = false;
  float hub_tune_ms[3] = {0, 0, 0};  // measured hub pass of each size (4096, 2048, 8192)

  // a load from host memory copies the edge labels on a second stream while
  // the relabelling's node phase runs; relabel_graph calls await_labels (if
  // set) before it needs them (and the label width they decide)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_copied = nullptr, ev_labels = nullptr;
  Status (*await_labels)(Store&) = nullptr;
  const unsigned int* lab_max_dev = nullptr;

  size_t bytes_held = 0;
  uint32_t busy = 0;           // scratch groups (kCache*) in use by the running call
  KernelTimer* timer = nullptr;
  double total_ms[KBISIM_KERNEL_COUNT] = {0};
  uint64_t launches[KBISIM_KERNEL_COUNT] = {0};
};

// Status carried through the host code.
struct Status {
  int code = KBISIM_OK;
  std::string msg;
  bool ok() const { return code == KBISIM_OK; }
  static Status Ok() { return Status(); }
  static Status Err(int c, const std::string& m) {
    Status s;
    s.code = c;
    s.msg = m;
    return s;
  }
};

constexpr int kStageBufs = Store::kStageBufsN;
constexpr int kUpdBufs = Store::kUpdBufsN;

// Allocation helpers (kbisim_api.cu)
Status ensure(Store& s, Buf& b, size_t bytes);
void read_fault_hooks(Store& s);
void release(Store& s, Buf& b);

// Scratch groups a handle keeps between calls (so that a call allocates and
// frees nothing in the steady state: cudaFree waits for the whole device).
// With an HBM budget, an allocation that would pass the budget first drops
// the groups no running code uses (trim_caches), then fails if it still does
// not fit.  Code that uses a group marks it with an InUse guard.
enum : uint32_t {
  kCacheStage = 1,    // stage[]: host inputs and COO grouping of a load
  kCacheUpd = 2,      // upd[]: a maintenance batch
  kCacheInplace = 4,  // inplace[]: a batch applied in place
  kCacheSpare = 8,    // spare_level / spare_alone: the levels a refinement replaces
  kCacheRelabel = 16, // rl_*: relabelling
  kCacheMaint = 32,   // the signature stores of incremental maintenance
};
struct InUse {
  Store& s;
  uint32_t bit;
  bool was;
  InUse(Store& st, uint32_t b) : s(st), bit(b), was((st.busy & b) != 0) { st.busy |= b; }
  ~InUse() {
    if (!was) s.busy &= ~bit;
  }
};
void trim_caches(Store& s);
Status cuda_check(cudaError_t e, const char* what);

// Graph preparation and round driver (kbisim_round.cu)
// Relabel a CSR given in original ids (device arrays owned by the caller;
// labels of lab_bytes each; alive0 may be null = all alive) into the store's
// internal layout.  s.n, s.m, s.label8 and s.label_bits must be set.
Status relabel_graph(Store& s, const uint64_t* off0, const uint32_t* dst0, const void* lab0,
                     const uint32_t* nlab0, const uint8_t* alive0, uint32_t lab_bytes);
// Apply a maintenance batch to the stored graph (kbisim_update.cu); leaves
// the store with the updated graph loaded and no levels.
Status apply_batch(Store& s, const kbisim_batch* b, uint64_t* missing);
Status compute_level0(Store& s);                  // pId_0 into level[0]
// Work lists of the degree classes from s.offsets (after a relabel, or after
// a batch applied in place); `fresh` drops what hub buckets learned.
Status build_chunk_lists(Store& s, bool fresh);
struct HubGrowth {
  std::vector<uint32_t> orig, xbits, shift;
  std::vector<uint64_t> deg;
  std::vector<uint8_t> force;
};
Status save_hub_growth(Store& s, HubGrowth* g);
// same_degree: a hub takes the saved growth only if its out-degree is unchanged
// (a newly loaded graph); otherwise any hub with the saved original id does
// (the same graph after an update).
Status restore_hub_growth(Store& s, const HubGrowth& g, bool same_degree);
Status compute_round(Store& s, uint32_t i);       // pId_i from pId_{i-1}
// Signatures of the nodes whose bit is set in fmask (bitmap over internal ids;
// NULL = every node) from identifiers prev (internal order), as 64-bit
// element words: each node's distinct words at its CSR offset in sigkey, its
// count in ucnt and its hash in hash (first component prev[p]).
Status masked_signatures(Store& s, const uint32_t* prev, const uint32_t* fmask);
// Group the nodes of list (internal ids) by exact signature, as left in
// sigkey / ucnt / hash by masked_signatures: rep[p] = the node of the list
// with the smallest original id that has p's signature.
Status group_list(Store& s, const uint32_t* list, uint64_t count, const uint32_t* prev);
// Write level `level` in original node order to dst (device memory).
Status unpermute_level(Store& s, uint32_t level, uint32_t* dst);
Status timer_collect(Store& s);
void timer_destroy(Store& s);
// Exclusive prefix sum of a uint64 array in place (kbisim_round.cu).
Status scan_u64(Store& s, uint64_t* a, uint64_t n);

// Incremental maintenance (kbisim_maint.cu).  maint_build makes the state for
// levels 1..k of the loaded graph from its canonical levels (which must be
// computed up to k, or be stable before).  maint_update applies a batch and
// brings levels and state up to date; *done = false means the batch was not
// applied because this path does not take it (node deletions, no state for
// k), and the caller recomputes.
Status maint_build(Store& s, uint32_t k);
Status maint_update(Store& s, const kbisim_batch* b, uint32_t k, uint64_t* missing, bool* done);
void maint_release(Store& s);     // frees the stores and their scratch
void maint_invalidate(Store& s);  // marks them stale, keeping the buffers

// Thread blocks of `kernel` (threads each, dyn_smem dynamic shared bytes) that
// are resident on all `sms` multiprocessors at once: the grid of a grid-stride
// loop, which then runs as one full wave (a larger grid that is not a whole
// number of waves leaves most multiprocessors idle in its last wave).
template <typename F>
inline unsigned resident_blocks(F kernel, int threads, size_t dyn_smem, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return (unsigned)per_sm * (unsigned)(sms > 0 ? sms : 1);
}

// Batched build (kbisim_many.cu): many_check_args before the union is loaded,
// many_setup after it, then a refinement with many_level as the level hook.
Status many_check_args(const kbisim_graph* g, const uint64_t* start, uint32_t G, const uint32_t* k,
                       uint32_t* kmax);
Status many_setup(Store& s, const uint64_t* start, uint32_t G, const uint32_t* k);
Status many_level(Store& s, uint32_t level);
void many_finish(Store& s);
Status many_pids(Store& s, uint32_t graph, uint32_t level, uint32_t* dst, bool dst_on_device);
Status many_info(const Store& s, uint32_t graph, uint32_t* rounds_run, uint64_t* counts);
void many_release(Store& s);

}  // namespace kb
