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
constexpr int kSmallMax = 32;      // out-degree <= 32: lanes of one warp per node
constexpr int kWarpMax = 256;      // 33..256: one warp per node, shared-memory dedupe
constexpr int kBlockMax = 4096;    // 257..4096: one CTA per node
constexpr int kBlockThreads = 512; // threads of the CTA-per-node and hub kernels
constexpr int kHubBucketTarget = 2048;  // expected distinct keys per hub bucket
constexpr int kHubUniqueCap = 4096;     // distinct keys one hub bucket can hold
constexpr int kHubChunk = 8192;         // hub edges per partition CTA (16 per thread)
constexpr int kSmallClasses = 6;        // P = 1, 2, 4, 8, 16, 32

// Device error flags (bit set in Store::d_err).
enum : uint32_t {
  kErrChecked = 1u,       // an index check failed
  kErrProbe = 2u,         // a hash probe sequence ran past its bound
  kErrHubOverflow = 4u,   // a hub bucket held more distinct keys than it can
  kErrBadInput = 8u,      // input validation failed (ids, offsets)
};

// ---------------------------------------------------------------------------
// Hashing.  mix64 is the output function of SplitMix64 (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014, with
// Vigna's constants); it is a bijection on 64-bit words.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// A signature element (edge label, child identifier) as one 64-bit word.
// pack() is one-to-one, mix64 is one-to-one, so equal words <=> equal
// elements.  Signatures are stored as the ascending sequence of these mixed
// words: a canonical order (equal sets give equal sequences) whose values are
// spread uniformly, which the bucketed sorts below rely on for balance.
__host__ __device__ __forceinline__ uint64_t elem_key(uint32_t label, uint32_t pid) {
  return mix64(((uint64_t)label << 32) | (uint64_t)pid);
}

// Commutative per-element hash term (summed over the set).
__host__ __device__ __forceinline__ uint64_t elem_term(uint64_t key, uint64_t seed) {
  return mix64(key + seed);
}

// Hash of a node's signature from its parts.  Never returns kEmpty64.
__host__ __device__ __forceinline__ uint64_t node_hash(uint64_t term_sum, uint32_t first,
                                                       uint64_t count, uint64_t seed,
                                                       uint64_t mask) {
  uint64_t h = mix64(term_sum ^ mix64(((uint64_t)first << 32) + count + seed * 3 + 1));
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

// The device graph store plus all scratch a round needs.  One per handle.
struct Store {
  // configuration
  int device = 0;
  cudaStream_t stream = nullptr;
  uint64_t budget = 0;
  bool early_stop = true;
  uint64_t seed = 0;
  uint64_t hash_mask = ~0ull;
  bool checked = false;
  bool timing = false;

  // graph (CSR by source, original node ids)
  uint64_t n = 0, m = 0;
  bool has_graph = false;
  bool label8 = true;          // edge labels stored as uint8 (else uint32)
  bool any_dead = false;       // some node is deleted
  Buf offsets;                 // uint64 [n+1]
  Buf dst;                     // uint32 [m]
  Buf elabel;                  // uint8 or uint32 [m]
  Buf nlabel;                  // uint32 [n]
  Buf alive;                   // uint8 [n] (1 = present)

  // degree classes, fixed per graph: alive nodes ordered by class, then id
  Buf class_nodes;             // uint32
  uint64_t class_start[kSmallClasses + 4] = {0};  // classes: P=1..32, warp, CTA, hub
  uint64_t small_count[kSmallClasses] = {0};
  uint64_t small_start[kSmallClasses + 1] = {0};
  uint64_t n_warp = 0;         // out-degree 33..256
  uint64_t n_block = 0;        // 257..4096
  // hubs: out-degree > 4096
  uint64_t n_hub = 0;
  Buf hub_bits;                // uint32 [n_hub]  log2(bucket count)
  Buf hub_bbase;               // uint64 [n_hub+1] first bucket of each hub
  Buf hub_chunks;              // uint4 [n_chunks] (hub index, begin lo, begin hi, length)
  uint64_t n_hub_chunks = 0;
  uint64_t n_hub_buckets = 0;
  uint64_t hub_edges = 0;
  uint32_t hub_extra_bits = 0; // grows if a bucket overflows
  std::vector<uint32_t> h_hub_degbits;  // host copy: ceil(log2(deg / target)) per hub
  std::vector<uint64_t> h_hub_deg;

  // levels (all kept: history for extend / maintenance)
  std::vector<Buf> level;      // uint32 [n] per computed level
  std::vector<uint64_t> counts;
  uint32_t computed = 0;       // highest computed level (valid if has_levels)
  bool has_levels = false;
  bool stable = false;         // computed level equals the one before it
  uint32_t k_requested = 0;
  uint32_t rounds_run = 0;
  std::vector<kbisim_round_stats> stats;  // index r-1 for round r

  // round scratch
  Buf sigkey;                  // uint64 [m]: sorted distinct keys per node at its CSR offset
  Buf ucnt;                    // uint32 [n]
  Buf hash;                    // uint64 [n]
  Buf tkey;                    // uint64 [cap] hash table keys
  Buf tmin;                    // uint32 [cap] smallest node per key
  uint64_t tcap = 0;
  Buf slot;                    // uint32 [n]
  Buf rep;                     // uint32 [n]
  Buf ulist[2];                // uint32 [n] unresolved nodes (ping-pong)
  Buf bsum;                    // uint64 scan block sums
  Buf hub_hist;                // uint64 [buckets]
  Buf hub_cursor;              // uint64 [buckets]
  Buf hub_ucnt;                // uint32 [buckets]
  Buf hub_hpart;               // uint64 [buckets]
  Buf hub_tmp;                 // uint64 [hub_edges]
  Buf hub_tmp2;                // uint64 [hub_edges]
  Buf d_err;                   // uint32 error flags
  Buf d_scalars;               // uint64 [8] small device counters
  Buf h_scalars;               // pinned host mirror of d_scalars

  size_t bytes_held = 0;
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

// Allocation helpers (kbisim_api.cu)
Status ensure(Store& s, Buf& b, size_t bytes);
void release(Store& s, Buf& b);
Status cuda_check(cudaError_t e, const char* what);

// Round driver (kbisim_round.cu)
Status prepare_classes(Store& s);                 // degree classes and hub layout
Status compute_level0(Store& s);                  // pId_0 into level[0]
Status compute_round(Store& s, uint32_t i);       // pId_i from pId_{i-1}
Status timer_begin(Store& s, int kernel_class);
Status timer_end(Store& s, int kernel_class);
Status timer_collect(Store& s);
void timer_destroy(Store& s);

}  // namespace kb
