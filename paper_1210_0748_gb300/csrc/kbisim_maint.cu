// Incremental maintenance of the k-partition (paper Section 4: Algorithm 2
// Add_Nodes, Algorithm 3 Add_Edges, and deletions of edges handled like
// insertions), on the GPU.
//
// Algorithm 3 keeps, per level, the signature storage S across updates: a
// node's identifier is what S returns for its signature, so a node whose
// signature does not change keeps its identifier, and only nodes whose
// identifier changed put their parents on the queue of the next level.
// Here S_j is a device hash table from a 64-bit signature hash to a stable
// label, with the signature of each label kept exactly (first component,
// element count, element words) so that a hash collision never merges two
// signatures.  Level 0 labels are the node labels themselves.
//
// One update (edge insertions, edge deletions, node additions):
//   1. the batch is applied to the stored edge multiset (kbisim_update.cu);
//   2. the frontier of level 1 is the set of nodes whose out-edges changed and
//      the new nodes (the paper enqueues (j, s) for every level j and every
//      source s of a new edge);
//   3. for j = 1..k: if the frontier holds more than a fixed fraction of the
//      nodes, switch back to the full computation (the paper's "When to switch
//      back to Algorithm 1": check the queue size at the start of an
//      iteration).  Otherwise sign the frontier nodes from the labels of level
//      j-1, group them by exact signature, look each group's signature up in
//      S_j (inserting it with a new label when absent), and give the nodes
//      their labels.  The frontier of level j+1 is the update's sources, the
//      nodes whose level-j label changed (their own first component changed)
//      and the parents of those nodes;
//   4. every level's canonical identifiers (blocks ranked by their smallest
//      node id) are formed from the labels.
// The result equals a full recomputation (Theorem 2); the tests check it
// against the oracle after every batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "kbisim_internal.cuh"

namespace kb {
namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr uint64_t kFrontierFloor = 4096;  // frontiers this small never switch back

template <typename T>
T* ptr(const Buf& b) {
  return static_cast<T*>(b.p);
}

unsigned grid_for(const Store& s, uint64_t n, int per) {
  const uint64_t g = (n + per - 1) / per;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)s.sms * 16));
}

#define GRID_STRIDE(i, n) \
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ bool bit(const uint32_t* m, uint64_t i) { return (m[i >> 5] >> (i & 31)) & 1u; }
__device__ __forceinline__ void set_bit(uint32_t* m, uint64_t i) { atomicOr(&m[i >> 5], 1u << (i & 31)); }

// Home slot of a signature hash in a table of mask + 1 slots.
__device__ __forceinline__ uint64_t home_slot(uint64_t h, uint64_t mask) { return mix64(h ^ 0x6a09e667f3bcc909ull) & mask; }

// --- labels -----------------------------------------------------------------
// Level 0 labels: the node label of every alive node, original order.
__global__ void k_lab0(uint64_t n, uint64_t n_alive, const uint32_t* o2p, const uint32_t* nlabel, uint32_t* lab) {
  GRID_STRIDE(o, n) {
    const uint32_t p = o2p[o];
    lab[o] = p < n_alive ? nlabel[p] : kDead;
  }
}

// Labels from a canonical level (internal order), original order.
__global__ void k_lab_from_level(uint64_t n, const uint32_t* o2p, const uint32_t* level, uint32_t* lab) {
  GRID_STRIDE(o, n) lab[o] = level[o2p[o]];
}

// Original-order labels to internal order.
__global__ void k_to_internal(uint64_t n, const uint32_t* p2o, const uint32_t* lab, uint32_t* out) {
  GRID_STRIDE(p, n) out[p] = lab[p2o[p]];
}

// Smallest original id and member count of every label (labels < lcap).
__global__ void k_label_heads(uint64_t n, const uint32_t* lab, uint32_t* minid, uint32_t* cnt) {
  GRID_STRIDE(o, n) {
    const uint32_t b = lab[o];
    if (b == kDead) continue;
    atomicMin(&minid[b], (uint32_t)o);
    if (cnt) atomicAdd(&cnt[b], 1u);
  }
}

// Head bitmap over original ids: o is the smallest node of its label.
__global__ void k_label_head_bits(uint64_t n, const uint32_t* lab, const uint32_t* minid, uint32_t* hbits) {
  GRID_STRIDE(o, n) {
    const uint32_t b = lab[o];
    if (b != kDead && minid[b] == (uint32_t)o) set_bit(hbits, o);
  }
}

__global__ void k_word_popc(const uint32_t* bits, uint64_t words, uint64_t* out) {
  GRID_STRIDE(w, words) out[w] = __popc(bits[w]);
}

// Canonical identifier of every node (internal order): the rank of its
// label's head among all heads; alone flags (label with one member).
__global__ void k_label_pid(uint64_t n, uint64_t n_alive, const uint32_t* p2o, const uint32_t* lab,
                            const uint32_t* minid, const uint32_t* cnt, const uint32_t* hbits, const uint64_t* hword,
                            uint32_t* pid, uint8_t* alone, unsigned long long* n_alone) {
  unsigned int na = 0;
  GRID_STRIDE(p, n) {
    if (p >= n_alive) {
      pid[p] = kDead;
      if (alone) alone[p] = 0;
      continue;
    }
    const uint32_t b = lab[p2o[p]];
    const uint32_t h = minid[b];
    const uint32_t w = h >> 5;
    pid[p] = (uint32_t)hword[w] + (uint32_t)__popc(hbits[w] & ((1u << (h & 31)) - 1u));
    if (alone) {
      const bool al = cnt[b] == 1u;
      alone[p] = al ? 1 : 0;
      na += al ? 1u : 0u;
    }
  }
  if (alone) {
    na = __reduce_add_sync(kFullMask, na);
    if ((threadIdx.x & 31) == 0 && na) atomicAdd(n_alone, (unsigned long long)na);
  }
}

// --- the signature store ----------------------------------------------------
struct StoreArgs {
  unsigned long long* tkey;
  uint32_t* tval;
  uint64_t tmask;
  uint32_t* sfirst;
  uint32_t* scount;
  unsigned long long* soff;
  unsigned long long* pool;
  unsigned long long* ctr;  // [0] labels handed out, [1] pool words used
  uint64_t lcap, pcap;
  uint32_t* err;            // bit 1: a capacity was exceeded
};

struct NodeSig {
  const uint64_t* off;      // CSR offsets (internal ids)
  const uint64_t* sigkey;   // element words of each node at its CSR offset (64-bit keys)
  const uint32_t* sigkey32; //   or these, when the stores use 32-bit keys (then sigkey is null)
  const uint32_t* ucnt;
  const uint64_t* hash;
  const uint32_t* prev;     // labels of the level below, internal order (first component)
};

// Element word i of the signature words (32-bit keys are widened; the stores
// keep 64-bit words either way).
__device__ __forceinline__ uint64_t sig_word(const NodeSig& g, uint64_t i) {
  return g.sigkey32 ? (uint64_t)g.sigkey32[i] : g.sigkey[i];
}

// Claim a table slot for hash h and label b (the signature is already stored).
__device__ bool store_slot(const StoreArgs& a, uint64_t h, uint32_t b) {
  uint64_t s = home_slot(h, a.tmask);
  for (uint64_t t = 0; t <= a.tmask; ++t) {
    if (atomicCAS(&a.tkey[s], kEmpty64, (unsigned long long)h) == kEmpty64) {
      a.tval[s] = b;
      return true;
    }
    s = (s + 1) & a.tmask;
  }
  return false;
}

// The warp stores node p's signature under label b (all lanes take part).
// Signatures of more than kInlineCopy elements are only reserved here and
// listed in `big` (node, pool offset); k_copy_big copies them before any
// comparison reads them (only signatures of at most 32 elements are compared
// inside k_lookup, and those are copied here, before their slot is named).
constexpr uint32_t kInlineCopy = 32;

__device__ void store_signature(const StoreArgs& a, const NodeSig& g, uint64_t p, uint32_t b, uint2* big,
                                unsigned long long* n_big) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t U = g.ucnt[p];
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&a.ctr[1], (unsigned long long)U);
  base = __shfl_sync(kFullMask, base, 0);
  if (base + U > a.pcap || b >= a.lcap) {
    if (lane == 0) atomicOr(a.err, 1u);
    return;
  }
  if (U <= kInlineCopy) {
    const uint64_t o = g.off[p];
    for (uint32_t i = lane; i < U; i += 32) a.pool[base + i] = sig_word(g, o + i);
  } else if (lane == 0) {
    big[atomicAdd(n_big, 1ull)] = make_uint2((uint32_t)p, b);
  }
  if (lane == 0) {
    a.sfirst[b] = g.prev[p];
    a.scount[b] = U;
    a.soff[b] = base;
  }
  __threadfence();  // the signature is visible before its slot names it
  __syncwarp();
  if (lane == 0 && !store_slot(a, g.hash[p], b)) atomicOr(a.err, 1u);
}

// Element words of the long new signatures (one CTA per signature); the
// longest (hubs: more than kHugeCopy words) are listed for k_copy_huge, so
// that no CTA copies a million words while the others wait.
constexpr uint32_t kHugeCopy = 1u << 15;

__global__ void k_copy_big(StoreArgs a, NodeSig g, const uint2* big, uint64_t n_big, uint2* huge,
                           unsigned long long* n_huge) {
  for (uint64_t q = blockIdx.x; q < n_big; q += gridDim.x) {
    const uint2 e = big[q];
    const uint32_t U = a.scount[e.y];
    if (U > kHugeCopy) {
      if (threadIdx.x == 0) huge[atomicAdd(n_huge, 1ull)] = e;
      continue;
    }
    const uint64_t o = g.off[e.x];
    unsigned long long* dstp = a.pool + a.soff[e.y];
    for (uint32_t i = threadIdx.x; i < U; i += blockDim.x) dstp[i] = sig_word(g, o + i);
  }
}

// Each listed signature split evenly over all CTAs of the grid.
__global__ void k_copy_huge(StoreArgs a, NodeSig g, const uint2* huge, const unsigned long long* n_huge) {
  const uint64_t nh = *n_huge;
  for (uint64_t q = 0; q < nh; ++q) {
    const uint2 e = huge[q];
    const uint64_t U = a.scount[e.y];
    const uint64_t lo = U * blockIdx.x / gridDim.x, hi = U * (blockIdx.x + 1) / gridDim.x;
    const uint64_t o = g.off[e.x];
    unsigned long long* dstp = a.pool + a.soff[e.y];
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) dstp[i] = sig_word(g, o + i);
  }
}

// Copies of the listed long signatures (big: n_big entries, known on the
// host), the longest split over the whole grid.
Status copy_long_signatures(Store& s, const StoreArgs& sa, const NodeSig& ns, const uint2* big, uint64_t n_big) {
  MaintState& m = s.mt;
  Status st;
  if (!n_big) return Status::Ok();
  if (!(st = ensure(s, m.huge, (std::max<uint64_t>(s.n_hub, 1) + 1) * sizeof(uint2))).ok()) return st;
  unsigned long long* n_huge = ptr<unsigned long long>(m.misc) + 14;
  cudaMemsetAsync(n_huge, 0, 8, s.stream);
  k_copy_big<<<(unsigned)std::min<uint64_t>(n_big, (uint64_t)s.sms * 8), kThreads, 0, s.stream>>>(
      sa, ns, big, n_big, ptr<uint2>(m.huge), n_huge);
  k_copy_huge<<<(unsigned)s.sms * 8, kThreads, 0, s.stream>>>(sa, ns, ptr<uint2>(m.huge), n_huge);
  return cuda_check(cudaGetLastError(), "copy signatures");
}

// Build: the heads of every label (smallest original id) store their
// signatures under their canonical id, at pool offsets from a prefix sum of
// the heads' element counts (woff).  One warp per node.
constexpr uint32_t kBuildInlineCopy = 8;  // longer signatures: k_copy_big, one CTA each

// One thread per node: a head (smallest original id of its label) stores its
// signature's first component, count and offset, copies short signatures
// itself, lists long ones for k_copy_big, and names its label in the table.
__global__ void k_store_heads(StoreArgs a, NodeSig g, uint64_t n_alive, const uint32_t* p2o, const uint32_t* lab,
                              const uint32_t* minid, const unsigned long long* woff, uint2* big,
                              unsigned long long* n_big) {
  GRID_STRIDE(p, n_alive) {
    const uint32_t o = p2o[p];
    const uint32_t b = lab[o];
    if (minid[b] != o) continue;
    const uint32_t U = g.ucnt[p];
    const unsigned long long base = woff[p];
    if (U <= kBuildInlineCopy) {
      const uint64_t o = g.off[p];
      for (uint32_t i = 0; i < U; ++i) a.pool[base + i] = sig_word(g, o + i);
    } else {
      big[atomicAdd(n_big, 1ull)] = make_uint2((uint32_t)p, b);
    }
    a.sfirst[b] = g.prev[p];
    a.scount[b] = U;
    a.soff[b] = base;
    if (!store_slot(a, g.hash[p], b)) atomicOr(a.err, 1u);
  }
}

// Element words of every head (0 for the other nodes), for the pool offsets.
__global__ void k_head_words(uint64_t n_alive, uint64_t n, const uint32_t* p2o, const uint32_t* lab,
                             const uint32_t* minid, const uint32_t* ucnt, unsigned long long* w) {
  GRID_STRIDE(p, n + 1) {
    unsigned long long v = 0;
    if (p < n_alive) {
      const uint32_t o = p2o[p];
      if (minid[lab[o]] == o) v = ucnt[p];
    }
    w[p] = v;
  }
}

// Set equality of node p's elements and stored signature b (same count U <=
// 32), by the warp: lane i holds the node's element i and checks that it is
// among the stored ones (both lists are duplicate-free).
__device__ bool warp_same_set(const StoreArgs& a, const NodeSig& g, uint64_t p, uint32_t b, uint32_t U) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t mine = lane < U ? sig_word(g, g.off[p] + lane) : 0ull;
  const uint64_t stored = lane < U ? a.pool[a.soff[b] + lane] : 0ull;
  bool found = lane >= U;
  for (uint32_t j = 0; j < U; ++j) found |= __shfl_sync(kFullMask, stored, j) == mine;
  return __all_sync(kFullMask, found);
}

// Look up the signature of every frontier head in S_j (one warp per head).
// heads: (node, first slot to probe).  A stored signature with the same hash,
// first component and count is compared here when it has at most 32 elements;
// longer ones go to `pend` (node, label, slot) for k_long_compare.  A head
// whose probe reaches an empty slot is listed in `missed`; k_assign_missed
// gives those their labels once every lookup of the level is done (distinct
// heads have distinct signatures, so no head could find another's).
struct LookupArgs {
  const uint32_t* heads;    // node ids
  const unsigned long long* start;  // per head: slot to start at, or all ones for the home slot
  uint64_t count;
  uint32_t* newlab;         // per node (internal id): the label found
  uint4* pend;              // (head index, label, slot lo, slot hi)
  unsigned long long* n_pend;
  uint2* big;               // new signatures copied by k_copy_big (node, label)
  unsigned long long* n_big;
  uint32_t* missed;         // heads whose signature no label holds
  unsigned long long* n_missed;
  uint32_t* hit;            // bitmap over labels: found by some head
};

__global__ void k_lookup(StoreArgs a, NodeSig g, LookupArgs l) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < l.count; i += warps) {
    const uint32_t p = l.heads[i];
    const uint64_t h = g.hash[p];
    const uint32_t U = g.ucnt[p], first = g.prev[p];
    uint64_t s = l.start && l.start[i] != kEmpty64 ? l.start[i] : home_slot(h, a.tmask);
    bool done = false;
    for (uint64_t t = 0; t <= a.tmask && !done; ++t, s = (s + 1) & a.tmask) {
      const unsigned long long key = *(volatile unsigned long long*)&a.tkey[s];
      if (key == kEmpty64) break;
      if (key != h) continue;
      const uint32_t b = *(volatile uint32_t*)&a.tval[s];
      if (b == kNone32) continue;  // being written by another head: another signature
      if (a.sfirst[b] != first || a.scount[b] != U) continue;
      if (U > 32) {
        if (lane == 0) {
          const unsigned long long q = atomicAdd(l.n_pend, 1ull);
          l.pend[q] = make_uint4((uint32_t)i, b, (uint32_t)s, (uint32_t)(s >> 32));
        }
        done = true;
        break;
      }
      if (warp_same_set(a, g, p, b, U)) {
        if (lane == 0) {
          l.newlab[p] = b;
          set_bit(l.hit, b);
        }
        done = true;
      }
    }
    if (!done && lane == 0) l.missed[atomicAdd(l.n_missed, 1ull)] = p;  // not in S_j
  }
}

// Labels of the heads no label matched (one warp per head).  A head keeps its
// members' old label B when the group is all of B (every member had label B,
// and as many as B has nodes) and no head found B in this level: B's block is
// unchanged as a set, it only takes the new signature, so B is pointed at it.
// Any other head gets a new label.  Each B is all of at most one group, so no
// two heads take the same label.
__global__ void k_assign_missed(StoreArgs a, NodeSig g, LookupArgs l, uint64_t n_missed, const uint32_t* gold,
                                const uint32_t* gsize, const uint32_t* cnt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n_missed; i += warps) {
    const uint32_t p = l.missed[i];
    uint32_t b = 0;
    if (lane == 0) {
      const uint32_t B = gold[p], sz = gsize[p];
      const bool keep = B != kNone32 && !(sz >> 31) && sz == cnt[B] && !bit(l.hit, B);
      b = keep ? B : (uint32_t)atomicAdd(&a.ctr[0], 1ull);
    }
    b = __shfl_sync(kFullMask, b, 0);
    store_signature(a, g, p, b, l.big, l.n_big);
    if (lane == 0) l.newlab[p] = b;
  }
}

// One CTA per pending (head, label): equal sets iff every element of the
// head is among the label's stored elements (equal counts, both duplicate
// free).  The stored elements go into a shared-memory set chunk by chunk.
constexpr int kCmpThreads = 256, kCmpChunk = 4096, kCmpSlots = 2 * kCmpChunk;

__global__ void __launch_bounds__(kCmpThreads) k_long_compare(StoreArgs a, NodeSig g, LookupArgs l,
                                                               uint64_t n_pend, uint32_t* match) {
  __shared__ unsigned long long set[kCmpSlots];
  __shared__ unsigned int found_sh;
  for (uint64_t q = blockIdx.x; q < n_pend; q += gridDim.x) {
    const uint4 e = l.pend[q];
    const uint32_t p = l.heads[e.x], b = e.y;
    const uint32_t U = g.ucnt[p];
    if (U > kCmpChunk) continue;  // compared by k_big_* through a set in global memory
    const uint64_t mo = g.off[p];
    const unsigned long long* stored = a.pool + a.soff[b];
    uint32_t found = 0;
    for (uint32_t c0 = 0; c0 < U; c0 += kCmpChunk) {
      const uint32_t cn = min((uint32_t)kCmpChunk, U - c0);
      for (int i = threadIdx.x; i < kCmpSlots; i += kCmpThreads) set[i] = kEmpty64;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < cn; i += kCmpThreads) {
        const unsigned long long k = stored[c0 + i];
        uint32_t s = (uint32_t)(mix64(k) & (kCmpSlots - 1));
        for (int t = 0; t < kCmpSlots; ++t) {  // a chunk fills at most half the set
          const unsigned long long old = atomicCAS(&set[s], kEmpty64, k);
          if (old == kEmpty64 || old == k) break;
          s = (s + 1) & (kCmpSlots - 1);
        }
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < U; i += kCmpThreads) {
        const unsigned long long k = sig_word(g, mo + i);
        uint32_t s = (uint32_t)(mix64(k) & (kCmpSlots - 1));
        for (int t = 0; t < kCmpSlots; ++t) {
          const unsigned long long cur = set[s];
          if (cur == k) {
            ++found;
            break;
          }
          if (cur == kEmpty64) break;
          s = (s + 1) & (kCmpSlots - 1);
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) found_sh = 0;
    __syncthreads();
    found = __reduce_add_sync(kFullMask, found);
    if ((threadIdx.x & 31) == 0) atomicAdd(&found_sh, found);
    __syncthreads();
    // the element equal to the empty marker cannot sit in the set: compare it apart
    if (threadIdx.x == 0) {
      uint32_t extra = 0;
      bool mine_has = false, stored_has = false;
      for (uint32_t i = 0; i < U; ++i) {
        mine_has |= sig_word(g, mo + i) == kEmpty64;
        stored_has |= stored[i] == kEmpty64;
      }
      if (mine_has && stored_has) extra = 1;
      match[q] = (found_sh + extra == U) ? 1u : 0u;
    }
    __syncthreads();
  }
}

// Long signatures (more than kCmpChunk elements), one pair at a time over the
// whole grid: the stored elements go into a hash set in global memory of 2U
// slots, then the node's elements are looked up.
__global__ void k_big_insert(const unsigned long long* stored, uint32_t U, unsigned long long* set, uint64_t smask,
                             unsigned int* flags) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < U; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = stored[i];
    if (k == kEmpty64) {
      flags[0] = 1u;
      continue;
    }
    uint64_t s = mix64(k) & smask;
    for (uint64_t t = 0; t <= smask; ++t) {
      const unsigned long long old = atomicCAS(&set[s], kEmpty64, k);
      if (old == kEmpty64 || old == k) break;
      s = (s + 1) & smask;
    }
  }
}

__global__ void k_big_lookup(NodeSig g, uint64_t mo, uint32_t U, const unsigned long long* set, uint64_t smask,
                             unsigned int* flags) {
  unsigned int found = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < U; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = sig_word(g, mo + i);
    if (k == kEmpty64) {
      found += flags[0];
      continue;
    }
    uint64_t s = mix64(k) & smask;
    for (uint64_t t = 0; t <= smask; ++t) {
      const unsigned long long cur = set[s];
      if (cur == k) {
        ++found;
        break;
      }
      if (cur == kEmpty64) break;
      s = (s + 1) & smask;
    }
  }
  found = __reduce_add_sync(kFullMask, found);
  if ((threadIdx.x & 31) == 0 && found) atomicAdd(&flags[1], found);
}

// Per pending pair: element count, the node's first element word, the
// stored signature's first pool word (for the host to route long pairs).
__global__ void k_pending_info(const uint4* pend, const uint32_t* heads, uint64_t np, const uint32_t* ucnt,
                               const uint64_t* off, const unsigned long long* soff, unsigned long long* info) {
  GRID_STRIDE(q, np) {
    const uint4 e = pend[q];
    const uint32_t p = heads[e.x];
    info[3 * q] = ucnt[p];
    info[3 * q + 1] = off[p];
    info[3 * q + 2] = soff[e.y];
  }
}

__global__ void k_big_result(const unsigned int* flags, uint32_t U, uint32_t* match) {
  *match = flags[1] == U ? 1u : 0u;
}

// After a long compare: matched heads take the label, the others probe on
// from the next slot (a new pending list for k_lookup).
__global__ void k_resolve(LookupArgs l, uint64_t n_pend, const uint32_t* match, uint32_t* retry_heads,
                          unsigned long long* retry_start, unsigned long long* n_retry, uint64_t tmask) {
  GRID_STRIDE(q, n_pend) {
    const uint4 e = l.pend[q];
    const uint32_t p = l.heads[e.x];
    if (match[q]) {
      l.newlab[p] = e.y;
      set_bit(l.hit, e.y);
    } else {
      const unsigned long long r = atomicAdd(n_retry, 1ull);
      retry_heads[r] = p;
      retry_start[r] = ((((uint64_t)e.w << 32) | e.z) + 1) & tmask;
    }
  }
}

// --- frontier -----------------------------------------------------------------
// List of the set bits of a bitmap over internal ids (order free).
__global__ void k_bits_to_list(const uint32_t* bits, uint64_t words, uint64_t n, uint32_t* list,
                               unsigned long long* count) {
  GRID_STRIDE(w, words) {
    uint32_t m = bits[w];
    if (!m) continue;
    const unsigned long long base = atomicAdd(count, (unsigned long long)__popc(m));
    uint32_t k = 0;
    while (m) {
      const uint32_t b = __ffs(m) - 1;
      m &= m - 1;
      const uint64_t p = (w << 5) + b;
      if (p < n) list[base + k] = (uint32_t)p;
      ++k;
    }
  }
}

// Sources of the batch's edges (original ids) and the new nodes into the
// seed bitmap (internal ids).
__global__ void k_seed_sources(uint64_t k, const uint32_t* src, const uint32_t* o2p, uint32_t* seeds) {
  GRID_STRIDE(i, k) set_bit(seeds, o2p[src[i]]);
}
__global__ void k_seed_new(uint64_t n0, uint64_t n1, const uint32_t* o2p, uint32_t* seeds) {
  GRID_STRIDE(o, n1 - n0) set_bit(seeds, o2p[n0 + o]);
}

// Labels of level j for the frontier: a head's new label goes to every node
// of its group; nodes whose label changed are marked and counted, and the
// labels' node counts follow.
__global__ void k_assign(const uint32_t* list, uint64_t count, const uint32_t* rep, const uint32_t* newlab,
                         const uint32_t* p2o, uint32_t* lab, uint32_t* changed, uint32_t* cnt,
                         unsigned long long* n_changed) {
  unsigned int nc = 0;
  GRID_STRIDE(i, count) {
    const uint32_t p = list[i];
    const uint32_t b = newlab[rep[p]];
    const uint32_t o = p2o[p];
    const uint32_t old = lab[o];
    if (old != b) {
      lab[o] = b;
      set_bit(changed, p);
      if (old != kNone32) atomicSub(&cnt[old], 1u);
      atomicAdd(&cnt[b], 1u);
      ++nc;
    }
  }
  nc = __reduce_add_sync(kFullMask, nc);
  if ((threadIdx.x & 31) == 0 && nc) atomicAdd(n_changed, (unsigned long long)nc);
}

// Next frontier: seeds | changed | parents of changed nodes (a node is a
// parent of a changed node if one of its out-edges points to it).
// The parents by one pass over all edges, streamed in order: a coarse
// bitmap (bit w set iff word w of `changed` is non-zero, 1 bit per 32 nodes;
// 62.5 KB at 16M nodes, so it stays in L1) decides most edges without touching
// the changed bitmap.  A warp takes kPullItems runs of 32 consecutive edges at
// a time, all their target loads in flight together; in a run with a hit,
// lane 0 finds the source of the run's first edge by binary search over the
// offsets and each hit lane walks on from there (its edge lies at most 31
// edges further), and lanes with the same source set its bit once.
__global__ void k_changed_words(const uint32_t* changed, uint64_t words, uint32_t* coarse) {
  GRID_STRIDE(w, words) {
    if (changed[w]) atomicOr(&coarse[w >> 5], 1u << (w & 31));
  }
}

__device__ __forceinline__ uint64_t source_of(const uint64_t* off, uint64_t n, uint64_t e) {
  uint64_t lo = 0, hi = n;  // off[lo] <= e < off[hi]: lo ends as the node whose edges hold e
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

constexpr int kPullItems = 8;

__global__ void k_frontier_pull(uint64_t m, uint64_t n, const uint64_t* off, const uint32_t* dst,
                                const uint32_t* changed, const uint32_t* coarse, const unsigned long long* n_changed,
                                uint32_t* next) {
  if (*n_changed == 0) return;  // no label changed: no parents to add
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  constexpr uint64_t kSpan = 32 * kPullItems;
  for (uint64_t base = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * kSpan; base < m;
       base += warps * kSpan) {
    uint32_t t[kPullItems];
#pragma unroll
    for (int r = 0; r < kPullItems; ++r) {
      const uint64_t e = base + 32 * r + lane;
      t[r] = e < m ? __ldg(dst + e) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < kPullItems; ++r) {
      const uint64_t e = base + 32 * r + lane;
      bool hit = false;
      if (t[r] != 0xFFFFFFFFu) {
        const uint32_t w = t[r] >> 5;
        hit = ((__ldg(coarse + (w >> 5)) >> (w & 31)) & 1u) && bit(changed, t[r]);
      }
      const unsigned hm = __ballot_sync(kFullMask, hit);
      if (!hm) continue;
      uint64_t p0 = 0;
      if (lane == 0) p0 = source_of(off, n, base + 32 * r);
      p0 = __shfl_sync(kFullMask, p0, 0);
      if (hit) {  // every lane of hm is here
        uint64_t p = p0;
        while (off[p + 1] <= e) ++p;  // ends: off[n] = m > e
        const unsigned same = __match_any_sync(hm, p);
        if (lane == (uint32_t)(__ffs(same) - 1) && !bit(next, p)) set_bit(next, p);
      }
    }
  }
}

__global__ void k_or3(uint64_t words, const uint32_t* a, const uint32_t* b, uint32_t* out) {
  GRID_STRIDE(w, words) out[w] |= a[w] | b[w];
}
__global__ void k_popc_sum(const uint32_t* bits, uint64_t words, unsigned long long* total) {
  unsigned long long c = 0;
  GRID_STRIDE(w, words) c += __popc(bits[w]);
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFullMask, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}

// Labels of added nodes: their node label at level 0, "none" above (a new
// node is always in the frontier, so it gets a label at every level).
__global__ void k_lab_grow(uint64_t n0, uint64_t n1, const uint32_t* o2p, const uint32_t* nlabel, int level0,
                           uint32_t* lab) {
  GRID_STRIDE(i, n1 - n0) lab[n0 + i] = level0 ? nlabel[o2p[n0 + i]] : kNone32;
}

// --- host ---------------------------------------------------------------------
Status sync_read(Store& s, void* dst, const void* src, size_t bytes, const char* what) {
  Status st = cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s.stream), what);
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), what);
  return st;
}

// Grow b to at least `bytes`, keeping its first `keep` bytes.
Status grow_keep(Store& s, Buf& b, size_t bytes, size_t keep) {
  if (bytes <= b.cap && b.p) return Status::Ok();
  Buf nb;
  Status st = ensure(s, nb, bytes);
  if (!st.ok()) return st;
  if (keep && b.p)
    st = cuda_check(cudaMemcpyAsync(nb.p, b.p, std::min(keep, b.cap), cudaMemcpyDeviceToDevice, s.stream), "grow");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "grow");
  release(s, b);
  b = nb;
  return st;
}

uint64_t pow2_at_least(uint64_t v) {
  uint64_t c = 1024;
  while (c < v) c <<= 1;
  return c;
}

StoreArgs store_args(Store& s, MaintLevel& L) {
  StoreArgs a;
  a.tkey = ptr<unsigned long long>(L.tkey);
  a.tval = ptr<uint32_t>(L.tval);
  a.tmask = L.tcap - 1;
  a.sfirst = ptr<uint32_t>(L.sfirst);
  a.scount = ptr<uint32_t>(L.scount);
  a.soff = ptr<unsigned long long>(L.soff);
  a.pool = ptr<unsigned long long>(L.pool);
  a.ctr = ptr<unsigned long long>(L.ctr);
  a.lcap = s.mt.key32 ? std::min<uint64_t>(L.lcap, 1ull << s.mt.pbits) : L.lcap;  // labels fit the element words
  a.pcap = L.pcap;
  a.err = ptr<uint32_t>(s.d_err);
  return a;
}

NodeSig node_sig(Store& s) {
  NodeSig g;
  g.off = ptr<uint64_t>(s.offsets);
  g.sigkey = s.mt.key32 ? nullptr : ptr<uint64_t>(s.sigkey);
  g.sigkey32 = s.mt.key32 ? ptr<uint32_t>(s.sigkey) : nullptr;
  g.ucnt = ptr<uint32_t>(s.ucnt);
  g.hash = ptr<uint64_t>(s.hash);
  g.prev = ptr<uint32_t>(s.mt.prev_int);
  return g;
}

Status ensure_common(Store& s) {
  MaintState& m = s.mt;
  const uint64_t n = std::max<uint64_t>(s.n, 1), words = (n + 31) / 32 + 1;
  Status st;
  Buf* bits[] = {&m.fmask, &m.fnext, &m.changed, &m.seeds};
  for (Buf* b : bits)
    if (!(st = ensure(s, *b, words * 4)).ok()) return st;
  if (!(st = ensure(s, m.list, n * 4)).ok()) return st;
  if (!(st = ensure(s, m.prev_int, n * 4)).ok()) return st;
  if (!(st = ensure(s, m.newlab, n * 4)).ok()) return st;
  if (!(st = ensure(s, m.misc, 16 * 8)).ok()) return st;
  return Status::Ok();
}

// Canonical identifiers of level j (internal order) from its labels; the
// number of blocks; alone flags when `alone` is set.
Status canonical_from_labels(Store& s, uint32_t j, uint32_t* pid, uint64_t* blocks, bool alone) {
  MaintState& m = s.mt;
  MaintLevel& L = m.lv[j];
  const uint64_t n = s.n, words = n / 32 + 1;
  Status st;
  if (!(st = ensure(s, m.minid, L.lcap * 4)).ok()) return st;
  if (!(st = ensure(s, s.hbits, words * 4 + 16)).ok()) return st;
  if (!(st = ensure(s, s.hword, words * 8)).ok()) return st;
  cudaMemsetAsync(m.minid.p, 0xFF, L.lcap * 4, s.stream);
  cudaMemsetAsync(s.hbits.p, 0, words * 4, s.stream);
  unsigned long long* sc = ptr<unsigned long long>(m.misc);
  cudaMemsetAsync(sc + 4, 0, 8, s.stream);
  const uint32_t* lab = ptr<uint32_t>(L.lab);
  // the labels' node counts are kept by the store build and every assignment
  k_label_heads<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, lab, ptr<uint32_t>(m.minid), nullptr);
  k_label_head_bits<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, lab, ptr<uint32_t>(m.minid),
                                                                          ptr<uint32_t>(s.hbits));
  k_word_popc<<<grid_for(s, words, kThreads), kThreads, 0, s.stream>>>(ptr<uint32_t>(s.hbits), words,
                                                                        ptr<uint64_t>(s.hword));
  if (!(st = cuda_check(cudaGetLastError(), "canonical ids")).ok()) return st;
  if (!(st = scan_u64(s, ptr<uint64_t>(s.hword), words)).ok()) return st;
  k_label_pid<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(
      n, s.n_alive, ptr<uint32_t>(s.p2o), lab, ptr<uint32_t>(m.minid), ptr<uint32_t>(L.cnt), ptr<uint32_t>(s.hbits),
      ptr<uint64_t>(s.hword), pid, alone ? ptr<uint8_t>(s.alone) : nullptr, sc + 4);
  if (!(st = cuda_check(cudaGetLastError(), "canonical ids")).ok()) return st;
  uint64_t tail[2] = {0, 0};
  // blocks = heads before the spare word past the last node
  if (!(st = sync_read(s, tail, ptr<uint64_t>(s.hword) + (words - 1), 8, "block count")).ok()) return st;
  uint32_t lastw = 0;
  if (!(st = sync_read(s, &lastw, ptr<uint32_t>(s.hbits) + (words - 1), 4, "block count")).ok()) return st;
  *blocks = tail[0] + (uint64_t)__builtin_popcount(lastw);
  if (alone && !(st = sync_read(s, &s.n_alone, sc + 4, 8, "alone")).ok()) return st;
  return Status::Ok();
}

// S_j for level j from the current labels of levels j-1 and j (canonical at
// build time): every label's head stores its signature.
Status build_level_store(Store& s, uint32_t j, uint64_t labels) {
  MaintState& m = s.mt;
  MaintLevel& L = m.lv[j];
  const uint64_t n = s.n, na = s.n_alive;
  Status st;
  k_to_internal<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, ptr<uint32_t>(s.p2o),
                                                                      ptr<uint32_t>(m.lv[j - 1].lab),
                                                                      ptr<uint32_t>(m.prev_int));
  if (!(st = masked_signatures(s, ptr<uint32_t>(m.prev_int), nullptr)).ok()) return st;
  L.lcap = pow2_at_least(2 * labels + 1024);
  if (!(st = ensure(s, m.minid, L.lcap * 4)).ok()) return st;
  if (!(st = ensure(s, L.cnt, L.lcap * 4)).ok()) return st;
  cudaMemsetAsync(m.minid.p, 0xFF, L.lcap * 4, s.stream);
  cudaMemsetAsync(L.cnt.p, 0, L.lcap * 4, s.stream);
  k_label_heads<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, ptr<uint32_t>(L.lab), ptr<uint32_t>(m.minid),
                                                                      ptr<uint32_t>(L.cnt));
  if (!(st = ensure(s, m.woff, (n + 1) * 8)).ok()) return st;
  unsigned long long* woff = ptr<unsigned long long>(m.woff);
  k_head_words<<<grid_for(s, n + 1, kThreads), kThreads, 0, s.stream>>>(na, n, ptr<uint32_t>(s.p2o),
                                                                          ptr<uint32_t>(L.lab), ptr<uint32_t>(m.minid),
                                                                          ptr<uint32_t>(s.ucnt), woff);
  if (!(st = cuda_check(cudaGetLastError(), "store size")).ok()) return st;
  if (!(st = scan_u64(s, reinterpret_cast<uint64_t*>(woff), n + 1)).ok()) return st;
  uint64_t words = 0;
  if (!(st = sync_read(s, &words, woff + n, 8, "store size")).ok()) return st;
  L.pcap = 3 * words + s.store_room;  // room for the signatures later updates add (then grown)
  L.tcap = pow2_at_least(2 * L.lcap);
  L.entries = labels;
  if (!(st = ensure(s, L.tkey, L.tcap * 8)).ok()) return st;
  if (!(st = ensure(s, L.tval, L.tcap * 4)).ok()) return st;
  if (!(st = ensure(s, L.sfirst, L.lcap * 4)).ok()) return st;
  if (!(st = ensure(s, L.scount, L.lcap * 4)).ok()) return st;
  if (!(st = ensure(s, L.soff, L.lcap * 8)).ok()) return st;
  if (!(st = ensure(s, L.pool, L.pcap * 8)).ok()) return st;
  if (!(st = ensure(s, L.ctr, 16)).ok()) return st;
  cudaMemsetAsync(L.tkey.p, 0xFF, L.tcap * 8, s.stream);
  cudaMemsetAsync(L.tval.p, 0xFF, L.tcap * 4, s.stream);
  uint64_t c0[2] = {labels, words};
  if (!(st = cuda_check(cudaMemcpyAsync(L.ctr.p, c0, 16, cudaMemcpyHostToDevice, s.stream), "store")).ok()) return st;
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  const uint64_t nbig = std::max<uint64_t>(s.n_alive - std::min(s.n_alive, s.class_start[kSmallClasses - 3]), 1);
  if (!(st = ensure(s, m.big, nbig * sizeof(uint2))).ok()) return st;
  unsigned long long* sc = ptr<unsigned long long>(m.misc);
  cudaMemsetAsync(sc + 12, 0, 8, s.stream);
  k_store_heads<<<grid_for(s, na, kThreads), kThreads, 0, s.stream>>>(store_args(s, L), node_sig(s), na,
                                                                ptr<uint32_t>(s.p2o), ptr<uint32_t>(L.lab),
                                                                ptr<uint32_t>(m.minid), woff, ptr<uint2>(m.big),
                                                                sc + 12);
  uint64_t hb = 0;
  if (!(st = cuda_check(cudaGetLastError(), "store heads")).ok()) return st;
  if (!(st = sync_read(s, &hb, sc + 12, 8, "store heads")).ok()) return st;
  if (!(st = copy_long_signatures(s, store_args(s, L), node_sig(s), ptr<uint2>(m.big), hb)).ok()) return st;
  uint32_t e = 0;
  if (!(st = cuda_check(cudaGetLastError(), "store heads")).ok()) return st;
  if (!(st = sync_read(s, &e, s.d_err.p, 4, "store heads")).ok()) return st;
  if (e & 1u) return Status::Err(KBISIM_ERR_TIMEOUT, "signature store capacity exceeded at build");
  return Status::Ok();
}

// Heads of the frontier groups (rep[p] == p), listed, and their element
// counts summed (the most pool words the level's new signatures can take);
// each head's old label starts its group's record (k_group_stats).
__global__ void k_group_heads(const uint32_t* list, uint64_t count, const uint32_t* rep, const uint32_t* ucnt,
                              const uint32_t* p2o, const uint32_t* lab, uint32_t* heads, unsigned long long* n,
                              unsigned long long* words, uint32_t* gold, uint32_t* gsize) {
  GRID_STRIDE(i, count) {
    const uint32_t p = list[i];
    if (rep[p] == p) {
      heads[atomicAdd(n, 1ull)] = p;
      atomicAdd(words, (unsigned long long)ucnt[p]);
      gold[p] = lab[p2o[p]];
      gsize[p] = 0;
    }
  }
}

// Per frontier group: how many members, and whether they all had the head's
// old label (top bit of gsize set otherwise).
__global__ void k_group_stats(const uint32_t* list, uint64_t count, const uint32_t* rep, const uint32_t* p2o,
                              const uint32_t* lab, const uint32_t* gold, uint32_t* gsize) {
  GRID_STRIDE(i, count) {
    const uint32_t p = list[i];
    const uint32_t h = rep[p];
    if (lab[p2o[p]] != gold[h]) atomicOr(&gsize[h], 0x80000000u);
    atomicAdd(&gsize[h], 1u);
  }
}

// Every occupied slot of a table into the (larger, empty) table of a.
__global__ void k_rehash(const unsigned long long* okey, const uint32_t* oval, uint64_t ocap, StoreArgs a) {
  GRID_STRIDE(i, ocap) {
    const unsigned long long h = okey[i];
    if (h != kEmpty64 && !store_slot(a, h, oval[i])) atomicOr(a.err, 1u);
  }
}

bool no_room(const Status& st) {
  return st.code == KBISIM_ERR_BUDGET || st.code == KBISIM_ERR_OUT_OF_MEMORY;
}

// Room in S_j for `labels` labels, `words` pool words and `entries` table
// slots: the label arrays, the table (kept at most half full) and the pool
// grow, keeping what they hold (new labels' node counts start at zero).
// *fits is false when the labels would not fit the element words of the
// level above, or the device has no room (the caller recomputes).
Status reserve_store(Store& s, MaintLevel& L, uint64_t used_labels, uint64_t labels, uint64_t used_words,
                     uint64_t words, uint64_t entries, bool* fits) {
  MaintState& m = s.mt;
  const uint64_t limit = m.key32 ? (1ull << m.pbits) : (uint64_t)kNone32;
  Status st;
  if (labels > limit) {
    *fits = false;
    return Status::Ok();
  }
  if (labels > L.lcap) {
    const uint64_t lcap = std::min<uint64_t>(pow2_at_least(2 * labels), limit);
    if ((st = grow_keep(s, L.sfirst, lcap * 4, used_labels * 4)).ok() &&
        (st = grow_keep(s, L.scount, lcap * 4, used_labels * 4)).ok() &&
        (st = grow_keep(s, L.cnt, lcap * 4, used_labels * 4)).ok())
      st = grow_keep(s, L.soff, lcap * 8, used_labels * 8);
    if (!st.ok()) {
      if (!no_room(st)) return st;
      *fits = false;
      return Status::Ok();
    }
    cudaMemsetAsync(ptr<uint32_t>(L.cnt) + used_labels, 0, (lcap - used_labels) * 4, s.stream);
    L.lcap = lcap;
  }
  if (2 * entries > L.tcap) {
    const uint64_t tcap = pow2_at_least(4 * entries);
    Buf nk, nv;
    if ((st = ensure(s, nk, tcap * 8)).ok()) st = ensure(s, nv, tcap * 4);
    if (!st.ok()) {
      release(s, nk);
      release(s, nv);
      if (!no_room(st)) return st;
      *fits = false;
      return Status::Ok();
    }
    cudaMemsetAsync(nk.p, 0xFF, tcap * 8, s.stream);
    cudaMemsetAsync(nv.p, 0xFF, tcap * 4, s.stream);
    StoreArgs a = store_args(s, L);
    a.tkey = ptr<unsigned long long>(nk);
    a.tval = ptr<uint32_t>(nv);
    a.tmask = tcap - 1;
    cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
    k_rehash<<<grid_for(s, L.tcap, kThreads), kThreads, 0, s.stream>>>(ptr<unsigned long long>(L.tkey),
                                                                      ptr<uint32_t>(L.tval), L.tcap, a);
    uint32_t e = 0;
    if ((st = cuda_check(cudaGetLastError(), "rehash")).ok()) st = sync_read(s, &e, s.d_err.p, 4, "rehash");
    if (st.ok() && (e & 1u)) st = Status::Err(KBISIM_ERR_TIMEOUT, "signature table rehash found no slot");
    if (!st.ok()) {
      release(s, nk);
      release(s, nv);
      return st;
    }
    release(s, L.tkey);
    release(s, L.tval);
    L.tkey = nk;
    L.tval = nv;
    L.tcap = tcap;
  }
  if (words > L.pcap) {
    const uint64_t pcap = words + std::max<uint64_t>(words / 2, 4u << 20);
    st = grow_keep(s, L.pool, pcap * 8, used_words * 8);
    if (!st.ok()) {
      if (!no_room(st)) return st;
      *fits = false;
      return Status::Ok();
    }
    L.pcap = pcap;
  }
  return Status::Ok();
}

// One level of an update: the frontier (fmask) gets its labels of level j.
// Returns false in *fits when a store capacity ran out (the caller recomputes).
Status update_level(Store& s, uint32_t j, uint64_t count, bool* fits) {
  MaintState& m = s.mt;
  MaintLevel& L = m.lv[j];
  Status st;
  *fits = true;
  uint32_t* list = ptr<uint32_t>(m.list);
  if (!(st = masked_signatures(s, ptr<uint32_t>(m.prev_int), ptr<uint32_t>(m.fmask))).ok()) return st;
  if (!(st = group_list(s, list, count, ptr<uint32_t>(m.prev_int))).ok()) return st;
  // heads of the frontier groups (rep[p] == p) look up S_j; scratch of the
  // lookup: pending long compares, restart slots, results, heads, retries,
  // heads no label matched
  const size_t cnt = std::max<uint64_t>(count, 1);
  if (!(st = ensure(s, m.pend, cnt * (sizeof(uint4) + 8 + 8 + 4 + 4 + 4 + 4))).ok()) return st;
  uint4* pend = ptr<uint4>(m.pend);
  unsigned long long* start = reinterpret_cast<unsigned long long*>(pend + cnt);
  uint2* big = reinterpret_cast<uint2*>(start + cnt);
  uint32_t* match = reinterpret_cast<uint32_t*>(big + cnt);
  uint32_t* heads = match + cnt;
  uint32_t* retry = heads + cnt;
  uint32_t* missed = retry + cnt;
  const uint64_t nn = std::max<uint64_t>(s.n, 1);
  if (!(st = ensure(s, m.gold, nn * 4)).ok()) return st;
  if (!(st = ensure(s, m.gsize, nn * 4)).ok()) return st;
  uint32_t* gold = ptr<uint32_t>(m.gold);
  uint32_t* gsize = ptr<uint32_t>(m.gsize);
  unsigned long long* sc = ptr<unsigned long long>(m.misc);
  cudaMemsetAsync(sc, 0, 48, s.stream);
  k_group_heads<<<grid_for(s, count, kThreads), kThreads, 0, s.stream>>>(
      list, count, ptr<uint32_t>(s.rep), ptr<uint32_t>(s.ucnt), ptr<uint32_t>(s.p2o), ptr<uint32_t>(L.lab), heads, sc,
      sc + 5, gold, gsize);
  k_group_stats<<<grid_for(s, count, kThreads), kThreads, 0, s.stream>>>(list, count, ptr<uint32_t>(s.rep),
                                                                        ptr<uint32_t>(s.p2o), ptr<uint32_t>(L.lab),
                                                                        gold, gsize);
  cudaMemcpyAsync(sc + 6, L.ctr.p, 16, cudaMemcpyDeviceToDevice, s.stream);
  uint64_t hv8[8] = {};
  if (!(st = cuda_check(cudaGetLastError(), "group heads")).ok()) return st;
  if (!(st = sync_read(s, hv8, sc, 64, "group heads")).ok()) return st;
  const uint64_t nheads = hv8[0];
  // every head may store a new signature: [6] labels handed out, [7] pool words used
  if (!(st = reserve_store(s, L, hv8[6], hv8[6] + nheads, hv8[7], hv8[7] + hv8[5], L.entries + nheads, fits)).ok())
    return st;
  if (!*fits) return Status::Ok();
  const uint64_t hwords = L.lcap / 32 + 1;
  if (!(st = ensure(s, m.hit, hwords * 4)).ok()) return st;
  cudaMemsetAsync(m.hit.p, 0, hwords * 4, s.stream);
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  LookupArgs la;
  la.heads = heads;
  la.start = nullptr;
  la.count = nheads;
  la.newlab = ptr<uint32_t>(m.newlab);
  la.pend = pend;
  la.n_pend = sc + 1;
  la.big = big;
  la.n_big = sc + 3;
  la.missed = missed;
  la.n_missed = sc + 4;  // zeroed above, summed over the passes
  la.hit = ptr<uint32_t>(m.hit);
  const StoreArgs sa = store_args(s, L);
  const NodeSig ns = node_sig(s);
  uint64_t n_missed = 0;
  for (int pass = 0; la.count; ++pass) {
    if (pass > 64) return Status::Err(KBISIM_ERR_TIMEOUT, "signature lookup made no progress");
    cudaMemsetAsync(sc + 1, 0, 16, s.stream);  // [1] pending, [2] retries
    k_lookup<<<(unsigned)std::min<uint64_t>((la.count + 7) / 8, (uint64_t)s.sms * 8), kThreads, 0, s.stream>>>(sa, ns,
                                                                                                            la);
    uint64_t hv[4] = {0, 0, 0, 0};  // [0] pending, [3] missed so far
    if (!(st = cuda_check(cudaGetLastError(), "lookup")).ok()) return st;
    if (!(st = sync_read(s, hv, sc + 1, 32, "lookup")).ok()) return st;
    n_missed = hv[3];
    const uint64_t np = hv[0];
    if (!np) break;
    k_long_compare<<<(unsigned)std::min<uint64_t>(np, (uint64_t)s.sms * 4), kCmpThreads, 0, s.stream>>>(sa, ns, la, np,
                                                                                                      match);
    // pairs above kCmpChunk elements: one at a time through a set in global memory
    if (!(st = ensure(s, m.cmp_info, np * 24)).ok()) return st;
    k_pending_info<<<grid_for(s, np, kThreads), kThreads, 0, s.stream>>>(
        pend, heads, np, ptr<uint32_t>(s.ucnt), ptr<uint64_t>(s.offsets), ptr<unsigned long long>(L.soff),
        ptr<unsigned long long>(m.cmp_info));
    std::vector<uint64_t> info(3 * np);
    if (!(st = cuda_check(cudaGetLastError(), "pending")).ok()) return st;
    if (!(st = sync_read(s, info.data(), m.cmp_info.p, np * 24, "pending")).ok()) return st;
    for (uint64_t q = 0; q < np; ++q) {
      const uint32_t U = (uint32_t)info[3 * q];
      if (U <= (uint32_t)kCmpChunk) continue;
      uint64_t slots = 1024;
      while (slots < 2ull * U) slots <<= 1;
      if (!(st = ensure(s, m.cmp, slots * 8 + 64)).ok()) return st;
      unsigned long long* set = ptr<unsigned long long>(m.cmp);
      unsigned int* flags = reinterpret_cast<unsigned int*>(set + slots);
      const uint64_t noff = info[3 * q + 1], soff = info[3 * q + 2];
      cudaMemsetAsync(set, 0xFF, slots * 8, s.stream);
      cudaMemsetAsync(flags, 0, 8, s.stream);
      const unsigned gb = grid_for(s, U, kThreads);
      k_big_insert<<<gb, kThreads, 0, s.stream>>>(ptr<unsigned long long>(L.pool) + soff, U, set, slots - 1, flags);
      k_big_lookup<<<gb, kThreads, 0, s.stream>>>(node_sig(s), noff, U, set, slots - 1, flags);
      k_big_result<<<1, 1, 0, s.stream>>>(flags, U, match + q);
      if (!(st = cuda_check(cudaGetLastError(), "long compare")).ok()) return st;
    }
    k_resolve<<<grid_for(s, np, kThreads), kThreads, 0, s.stream>>>(la, np, match, retry, start, sc + 2, L.tcap - 1);
    uint64_t nr = 0;
    if (!(st = cuda_check(cudaGetLastError(), "long compare")).ok()) return st;
    if (!(st = sync_read(s, &nr, sc + 2, 8, "long compare")).ok()) return st;
    // the heads still unmatched probe on from their next slot
    if (nr) {
      cudaMemcpyAsync(heads, retry, nr * 4, cudaMemcpyDeviceToDevice, s.stream);
    }
    la.start = start;
    la.count = nr;
  }
  if (n_missed) {  // their labels: kept by unchanged blocks, else new; then their signatures stored
    cudaMemsetAsync(sc + 3, 0, 8, s.stream);
    k_assign_missed<<<(unsigned)std::min<uint64_t>((n_missed + 7) / 8, (uint64_t)s.sms * 8), kThreads, 0, s.stream>>>(
        sa, ns, la, n_missed, gold, gsize, ptr<uint32_t>(L.cnt));
    uint64_t nb = 0;
    if (!(st = cuda_check(cudaGetLastError(), "new labels")).ok()) return st;
    if (!(st = sync_read(s, &nb, sc + 3, 8, "new labels")).ok()) return st;
    if (!(st = copy_long_signatures(s, sa, ns, big, nb)).ok()) return st;
    L.entries += n_missed;
  }
  uint32_t e = 0;
  if (!(st = sync_read(s, &e, s.d_err.p, 4, "store")).ok()) return st;
  if (e & 1u) {
    *fits = false;
    return Status::Ok();
  }
  const uint64_t words = s.n / 32 + 1;
  cudaMemsetAsync(m.changed.p, 0, words * 4, s.stream);
  k_assign<<<grid_for(s, count, kThreads), kThreads, 0, s.stream>>>(
      list, count, ptr<uint32_t>(s.rep), ptr<uint32_t>(m.newlab), ptr<uint32_t>(s.p2o), ptr<uint32_t>(L.lab),
      ptr<uint32_t>(m.changed), ptr<uint32_t>(L.cnt), sc + 11);
  return cuda_check(cudaGetLastError(), "assign labels");
}

}  // namespace

void release_level(Store& s, MaintLevel& L) {
  Buf* b[] = {&L.lab, &L.tkey, &L.tval, &L.sfirst, &L.scount, &L.soff, &L.pool, &L.cnt, &L.ctr};
  for (Buf* x : b) release(s, *x);
}

void maint_invalidate(Store& s) {
  s.mt.valid = false;
  s.mt.k = 0;
}

void maint_release(Store& s) {
  MaintState& m = s.mt;
  for (MaintLevel& L : m.lv) release_level(s, L);
  m.lv.clear();
  Buf* b[] = {&m.fmask, &m.fnext, &m.changed, &m.seeds, &m.list, &m.pend, &m.prev_int, &m.newlab,
              &m.minid, &m.src, &m.misc, &m.woff, &m.cmp, &m.cmp_info, &m.big, &m.huge, &m.coarse,
              &m.gold, &m.gsize, &m.hit};
  for (Buf* x : b) release(s, *x);
  m.valid = false;
  m.k = 0;
}

// Largest node label of the alive nodes (internal order: alive ones first).
__global__ void k_max_node_label(uint64_t n_alive, const uint32_t* nlabel, unsigned int* out) {
  unsigned int mx = 0;
  GRID_STRIDE(p, n_alive) mx = max(mx, nlabel[p]);
  mx = __reduce_max_sync(kFullMask, mx);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

Status max_node_label(Store& s, uint32_t* out) {
  unsigned long long* sc = ptr<unsigned long long>(s.mt.misc);
  cudaMemsetAsync(sc + 13, 0, 8, s.stream);
  k_max_node_label<<<grid_for(s, std::max<uint64_t>(s.n_alive, 1), kThreads), kThreads, 0, s.stream>>>(
      s.n_alive, ptr<uint32_t>(s.nlabel), reinterpret_cast<unsigned int*>(sc + 13));
  uint64_t v = 0;
  Status st = cuda_check(cudaGetLastError(), "node labels");
  if (st.ok()) st = sync_read(s, &v, sc + 13, 8, "node labels");
  *out = (uint32_t)v;
  return st;
}

uint32_t bits_of(uint64_t v) {  // bits for values 0..v
  uint32_t b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

// The labels a store's keys carry fit its pbits: node labels (level 0) and
// original ids (every later label, < n).
Status labels_fit(Store& s, bool* fit) {
  uint32_t mx = 0;
  Status st = max_node_label(s, &mx);
  if (!st.ok()) return st;
  const uint64_t top = std::max<uint64_t>((uint64_t)mx, std::max<uint64_t>(s.n, 1) - 1);
  *fit = bits_of(top) <= s.mt.pbits && s.label_bits + s.mt.pbits <= 32;
  return Status::Ok();
}

Status maint_build(Store& s, uint32_t k) {
  MaintState& m = s.mt;
  m.valid = false;
  if (!s.has_levels) return Status::Err(KBISIM_ERR_STATE, "no computed levels");
  Status st;
  if (!(st = ensure_common(s)).ok()) return st;
  {  // the stores' key width: 32-bit words when labels up to twice the node count fit
    uint32_t mx = 0;
    if (!(st = max_node_label(s, &mx)).ok()) return st;
    m.pbits = bits_of(std::max<uint64_t>((uint64_t)mx, 2 * std::max<uint64_t>(s.n, 1) - 1));
    m.key32 = s.label_bits + m.pbits <= 32;
  }
  for (size_t j = k + 1; j < m.lv.size(); ++j) release_level(s, m.lv[j]);
  m.lv.resize(k + 1);
  const uint64_t n = s.n;
  for (uint32_t j = 0; j <= k; ++j)
    if (!(st = ensure(s, m.lv[j].lab, std::max<uint64_t>(n, 1) * 4)).ok()) return st;
  k_lab0<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, s.n_alive, ptr<uint32_t>(s.o2p),
                                                              ptr<uint32_t>(s.nlabel), ptr<uint32_t>(m.lv[0].lab));
  for (uint32_t j = 1; j <= k; ++j) {
    const uint32_t l = std::min(j, s.computed);
    k_lab_from_level<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, ptr<uint32_t>(s.o2p),
                                                                          ptr<uint32_t>(s.level[l]),
                                                                          ptr<uint32_t>(m.lv[j].lab));
    if (!(st = build_level_store(s, j, s.counts[l])).ok()) return st;
  }
  m.k = k;
  m.valid = true;
  return Status::Ok();
}

Status maint_update(Store& s, const kbisim_batch* b, uint32_t k, uint64_t* missing, bool* done) {
  MaintState& m = s.mt;
  *done = false;
  if (!m.valid || k > m.k || !b || b->n_del_nodes) return Status::Ok();
  Status st;
  // the batch's edge sources, staged before the graph changes (original ids)
  const uint64_t ns = b->n_ins + b->n_del;
  if (!(st = ensure(s, m.src, std::max<uint64_t>(ns, 1) * 4)).ok()) return st;
  const cudaMemcpyKind kind = b->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (b->n_ins && !(st = cuda_check(cudaMemcpyAsync(m.src.p, b->ins_src, b->n_ins * 4, kind, s.stream), "stage")).ok())
    return st;
  if (b->n_del && !(st = cuda_check(cudaMemcpyAsync(ptr<uint32_t>(m.src) + b->n_ins, b->del_src, b->n_del * 4, kind,
                                                    s.stream), "stage")).ok())
    return st;
  const uint64_t n0 = s.n;
  if (!(st = apply_batch(s, b, missing)).ok()) return st;
  *done = true;  // from here on the graph is the updated one
  if (m.key32 && (s.n > n0 || s.label_bits + m.pbits > 32)) {  // new nodes or wider labels may no longer fit
    bool fit = true;
    if (!(st = labels_fit(s, &fit)).ok()) return st;
    if (!fit) {
      m.valid = false;
      m.reason = KBISIM_MAINT_CAPACITY;
      return Status::Ok();
    }
  }
  m.incremental = 0;
  m.frontier_nodes = 0;
  m.levels = 0;
  const uint64_t n = s.n, words = n / 32 + 1;
  if (!(st = ensure_common(s)).ok()) return st;
  // labels of added nodes
  for (uint32_t j = 0; j <= m.k; ++j) {
    if (!(st = grow_keep(s, m.lv[j].lab, std::max<uint64_t>(n, 1) * 4, n0 * 4)).ok()) return st;
    if (n > n0)
      k_lab_grow<<<grid_for(s, n - n0, kThreads), kThreads, 0, s.stream>>>(n0, n, ptr<uint32_t>(s.o2p),
                                                                           ptr<uint32_t>(s.nlabel), j == 0,
                                                                           ptr<uint32_t>(m.lv[j].lab));
  }
  // seeds: sources of the batch's edges and the new nodes
  cudaMemsetAsync(m.seeds.p, 0, words * 4, s.stream);
  if (ns) k_seed_sources<<<grid_for(s, ns, kThreads), kThreads, 0, s.stream>>>(ns, ptr<uint32_t>(m.src),
                                                                               ptr<uint32_t>(s.o2p),
                                                                               ptr<uint32_t>(m.seeds));
  if (n > n0) k_seed_new<<<grid_for(s, n - n0, kThreads), kThreads, 0, s.stream>>>(n0, n, ptr<uint32_t>(s.o2p),
                                                                                  ptr<uint32_t>(m.seeds));
  cudaMemcpyAsync(m.fmask.p, m.seeds.p, words * 4, cudaMemcpyDeviceToDevice, s.stream);
  k_to_internal<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, ptr<uint32_t>(s.p2o),
                                                                      ptr<uint32_t>(m.lv[0].lab),
                                                                      ptr<uint32_t>(m.prev_int));
  if (!(st = cuda_check(cudaGetLastError(), "seeds")).ok()) return st;
  unsigned long long* sc = ptr<unsigned long long>(m.misc);
  bool fits = true;
  uint64_t nodes = 0;
  for (uint32_t j = 1; j <= m.k && fits; ++j) {
    // frontier of level j: count, switch back when large, list
    cudaMemsetAsync(sc + 8, 0, 16, s.stream);
    cudaMemsetAsync(sc + 11, 0, 8, s.stream);  // labels changed at this level (k_assign)
    k_popc_sum<<<grid_for(s, words, kThreads), kThreads, 0, s.stream>>>(ptr<uint32_t>(m.fmask), words, sc + 8);
    uint64_t count = 0;
    if (!(st = cuda_check(cudaGetLastError(), "frontier")).ok()) return st;
    if (!(st = sync_read(s, &count, sc + 8, 8, "frontier")).ok()) return st;
    if (count > kFrontierFloor && (double)count > s.maint_frontier_max * (double)std::max<uint64_t>(s.n_alive, 1)) {
      fits = false;
      m.reason = KBISIM_MAINT_FRONTIER;
      break;
    }
    nodes += count;
    if (count) {
      k_bits_to_list<<<grid_for(s, words, kThreads), kThreads, 0, s.stream>>>(ptr<uint32_t>(m.fmask), words, n,
                                                                              ptr<uint32_t>(m.list), sc + 9);
      if (!(st = cuda_check(cudaGetLastError(), "frontier list")).ok()) return st;
      if (!(st = update_level(s, j, count, &fits)).ok()) return st;
      if (!fits) {
        m.reason = KBISIM_MAINT_CAPACITY;
        break;
      }
    } else {
      cudaMemsetAsync(m.changed.p, 0, words * 4, s.stream);
    }
    if (j == m.k) break;
    // next frontier: seeds | changed | parents of changed
    cudaMemsetAsync(m.fnext.p, 0, words * 4, s.stream);
    if (s.m) {
      const uint64_t cwords = (words + 31) / 32;
      if (!(st = ensure(s, m.coarse, cwords * 4)).ok()) return st;
      cudaMemsetAsync(m.coarse.p, 0, cwords * 4, s.stream);
      k_changed_words<<<grid_for(s, words, kThreads), kThreads, 0, s.stream>>>(ptr<uint32_t>(m.changed), words,
                                                                            ptr<uint32_t>(m.coarse));
      k_frontier_pull<<<(unsigned)s.sms * 8, kThreads, 0, s.stream>>>(
          s.m, n, ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst), ptr<uint32_t>(m.changed), ptr<uint32_t>(m.coarse),
          sc + 11, ptr<uint32_t>(m.fnext));
    }
    k_or3<<<grid_for(s, words, kThreads), kThreads, 0, s.stream>>>(words, ptr<uint32_t>(m.seeds),
                                                                    ptr<uint32_t>(m.changed), ptr<uint32_t>(m.fnext));
    std::swap(m.fmask, m.fnext);
    k_to_internal<<<grid_for(s, n, kThreads), kThreads, 0, s.stream>>>(n, ptr<uint32_t>(s.p2o),
                                                                        ptr<uint32_t>(m.lv[j].lab),
                                                                        ptr<uint32_t>(m.prev_int));
    if (!(st = cuda_check(cudaGetLastError(), "next frontier")).ok()) return st;
  }
  if (!fits) {
    // switch back: the caller recomputes every level and rebuilds the state
    m.valid = false;
    return Status::Ok();
  }
  m.frontier_nodes = nodes;
  m.levels = m.k;
  m.incremental = 1;
  m.reason = 0;
  // canonical identifiers of levels 0..k: level 0 by its own grouping, the
  // others from their labels; rounds and early stop as a full computation
  // decides them
  if (s.level.size() < (size_t)m.k + 1) s.level.resize(m.k + 1);
  for (uint32_t j = 0; j <= m.k; ++j)
    if (!(st = ensure(s, s.level[j], std::max<uint64_t>(n, 1) * 4)).ok()) return st;
  if (s.counts.size() < (size_t)m.k + 1) s.counts.resize(m.k + 1, 0);
  if (!(st = compute_level0(s)).ok()) return st;
  // (every level writes its alone flags, so they are those of the last
  // computed level when the loop ends; with k = 0, level 0's own)
  uint32_t rounds = k;
  for (uint32_t j = 1; j <= k; ++j) {
    uint64_t blocks = 0;
    if (!(st = canonical_from_labels(s, j, ptr<uint32_t>(s.level[j]), &blocks, true)).ok()) return st;
    s.counts[j] = blocks;
    if (s.early_stop && blocks == s.counts[j - 1]) {
      rounds = j;
      break;
    }
  }
  if (k == 0) rounds = 0;
  s.computed = rounds;
  s.rounds_run = rounds;
  s.stable = rounds > 0 && s.counts[rounds] == s.counts[rounds - 1];
  s.stats.assign(rounds, kbisim_round_stats());
  for (uint32_t r = 1; r <= rounds; ++r) s.stats[r - 1].blocks = s.counts[r];
  s.has_levels = true;
  return cuda_check(cudaStreamSynchronize(s.stream), "maintenance");
}

}  // namespace kb
