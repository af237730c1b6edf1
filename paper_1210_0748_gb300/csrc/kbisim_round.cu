// One refinement round of k-bisimulation on the GPU, level 0, and the
// once-per-graph relabelling of node ids.
//
// Round i (Algorithm 1, the k > 0 branch; Definition 3; Proposition 2):
//   (a) gather: for every edge e = (u, l, v) of the source-sorted edge table,
//       the element (l, pId_{i-1}(v))  -- Algorithm 1 fills pId_old(tId) by a
//       merge join of the edge and node tables; here it is a direct gather;
//   (b) per source node: drop duplicate elements and sort the rest (the
//       sorted, duplicate-free F of Algorithm 1), written at the node's CSR
//       offset;
//   (c) a 64-bit hash of (pId_{i-1}(u), the element set)  -- it only routes
//       nodes to candidate groups; it stands in for the signature store S
//       (Section 3, "Data structures for S");
//   (d) group nodes with equal hash in an open-addressing table that keeps the
//       smallest original node id per hash, compare every node's signature
//       with that node's exactly (a hash collision never merges two blocks),
//       repair collisions, and number blocks by their smallest original id;
//   (e) the caller stops when the block count is unchanged.
// Level 0 groups nodes by label the same way (Algorithm 1, k = 0 branch).
//
// Degree tiers of step (a)-(c): out-degree <= 32 uses P = 2^c lanes per node
// and a bitonic network in registers; 33..256 one warp per node; 257..4096
// one CTA per node (both with a shared-memory hash set, then a counting sort);
// larger "hubs" are partitioned by key bits into buckets of about 2048
// distinct keys, each bucket deduplicated and sorted by one CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "kbisim_internal.cuh"

namespace kb {

namespace {
constexpr unsigned kFull = 0xFFFFFFFFu;
}  // namespace

// --------------------------------------------------------------------------
// Kernel timing (CUDA events on the handle's stream)
// --------------------------------------------------------------------------
struct KernelTimer {
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> done;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

Status timer_collect(Store& s) {
  if (!s.timer) return Status::Ok();
  for (auto& r : s.timer->done) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    s.total_ms[r.cls] += ms;
    s.timer->pool.push_back(r.a);
    s.timer->pool.push_back(r.b);
  }
  s.timer->done.clear();
  return cuda_check(cudaGetLastError(), "timer");
}

void timer_destroy(Store& s) {
  if (!s.timer) return;
  for (auto e : s.timer->pool) cudaEventDestroy(e);
  for (auto& r : s.timer->done) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete s.timer;
  s.timer = nullptr;
}

namespace {

// Records one CUDA event pair around the kernels launched in its scope.
// Events around a group of launches of one kernel class; `kernels` is the
// number of this library's kernels the group launches (clears by
// cudaMemsetAsync are not counted).
struct TimedScope {
  Store& s;
  int cls;
  KernelTimer::Rec rec;
  TimedScope(Store& st, int c, int kernels) : s(st), cls(c) {
    s.launches[c] += (uint64_t)kernels;
    if (!s.timing) return;
    if (!s.timer) s.timer = new KernelTimer();
    rec.cls = c;
    rec.a = s.timer->get();
    rec.b = s.timer->get();
    cudaEventRecord(rec.a, s.stream);
  }
  ~TimedScope() {
    if (!s.timing) return;
    cudaEventRecord(rec.b, s.stream);
    s.timer->done.push_back(rec);
  }
};

template <typename T>
T* ptr(Buf& b) { return static_cast<T*>(b.p); }

inline unsigned grid_for(uint64_t work, unsigned per_block) {
  uint64_t g = (work + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, 0x7FFFFFFFull));
}

Status launch_check(const char* what) { return cuda_check(cudaGetLastError(), what); }

int sm_count(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 148;
  if (!cached[device]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    cached[device] = v > 0 ? v : 148;
  }
  return cached[device];
}

// --------------------------------------------------------------------------
// Small device helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cas(uint32_t* a, uint32_t c, uint32_t v) { return atomicCAS(a, c, v); }
__device__ __forceinline__ uint64_t cas(uint64_t* a, uint64_t c, uint64_t v) {
  return atomicCAS((unsigned long long*)a, (unsigned long long)c, (unsigned long long)v);
}

// L2 cache policies (sm_90+ createpolicy): streamed edge data and signature
// words are marked evict-first, the gathered identifier array evict-last, so
// the random gathers of pId_{i-1}[dst] keep hitting L2 while the edge table
// streams past.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Loads with an L2 policy, predicated (0 when p is false, no access), so
// loads of several items are issued back to back without a branch between them.
__device__ __forceinline__ uint32_t ld_hint_if(const uint32_t* a, uint64_t pol, bool p) {
  uint32_t v;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tmov.u32 %0, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;\n\t}"
      : "=r"(v) : "l"(a), "l"(pol), "r"((uint32_t)p));
  return v;
}
__device__ __forceinline__ uint32_t ld_hint_if(const uint8_t* a, uint64_t pol, bool p) {
  uint32_t v;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tmov.u32 %0, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;\n\t}"
      : "=r"(v) : "l"(a), "l"(pol), "r"((uint32_t)p));
  return v;
}

// Lanes of a sub-warp team (NT < 32) or the whole warp.
template <int NT>
__device__ __forceinline__ unsigned team_mask() {
  if (NT >= 32) return kFull;
  const unsigned lane = threadIdx.x & 31;
  return ((1u << (NT & 31)) - 1u) << (lane & ~(unsigned)(NT - 1));
}

template <int NT>
__device__ __forceinline__ void team_sync() {
  if (NT <= 32) __syncwarp(team_mask<NT>()); else __syncthreads();
}

// --------------------------------------------------------------------------
// Team dedupe in shared memory (no sorting)
// --------------------------------------------------------------------------
// A team (one warp, or one CTA) inserts keys into an open-addressing set in
// shared memory.  The first inserter of a key owns it: it writes the key to
// the node's output at the next free position and adds its hash term.  The
// order of a node's distinct keys is therefore arbitrary: signatures are
// compared as sets (see k_group_verify / k_verify_long).
template <typename K>
struct TeamSet {
  K* set;          // [hcap]
  K* uniq;         // [ucap] distinct keys (hub buckets only)
  uint32_t* sh;    // [4]: distinct count, saw-the-empty-key flag, overflow flag, spare
  uint32_t* red;   // [NT/32] reduction scratch
};

template <typename K>
__host__ __device__ constexpr size_t team_set_bytes(int hcap, int ucap, int nt) {
  return ((size_t)hcap * sizeof(K) + (size_t)ucap * sizeof(K) + 16 + (size_t)(nt / 32) * 8 + 15) / 16 * 16;
}

template <typename K>
__device__ __forceinline__ TeamSet<K> carve_set(char* base, int hcap, int ucap) {
  TeamSet<K> t;
  t.set = reinterpret_cast<K*>(base);
  t.uniq = t.set + hcap;
  t.sh = reinterpret_cast<uint32_t*>(t.uniq + ucap);
  t.red = t.sh + 4;
  return t;
}

// Smallest power of two >= 2 n, clamped to [64, cap].
__device__ __forceinline__ int set_size_for(uint64_t n, int cap) {
  int h = 64;
  while (h < cap && (uint64_t)h < 2 * n) h <<= 1;
  return h;
}

template <int NT, typename K>
__device__ __forceinline__ void set_clear(const TeamSet<K>& ts, int hcap, int rank) {
  for (int i = rank; i < hcap; i += NT) ts.set[i] = KeyOps<K>::kEmpty;
  if (rank < 4) ts.sh[rank] = 0;
}

// Insert k; true if this call inserted it first.  Probing is bounded by the
// set size; a full set raises the overflow flag.
template <typename K>
__device__ __forceinline__ bool set_insert(const TeamSet<K>& ts, int hcap, K k) {
  if (k == KeyOps<K>::kEmpty) return atomicExch(&ts.sh[1], 1u) == 0u;
  volatile K* vset = ts.set;
  const uint32_t hmask = (uint32_t)(hcap - 1);
  uint32_t s = (uint32_t)k & hmask;
  for (int t = 0; t < hcap; ++t) {
    const K cur = vset[s];
    if (cur == k) return false;
    if (cur == KeyOps<K>::kEmpty) {
      const K old = cas(&ts.set[s], KeyOps<K>::kEmpty, k);
      if (old == KeyOps<K>::kEmpty) return true;
      if (old == k) return false;
    }
    s = (s + 1) & hmask;
  }
  ts.sh[2] = 1u;
  return false;
}

// Membership test in a set built by set_insert.
template <typename K>
__device__ __forceinline__ bool set_find(const TeamSet<K>& ts, int hcap, K k) {
  if (k == KeyOps<K>::kEmpty) return ts.sh[1] != 0u;
  const uint32_t hmask = (uint32_t)(hcap - 1);
  uint32_t s = (uint32_t)k & hmask;
  for (int t = 0; t < hcap; ++t) {
    const K cur = ts.set[s];
    if (cur == k) return true;
    if (cur == KeyOps<K>::kEmpty) return false;
    s = (s + 1) & hmask;
  }
  return false;
}

// Sum over the team (modulo 2^32); valid in every lane for NT <= 32, in rank
// 0 otherwise.
template <int NT>
__device__ __forceinline__ uint32_t team_sum(uint32_t t, uint32_t* red, int rank) {
  const unsigned m = team_mask<NT>();
  t = __reduce_add_sync(m, t);
  if (NT <= 32) return t;
  if ((rank & 31) == 0) red[rank >> 5] = t;
  __syncthreads();
  uint32_t tot = 0;
  if (rank == 0)
    for (int w = 0; w < NT / 32; ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// --------------------------------------------------------------------------
// Signature kernels
// --------------------------------------------------------------------------
struct SigArgs {
  const uint64_t* off;
  const uint32_t* dst;
  const void* lab;
  const uint32_t* prev;
  void* sigkey;
  uint32_t* ucnt;
  uint64_t* hash;
  uint64_t seed;
  uint64_t mask;
  int pbits;          // bits of a child identifier in a 32-bit key
  uint32_t* err;
  const uint32_t* fmask;  // bitmap over internal ids of the nodes to sign (NULL = all)
};

// The node is to be signed this pass (every node unless a frontier mask is set).
__device__ __forceinline__ bool in_mask(const SigArgs& a, uint64_t p) {
  return !a.fmask || ((a.fmask[p >> 5] >> (p & 31)) & 1u);
}

constexpr int kLoadBatch = 16;  // edges whose loads a thread-per-node kernel issues together

struct Policies {
  uint64_t stream, keep;
  __device__ __forceinline__ Policies() : stream(policy_evict_first()), keep(policy_evict_last()) {}
};

// Keys of N edges base + i * stride into key[O + i] (i < N; an edge counts
// while it is below end): labels and targets first, then the identifier
// gathers, then the packing, so all loads of the batch are in flight together.
template <int N, int O, int M, typename LabelT, typename K>
__device__ __forceinline__ void edge_keys(const SigArgs& a, uint64_t base, uint32_t stride, uint64_t end,
                                          const Policies& pol, K (&key)[M]) {
  static_assert(O + N <= M, "batch out of range");
  const LabelT* lab = static_cast<const LabelT*>(a.lab);
  uint32_t l[N], t[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t e = base + (uint64_t)i * stride;
    l[i] = ld_hint_if(lab + e, pol.stream, e < end);
    t[i] = ld_hint_if(a.dst + e, pol.stream, e < end);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = ld_hint_if(a.prev + t[i], pol.keep, base + (uint64_t)i * stride < end);
#pragma unroll
  for (int i = 0; i < N; ++i) key[O + i] = KeyOps<K>::make(l[i], t[i], a.pbits);
}

// Keys of edges off .. off + S (those below end) in batches of B.
template <int O, int B, int S, typename LabelT, typename K>
__device__ __forceinline__ void edge_key_batches(const SigArgs& a, uint64_t off, uint64_t end, const Policies& pol,
                                                 K (&key)[S]) {
  if constexpr (O < S) {
    edge_keys<B, O, S, LabelT, K>(a, off + O, 1u, end, pol, key);
    edge_key_batches<O + B, B, S, LabelT, K>(a, off, end, pol, key);
  }
}

// Out-degree <= 64: one thread per node, its keys in registers (S = 2^c
// slots, S >= out-degree).  A key is kept unless an earlier slot holds the
// same key, so no shuffles, sorting or shared memory are needed.
template <int S, typename LabelT, typename K>
__device__ __forceinline__ void sig_thread_node(const SigArgs& a, uint64_t p, const Policies& pol) {
  if (!in_mask(a, p)) return;
  const uint64_t off = a.off[p];
  const uint32_t d = (uint32_t)(a.off[p + 1] - off);
  K k[S];
  edge_key_batches<0, (S < kLoadBatch ? S : kLoadBatch), S, LabelT, K>(a, off, off + d, pol, k);
  K* out = static_cast<K*>(a.sigkey) + off;
  uint64_t term = 0;
  uint32_t U = 0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    bool keep = i < (int)d;
#pragma unroll
    for (int j = 0; j < i; ++j) keep = keep && k[j] != k[i];
    if (keep) {
      out[U] = k[i];
      term = term_add(term, elem_term(k[i], a.seed));
      ++U;
    }
  }
  a.ucnt[p] = U;
  a.hash[p] = node_hash(term, a.prev[p], U, a.seed, a.mask);
}

// The same for the 32 nodes of a warp (consecutive internal ids, so their
// edges are one contiguous range of at most 32 * S edges), with the edges
// staged through the warp's shared-memory buffer: the warp loads the range
// coalesced (lane l takes edges l, l + 32, ...) and makes the keys, each
// thread reads its node's keys back, keeps the distinct ones as above and
// writes them over its own keys, and the warp stores the whole range
// coalesced (slots past a node's distinct count keep leftovers that nothing
// reads).  Lanes past the class end take part without a node.
template <int S, typename LabelT, typename K>
__device__ __forceinline__ void sig_warp_staged(const SigArgs& a, uint64_t p_first, uint32_t nvalid, K* wsm,
                                                const Policies& pol) {
  const uint32_t lane = threadIdx.x & 31;
  const bool valid = lane < nvalid;
  const uint64_t p = p_first + lane;
  if (a.fmask && !__any_sync(0xFFFFFFFFu, valid && in_mask(a, p))) return;
  const uint64_t base = a.off[p_first];
  const uint64_t end = a.off[p_first + nvalid];
  const uint32_t T = (uint32_t)(end - base);  // at most 32 * S
  {
    K kk[S];
    edge_keys<S, 0, S, LabelT, K>(a, base + lane, 32u, end, pol, kk);
#pragma unroll
    for (int t = 0; t < S; ++t)
      if (lane + 32u * t < T) wsm[lane + 32u * t] = kk[t];
  }
  __syncwarp();
  uint32_t r0 = 0, d = 0;
  if (valid) {
    const uint64_t o = a.off[p];
    r0 = (uint32_t)(o - base);
    d = (uint32_t)(a.off[p + 1] - o);
  }
  K k[S];
#pragma unroll
  for (int i = 0; i < S; ++i) k[i] = i < (int)d ? wsm[r0 + i] : (K)0;
  __syncwarp();  // every read is done before the distinct keys go back
  uint64_t term = 0;
  uint32_t U = 0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    bool keep = i < (int)d;
#pragma unroll
    for (int j = 0; j < i; ++j) keep = keep && k[j] != k[i];
    if (keep) {
      wsm[r0 + U] = k[i];
      term = term_add(term, elem_term(k[i], a.seed));
      ++U;
    }
  }
  __syncwarp();
  K* out = static_cast<K*>(a.sigkey) + base;
#pragma unroll
  for (int t = 0; t < S; ++t)
    if (lane + 32u * t < T) out[lane + 32u * t] = wsm[lane + 32u * t];
  if (valid) {
    a.ucnt[p] = U;
    a.hash[p] = node_hash(term, a.prev[p], U, a.seed, a.mask);
  }
}

// Largest S staged through shared memory (out-degree 9..16); the 17..32 class
// keeps one node per thread, whose registers a staged copy would double.
template <typename K>
__host__ __device__ constexpr int staged_max_s() {
  return 16;
}

// Resident CTAs per multiprocessor the small-class kernels are compiled for:
// all 8 (32 registers) for out-degree <= 8 with 32-bit keys, fewer where more
// keys sit in registers.
template <int LAST, typename K>
__host__ __device__ constexpr int small_min_blocks() {
  return LAST <= 4 ? (sizeof(K) == 4 ? 8 : 6) : (LAST == 5 ? 4 : (sizeof(K) == 4 ? 4 : 2));
}

struct SmallLaunch {
  uint64_t start[kSmallClasses];
  uint64_t count[kSmallClasses];
  uint32_t bstart[kSmallClasses + 1];
};

constexpr int kSmallThreads = 256;

// Class 0 (no out-edges): signature (pId_{i-1}(u), {}); classes 1..7
// (out-degree 1..64): one node per thread.  Classes FIRST..LAST per launch,
// so the 64-slot class (most registers) does not limit the occupancy of the
// others.
template <int FIRST, int LAST, typename LabelT, typename K>
__global__ void __launch_bounds__(kSmallThreads, small_min_blocks<LAST, K>()) k_sig_small(SigArgs a, SmallLaunch L) {
  // per-warp staging buffer for the largest class of this launch that is staged
  constexpr int kSLast = LAST == 0 ? 1 : (1 << (LAST - 1));
  constexpr int kSBuf = kSLast <= staged_max_s<K>() ? kSLast : 1;
  __shared__ K stage[kSmallThreads / 32][32 * kSBuf];
  int c = FIRST;
  while (c < LAST && blockIdx.x >= L.bstart[c + 1]) ++c;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t idx = (uint64_t)(blockIdx.x - L.bstart[c]) * kSmallThreads + threadIdx.x;
  const uint64_t widx = idx - lane;
  if (widx >= L.count[c]) return;  // the whole warp is past the class end
  const uint64_t left = L.count[c] - widx;
  const uint32_t nvalid = left < 32 ? (uint32_t)left : 32u;
  const uint64_t p = L.start[c] + idx;
  const Policies pol;
  K* wsm = stage[threadIdx.x >> 5];
#define KB_SMALL_CLASS(C, S)                                                                  \
  case C:                                                                                     \
    if constexpr (LAST >= C) {                                                                \
      if constexpr (S <= kSBuf) sig_warp_staged<S, LabelT, K>(a, L.start[c] + widx, nvalid, wsm, pol); \
      else if (idx < L.count[c]) sig_thread_node<S, LabelT, K>(a, p, pol);                    \
    }                                                                                         \
    break;
  switch (c) {
    case 0:
      if (idx < L.count[c] && in_mask(a, p)) {
        a.ucnt[p] = 0;
        a.hash[p] = node_hash(0, a.prev[p], 0, a.seed, a.mask);
      }
      break;
    KB_SMALL_CLASS(1, 1)
    KB_SMALL_CLASS(2, 2)
    KB_SMALL_CLASS(3, 4)
    KB_SMALL_CLASS(4, 8)
    KB_SMALL_CLASS(5, 16)
    KB_SMALL_CLASS(6, 32)
    default:
      if constexpr (LAST >= 7)
        if (idx < L.count[c]) sig_thread_node<64, LabelT, K>(a, p, pol);
      break;
  }
#undef KB_SMALL_CLASS
}

// ---- out-degree 65..4096: CTA chunks of whole nodes -----------------------
// A chunk is a run of consecutive medium nodes with at most kChunkEdges edges
// in all; their edges are contiguous in the relabelled CSR.  One CTA:
//  1. loads the chunk's edges coalesced, kChunkItems per thread, and makes
//     their keys (every load is in flight before the first key is used);
//  2. inserts each key into its node's region of a shared-memory hash set
//     (node j owns slots [2 o_j, 2 o_{j+1}), o_j its first edge in the chunk,
//     so a region is at most half full).  The lane whose insert puts a key
//     into the set writes it out at once: the 32 consecutive edges of a warp
//     belong to at most two nodes, so each node's output position is claimed
//     once per warp step;
//  3. adds the hash terms of the keys a warp step inserted to their node's
//     sums as it claims their output positions, and at the end writes each
//     node's distinct-key count and hash.
// The key equal to the empty-slot marker is kept as a per-node flag.

// A chunk CTA of NT threads takes up to NT * kChunkItems edges of nodes with
// out-degree >= MIN_DEG (> 32, so that 32 consecutive edges meet at most two
// nodes).
template <int NT, int MIN_DEG>
struct ChunkShape {
  static_assert(MIN_DEG > 32, "a warp step must meet at most two nodes");
  static constexpr int kEdges = NT * kChunkItems;
  static constexpr int kSlots = 2 * kEdges;
  static constexpr int kMaxNodes = kEdges / MIN_DEG + 1;
};

template <typename K, int NT, int MIN_DEG>
struct ChunkSmem {
  using Shape = ChunkShape<NT, MIN_DEG>;
  K slot[Shape::kSlots];
  uint32_t off[Shape::kMaxNodes + 1];  // node starts relative to the chunk's first edge
  uint32_t cnt[Shape::kMaxNodes];      // distinct keys written per node
  uint32_t empty[Shape::kMaxNodes];    // the node's key equal to KeyOps<K>::kEmpty was seen
  uint32_t lo[Shape::kMaxNodes];       // term sum halves of the node's distinct keys
  uint32_t hi[Shape::kMaxNodes];
};

// Chunk kernel shapes: out-degree 33..64 and 65..1024 in 128-thread CTAs,
// 1025..4096 and hub pieces in 512-thread CTAs.
constexpr int kChunkMin64 = kSmallMax / 2 + 1, kChunkMin1K = kSmallMax + 1, kChunkMin4K = kWarp2Max + 1;
constexpr int kChunkMinHub = kBlockMax + 1;

__device__ __forceinline__ uint32_t key_h32(uint32_t k) { return k; }
__device__ __forceinline__ uint32_t key_h32(uint64_t k) { return (uint32_t)(k >> 32) ^ (uint32_t)k; }

// Home slot of k in a region of rs slots: monotone in the key's top bits.
template <typename K>
__device__ __forceinline__ uint32_t region_home(K k, uint32_t rs) {
  return (uint32_t)(((uint64_t)key_h32(k) * rs) >> 32);
}

// Shared-memory compare-and-swap by shared-window address (no generic addressing).
__device__ __forceinline__ uint32_t atoms_cas(uint32_t a, uint32_t c, uint32_t v) {
  uint32_t r;
  asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(r) : "r"(a), "r"(c), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint64_t atoms_cas(uint32_t a, uint64_t c, uint64_t v) {
  uint64_t r;
  asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(r) : "r"(a), "l"(c), "l"(v) : "memory");
  return r;
}

// Insert k (!= kEmpty) into the set held in slots [rb, rb + rs) of the slot
// array at shared-window address `base`; true iff this call put it there.
// The region has more slots than keys are ever inserted into it, and probing
// is bounded by its size; the compare-and-swap is the probe itself.
template <typename K>
__device__ __forceinline__ bool region_insert(uint32_t base, uint32_t rb, uint32_t rs, K k) {
  uint32_t s = rb + region_home(k, rs);
  const uint32_t re = rb + rs;
  for (uint32_t t = 0; t < rs; ++t) {
    const K cur = atoms_cas(base + s * (uint32_t)sizeof(K), KeyOps<K>::kEmpty, k);
    if (cur == KeyOps<K>::kEmpty) return true;
    if (cur == k) return false;
    if (++s == re) s = rb;
  }
  return false;
}

template <typename K, int NT, int MIN_DEG>
__device__ __forceinline__ void chunk_clear(ChunkSmem<K, NT, MIN_DEG>& sm, uint32_t slots) {
  uint4* s4 = reinterpret_cast<uint4*>(sm.slot);
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (uint32_t i = threadIdx.x; i < slots * sizeof(K) / 16; i += NT) s4[i] = ones;
  for (uint32_t i = threadIdx.x; i < (uint32_t)ChunkShape<NT, MIN_DEG>::kMaxNodes; i += NT) {
    sm.cnt[i] = 0;
    sm.empty[i] = 0;
    sm.lo[i] = 0;
    sm.hi[i] = 0;
  }
}

template <int NT, typename LabelT, typename K>
__device__ __forceinline__ void chunk_keys(const SigArgs& a, uint64_t ebase, uint32_t E, K (&key)[kChunkItems]) {
  const Policies pol;
  edge_keys<kChunkItems, 0, kChunkItems, LabelT, K>(a, ebase + threadIdx.x, NT, ebase + E, pol, key);
}

// Lanes below `lane`.
__device__ __forceinline__ unsigned lanes_below(uint32_t lane) { return (1u << lane) - 1u; }

template <int NT, int MIN_DEG, typename LabelT, typename K>
__global__ void __launch_bounds__(NT) k_sig_chunk(SigArgs a, const uint2* chunks) {
  extern __shared__ __align__(16) char smem_raw[];
  ChunkSmem<K, NT, MIN_DEG>& sm = *reinterpret_cast<ChunkSmem<K, NT, MIN_DEG>*>(smem_raw);
  const uint2 c = chunks[blockIdx.x];
  const uint64_t first = c.x;
  const uint32_t nn = c.y;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  if (a.fmask && !__syncthreads_or(tid < nn && in_mask(a, first + tid))) return;
  const uint64_t ebase = a.off[first];
  const uint32_t E = (uint32_t)(a.off[first + nn] - ebase);
  for (uint32_t i = tid; i <= nn; i += NT) sm.off[i] = (uint32_t)(a.off[first + i] - ebase);
  chunk_clear(sm, (2 * E + 3) & ~3u);
  __syncthreads();
  K key[kChunkItems];
  chunk_keys<NT, LabelT, K>(a, ebase, E, key);
  K* out = static_cast<K*>(a.sigkey) + ebase;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm.slot);
  uint32_t j = 0;
  // one copy of the loop body: the keys rotate through key[0]
#pragma unroll 1
  for (int t = 0; t < kChunkItems; ++t) {
    const uint32_t e = tid + t * NT;
    const K kt = key[0];
#pragma unroll
    for (int q = 0; q + 1 < kChunkItems; ++q) key[q] = key[q + 1];
    bool fresh = false;
    if (e < E) {
      while (sm.off[j + 1] <= e) ++j;
      fresh = kt == KeyOps<K>::kEmpty
                  ? atomicExch(&sm.empty[j], 1u) == 0u
                  : region_insert(sbase, 2 * sm.off[j], 2 * (sm.off[j + 1] - sm.off[j]), kt);
    }
    const unsigned fm = __ballot_sync(kFull, fresh);
    if (fm == 0u) continue;
    // valid lanes are a prefix of the warp and span nodes jA and jA + 1
    const uint32_t jA = __shfl_sync(kFull, j, 0);
    const bool inA = j == jA;
    const unsigned fa = fm & __ballot_sync(kFull, inA), fb = fm & ~fa;
    // the fresh keys' term sums, per node of the step, go with their count
    const uint64_t tm = fresh ? elem_term(kt, a.seed) : 0ull;
    const uint32_t loA = __reduce_add_sync(kFull, inA ? (uint32_t)tm : 0u);
    const uint32_t hiA = __reduce_add_sync(kFull, inA ? (uint32_t)(tm >> 32) : 0u);
    const uint32_t loB = __reduce_add_sync(kFull, inA ? 0u : (uint32_t)tm);
    const uint32_t hiB = __reduce_add_sync(kFull, inA ? 0u : (uint32_t)(tm >> 32));
    uint32_t base = 0;
    if (lane == 0 && fa) {
      base = atomicAdd(&sm.cnt[jA], (uint32_t)__popc(fa));
      atomicAdd(&sm.lo[jA], loA);
      atomicAdd(&sm.hi[jA], hiA);
    }
    if (lane == 31 && fb) {
      base = atomicAdd(&sm.cnt[jA + 1], (uint32_t)__popc(fb));
      atomicAdd(&sm.lo[jA + 1], loB);
      atomicAdd(&sm.hi[jA + 1], hiB);
    }
    const uint32_t bA = __shfl_sync(kFull, base, 0), bB = __shfl_sync(kFull, base, 31);
    if (fresh)
      out[sm.off[j] + (inA ? bA + __popc(fa & lanes_below(lane)) : bB + __popc(fb & lanes_below(lane)))] = kt;
  }
  __syncthreads();
  // count and hash of each node of the chunk
  for (uint32_t i = tid; i < nn; i += NT) {
    const uint64_t p = first + i;
    const uint32_t U = sm.cnt[i];
    a.ucnt[p] = U;
    a.hash[p] = node_hash(((uint64_t)sm.hi[i] << 32) | sm.lo[i], a.prev[p], U, a.seed, a.mask);
  }
}

// ---- hubs: out-degree > kBlockMax ----------------------------------------
// Pass 1 (k_hub_chunk): a CTA takes kHubChunk edges of one hub, deduplicates
// their keys in shared memory as above (one region), listing each distinct
// key once, and appends the list to the hub's buckets; the bucket of a key is
// its top bits, so equal keys from different chunks meet in one bucket.
// Hubs whose keys rarely repeat (k_hub_sample) skip the chunk set
// (k_hub_scatter).  Buckets have a fixed capacity: an append past it flags the
// hub (kErrHubOverflow) and the host repeats the hub passes with larger
// buckets for that hub, or, for a scattering hub whose buckets have grown
// twice already, with the deduplicating pass (a key repeated that often stays
// repeated in later rounds); a bucket with more distinct keys than its set
// (kErrHubSet) gives its hub more buckets.  Pass 2 (k_hub_bucket):
// one CTA per bucket deduplicates across chunks and appends the bucket's
// distinct keys at the hub's CSR offset, adding to the hub's count and term
// sums; k_hub_finish then writes each hub's count and hash.
struct HubArgs {
  uint64_t first;           // internal id of hub 0
  const uint32_t* hub_bits;
  const uint64_t* hub_bbase;
  const uint32_t* hub_cap;
  const uint64_t* hub_tbase;
  const uint32_t* bucket_hub;
  const uint4* chunks;
  uint32_t* cursor;              // per bucket: key words appended
  unsigned long long* hub_cur;   // per hub: distinct keys written
  uint32_t* hub_term;            // per hub: term sum halves (low, high)
  void* tmp;
  uint8_t* mode;                 // per hub: 1 = chunks skip their set (few repeated keys)
  const uint8_t* force;          // per hub: 1 = always the deduplicating chunk pass
  uint32_t* hub_err;             // per hub: kErrHubOverflow / kErrHubSet raised for it
};

__device__ __forceinline__ void hub_fail(const SigArgs& a, const HubArgs& h, uint32_t hub, uint32_t e) {
  atomicOr(&h.hub_err[hub], e);
  atomicOr(a.err, e);
}

// Key words a hub bucket holds at most: the sizes options.hub_bucket_keys
// accepts; the first is the size before tuning, and the tuning compares the
// first two (8192 measured slower on every workload here once bucket growth
// had settled, while its first pass, with fewer overflows, times faster).
constexpr int kHubUcaps[3] = {4096, 2048, 8192};
constexpr int kHubSmemBuckets = 1024;  // per-chunk bucket counts in shared memory up to this many buckets
constexpr int kHubSample = 128;        // keys sampled per hub to choose its chunk pass
constexpr int kHubSamplePairs = 16;    // equal sampled pairs from which a hub keeps the chunk set
constexpr uint32_t kHubScatterShiftMax = 2;  // bucket growth of a scattering hub before it takes the set

template <typename K>
__host__ __device__ constexpr size_t hub_chunk_smem() {
  return sizeof(ChunkSmem<K, kChunkThreads, kChunkMinHub>) + (size_t)kHubChunk * sizeof(K) + 2 * kHubSmemBuckets * sizeof(uint32_t);
}


template <typename K>
__device__ __forceinline__ uint32_t hub_bucket(K k, uint32_t bits) {
  return bits ? (uint32_t)(k >> (KeyOps<K>::kBits - bits)) : 0u;
}

template <typename LabelT, typename K>
__global__ void __launch_bounds__(kChunkThreads) k_hub_chunk(SigArgs a, HubArgs h) {
  extern __shared__ __align__(16) char smem_raw[];
  ChunkSmem<K, kChunkThreads, kChunkMinHub>& sm = *reinterpret_cast<ChunkSmem<K, kChunkThreads, kChunkMinHub>*>(smem_raw);
  K* list = reinterpret_cast<K*>(smem_raw + sizeof(ChunkSmem<K, kChunkThreads, kChunkMinHub>));
  uint32_t* bcnt = reinterpret_cast<uint32_t*>(list + kHubChunk);
  uint32_t* bpos = bcnt + kHubSmemBuckets;
  const uint4 c = h.chunks[blockIdx.x];
  const uint32_t hub = c.x;
  if (h.mode[hub]) return;  // this hub's chunks run k_hub_scatter
  if (!in_mask(a, h.first + hub)) return;
  const uint64_t ebase = ((uint64_t)c.z << 32) | c.y;
  const uint32_t E = c.w;
  const uint32_t bits = h.hub_bits[hub];
  const uint32_t nb = 1u << bits;
  const bool in_smem = nb <= (uint32_t)kHubSmemBuckets;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  chunk_clear(sm, (2 * E + 3) & ~3u);
  if (in_smem)
    for (uint32_t i = tid; i < nb; i += kChunkThreads) bcnt[i] = 0;
  __syncthreads();
  K key[kChunkItems];
  chunk_keys<kChunkThreads, LabelT, K>(a, ebase, E, key);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm.slot);
#pragma unroll 1
  for (int t = 0; t < kChunkItems; ++t) {
    const K kt = key[0];
#pragma unroll
    for (int q = 0; q + 1 < kChunkItems; ++q) key[q] = key[q + 1];
    bool fresh = false;
    if (tid + t * kChunkThreads < E)
      fresh = kt == KeyOps<K>::kEmpty ? atomicExch(&sm.empty[0], 1u) == 0u : region_insert(sbase, 0u, 2 * E, kt);
    const unsigned fm = __ballot_sync(kFull, fresh);
    if (fm == 0u) continue;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&sm.cnt[0], (uint32_t)__popc(fm));
    base = __shfl_sync(kFull, base, 0);
    if (fresh) list[base + __popc(fm & lanes_below(lane))] = kt;
  }
  __syncthreads();
  const uint32_t U = sm.cnt[0];
  const uint32_t cap = h.hub_cap[hub];
  uint32_t* cur = h.cursor + h.hub_bbase[hub];
  K* tmp = static_cast<K*>(h.tmp) + h.hub_tbase[hub];
  if (in_smem) {
    for (uint32_t i = tid; i < U; i += kChunkThreads) atomicAdd(&bcnt[hub_bucket(list[i], bits)], 1u);
    __syncthreads();
    for (uint32_t b = tid; b < nb; b += kChunkThreads) {
      const uint32_t n_b = bcnt[b];
      bpos[b] = n_b ? atomicAdd(&cur[b], n_b) : 0u;
      bcnt[b] = 0;
    }
    __syncthreads();
  }
  for (uint32_t i = tid; i < U; i += kChunkThreads) {
    const K v = list[i];
    const uint32_t b = hub_bucket(v, bits);
    const uint32_t q = in_smem ? bpos[b] + atomicAdd(&bcnt[b], 1u) : atomicAdd(&cur[b], 1u);
    if (q < cap) tmp[(uint64_t)b * cap + q] = v;
    else hub_fail(a, h, hub, kErrHubOverflow);
  }
}

// Hub pieces without the chunk-level set, for hubs whose keys rarely repeat
// (k_hub_sample): the keys of a chunk go straight to the hub's buckets
// (ranked per bucket in shared memory, one global reservation per bucket,
// then ordered by bucket in shared memory so that each bucket's keys are
// stored as one run), and the bucket pass removes every duplicate.

// One warp per hub: kHubSample keys at an even stride over the hub's edges.
// Among S samples from U equally frequent distinct keys about S(S-1)/2 / U
// pairs are equal: kHubSamplePairs or more equal pairs mean about 500
// distinct keys or fewer (the few blocks of an early level), or a key that
// makes up some 5% of the hub's edges or more, and the hub keeps the chunk
// set, which sends each distinct key of a chunk to the buckets once.  Other
// hubs skip it, unless an earlier overflow forced the set on them.
template <typename LabelT, typename K>
__global__ void __launch_bounds__(256) k_hub_sample(SigArgs a, HubArgs h, uint64_t n_hub) {
  constexpr int kPer = kHubSample / 32;
  __shared__ K sk[256 / 32][kHubSample];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t hub = (uint64_t)blockIdx.x * (256 / 32) + w;
  if (hub >= n_hub) return;
  const uint64_t p = h.first + hub;
  const uint64_t e0 = a.off[p], D = a.off[p + 1] - e0;
  const uint32_t st = (uint32_t)(D / kHubSample);  // >= 1: hubs have more than 4096 edges
  const Policies pol;
  K key[kPer];
  edge_keys<kPer, 0, kPer, LabelT, K>(a, e0 + (uint64_t)lane * st, 32u * st, e0 + D, pol, key);
#pragma unroll
  for (int t = 0; t < kPer; ++t) sk[w][lane + 32 * t] = key[t];
  __syncwarp();
  uint32_t pairs = 0;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const uint32_t i = lane + 32 * t;
    for (uint32_t j = i + 1; j < (uint32_t)kHubSample; ++j) pairs += sk[w][j] == key[t] ? 1u : 0u;
  }
  pairs = __reduce_add_sync(kFull, pairs);
  if (lane == 0) h.mode[hub] = (!h.force[hub] && pairs < (uint32_t)kHubSamplePairs) ? 1 : 0;
}
// Exclusive prefix sums of v[0..n) in place (n <= 2 * NT), by the whole CTA;
// wsum holds NT / 32 words.  Ends with a barrier.
template <int NT>
__device__ __forceinline__ void cta_exclusive_scan(uint32_t* v, uint32_t n, uint32_t* wsum) {
  static_assert(NT % 32 == 0 && NT / 32 <= 32, "one warp scans the warp totals");
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t a = 2 * tid < n ? v[2 * tid] : 0u, b = 2 * tid + 1 < n ? v[2 * tid + 1] : 0u;
  uint32_t x = a + b;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (uint32_t)(NT / 32) ? wsum[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, t, d);
      if (lane >= (uint32_t)d) t += y;
    }
    if (lane < (uint32_t)(NT / 32)) wsum[lane] = t;
  }
  __syncthreads();
  const uint32_t before = (w ? wsum[w - 1] : 0u) + x - (a + b);
  if (2 * tid < n) v[2 * tid] = before;
  if (2 * tid + 1 < n) v[2 * tid + 1] = before + a;
  __syncthreads();
}

template <typename LabelT, typename K>
__global__ void __launch_bounds__(kChunkThreads) k_hub_scatter(SigArgs a, HubArgs h) {
  __shared__ uint32_t bcnt[kHubSmemBuckets];
  __shared__ uint32_t bpos[kHubSmemBuckets];
  __shared__ uint32_t lstart[kHubSmemBuckets];
  __shared__ uint32_t wsum[kChunkThreads / 32];
  __shared__ K stage[kHubChunk];
  const uint4 c = h.chunks[blockIdx.x];
  const uint32_t hub = c.x;
  if (!h.mode[hub]) return;  // this hub's chunks run k_hub_chunk
  if (!in_mask(a, h.first + hub)) return;
  const uint64_t ebase = ((uint64_t)c.z << 32) | c.y;
  const uint32_t E = c.w;
  const uint32_t bits = h.hub_bits[hub];
  const uint32_t nb = 1u << bits;
  const bool in_smem = nb <= (uint32_t)kHubSmemBuckets;
  const uint32_t tid = threadIdx.x;
  if (in_smem)
    for (uint32_t i = tid; i < nb; i += kChunkThreads) bcnt[i] = 0;
  __syncthreads();
  K key[kChunkItems];
  chunk_keys<kChunkThreads, LabelT, K>(a, ebase, E, key);
  const uint32_t cap = h.hub_cap[hub];
  uint32_t* cur = h.cursor + h.hub_bbase[hub];
  K* tmp = static_cast<K*>(h.tmp) + h.hub_tbase[hub];
  // rank of each key within its bucket in this chunk (shared counts), then one
  // global reservation per bucket
  uint32_t rank[kChunkItems];
#pragma unroll
  for (int t = 0; t < kChunkItems; ++t) {
    rank[t] = 0;
    if (tid + t * kChunkThreads < E) {
      const uint32_t b = hub_bucket(key[t], bits);
      rank[t] = in_smem ? atomicAdd(&bcnt[b], 1u) : atomicAdd(&cur[b], 1u);
    }
  }
  if (!in_smem) {
#pragma unroll
    for (int t = 0; t < kChunkItems; ++t) {
      if (tid + t * kChunkThreads >= E) continue;
      const uint32_t b = hub_bucket(key[t], bits);
      if (rank[t] < cap) tmp[(uint64_t)b * cap + rank[t]] = key[t];
      else hub_fail(a, h, hub, kErrHubOverflow);
    }
    return;
  }
  __syncthreads();
  for (uint32_t b = tid; b < nb; b += kChunkThreads) {
    const uint32_t n_b = bcnt[b];
    bpos[b] = n_b ? atomicAdd(&cur[b], n_b) : 0u;
    lstart[b] = n_b;
  }
  __syncthreads();
  // the chunk's keys ordered by bucket in shared memory, so that each
  // bucket's keys leave as one run of consecutive words
  cta_exclusive_scan<kChunkThreads>(lstart, nb, wsum);
#pragma unroll
  for (int t = 0; t < kChunkItems; ++t)
    if (tid + t * kChunkThreads < E) stage[lstart[hub_bucket(key[t], bits)] + rank[t]] = key[t];
  __syncthreads();
  for (uint32_t i = tid; i < E; i += kChunkThreads) {
    const K k = stage[i];
    const uint32_t b = hub_bucket(k, bits);
    const uint32_t q = bpos[b] + (i - lstart[b]);
    if (q < cap) tmp[(uint64_t)b * cap + q] = k;
    else hub_fail(a, h, hub, kErrHubOverflow);
  }
}

// Insert k (!= kEmpty) into a power-of-two set of hmask + 1 slots at
// shared-window address `base`, home slot from the key's low bits (the keys of
// one hub bucket share their top bits).  The compare-and-swap is the probe
// itself: one shared access per probed slot, whether the slot is empty, holds
// k or holds another key.  Returns 1 if this call inserted k, 0 if k was
// present, -1 if the set is full.
template <typename K>
__device__ __forceinline__ int pow2_insert(uint32_t base, uint32_t hmask, K k) {
  uint32_t s = key_h32(k) & hmask;
  for (uint32_t t = 0; t <= hmask; ++t) {
    const K cur = atoms_cas(base + s * (uint32_t)sizeof(K), KeyOps<K>::kEmpty, k);
    if (cur == KeyOps<K>::kEmpty) return 1;
    if (cur == k) return 0;
    s = (s + 1) & hmask;
  }
  return -1;
}

constexpr int kBucketThreads = 256, kBucketItems = 8;

template <typename K, int UCAP>
struct BucketSmem {
  K set[2 * UCAP];
  uint32_t empty, full, lo, hi;
};

// One CTA per hub bucket (grid-stride): distinct keys of the bucket into a
// shared set; a warp appends the keys it finds fresh straight after the
// hub's keys written so far (one reservation per warp step on the hub's
// counter) and adds their term sums to the bucket's, which go to the hub's
// at the end.  If the set fills, the host repeats the hub with more buckets
// (its counter restarts from zero, so the keys written are written again).
template <typename K, int UCAP>
__global__ void __launch_bounds__(kBucketThreads, sizeof(K) == 4 ? 6 : 3) k_hub_bucket(SigArgs a, HubArgs h, uint64_t n_buckets) {
  extern __shared__ __align__(16) char smem_raw[];
  BucketSmem<K, UCAP>& sm = *reinterpret_cast<BucketSmem<K, UCAP>*>(smem_raw);
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm.set);
  K* out = static_cast<K*>(a.sigkey);
  // a bucket's hub, key count and first kBucketThreads * kBucketItems keys are
  // loaded one bucket ahead, so that their latency overlaps the work on the
  // bucket before
  uint32_t nx_hub = 0, nx_n = 0;
  const K* nx_tmp = nullptr;
  K kk[kBucketItems];
  auto fetch = [&](uint64_t bb) {
    nx_hub = h.bucket_hub[bb];
    const uint32_t cap = h.hub_cap[nx_hub];
    nx_tmp = static_cast<const K*>(h.tmp) + h.hub_tbase[nx_hub] + (bb - h.hub_bbase[nx_hub]) * cap;
    nx_n = min(h.cursor[bb], cap);
#pragma unroll
    for (int t = 0; t < kBucketItems; ++t) {
      const uint32_t i = tid + t * kBucketThreads;
      kk[t] = i < nx_n ? nx_tmp[i] : (K)0;
    }
  };
  if (blockIdx.x < n_buckets) fetch(blockIdx.x);
  for (uint64_t b = blockIdx.x; b < n_buckets; b += gridDim.x) {
    const uint32_t hub = nx_hub, n = nx_n;
    const uint64_t p = h.first + hub;
    const K* tmp = nx_tmp;
    if (n == 0) {  // nothing appended (a hub outside a frontier mask): no barrier, no output
      if (b + gridDim.x < n_buckets) fetch(b + gridDim.x);
      continue;
    }
    uint32_t hcap = 64;
    while (hcap < 2 * n && hcap < 2 * UCAP) hcap <<= 1;
    {
      uint4* s4 = reinterpret_cast<uint4*>(sm.set);
      const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
      for (uint32_t i = tid; i < hcap * sizeof(K) / 16; i += kBucketThreads) s4[i] = ones;
    }
    if (tid == 0) {
      sm.empty = 0;
      sm.full = 0;
      sm.lo = 0;
      sm.hi = 0;
    }
    __syncthreads();
    K* hout = out + a.off[p];
    unsigned long long* hcur = &h.hub_cur[hub];
    for (uint32_t i0 = 0; i0 < n; i0 += kBucketThreads * kBucketItems) {
      if (i0) {
#pragma unroll
        for (int t = 0; t < kBucketItems; ++t) {
          const uint32_t i = i0 + tid + t * kBucketThreads;
          kk[t] = i < n ? tmp[i] : (K)0;
        }
      }
      // the keys of kBucketItems steps are inserted first; then the warp
      // takes the places of all its fresh keys with one reservation on the
      // hub's counter (its latency paid once, not per step) and adds their
      // term sums once
      unsigned fms[kBucketItems];
      uint32_t lo = 0, hi = 0, total = 0;
#pragma unroll
      for (int t = 0; t < kBucketItems; ++t) {
        fms[t] = 0u;
        if (i0 + (uint32_t)t * kBucketThreads >= n) continue;  // the same for the whole CTA
        const uint32_t i = i0 + tid + t * kBucketThreads;
        const K k = kk[t];
        bool fresh = false;
        if (i < n) {
          if (k == KeyOps<K>::kEmpty) {
            fresh = atomicExch(&sm.empty, 1u) == 0u;
          } else {
            const int r = pow2_insert(sbase, hcap - 1, k);
            fresh = r > 0;
            if (r < 0) sm.full = 1u;
          }
        }
        fms[t] = __ballot_sync(kFull, fresh);
        total += __popc(fms[t]);
        if (fresh) {
          const uint64_t tm = elem_term(k, a.seed);
          lo += (uint32_t)tm;
          hi += (uint32_t)(tm >> 32);
        }
      }
      if (total) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(hcur, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 0);
#pragma unroll
        for (int t = 0; t < kBucketItems; ++t) {
          if ((fms[t] >> lane) & 1u) hout[base + __popc(fms[t] & lanes_below(lane))] = kk[t];
          base += __popc(fms[t]);
        }
        lo = __reduce_add_sync(kFull, lo);
        hi = __reduce_add_sync(kFull, hi);
        if (lane == 0) {
          atomicAdd(&sm.lo, lo);
          atomicAdd(&sm.hi, hi);
        }
      }
    }
    if (b + gridDim.x < n_buckets) fetch(b + gridDim.x);
    __syncthreads();
    if (tid == 0) {
      if (sm.full) hub_fail(a, h, hub, kErrHubSet);  // more distinct keys than the set holds: the host adds buckets
      atomicAdd(&h.hub_term[2 * hub], sm.lo);      // (a failed hub's sums are cleared before its repeat)
      atomicAdd(&h.hub_term[2 * hub + 1], sm.hi);
    }
    // no barrier here: thread 0 alone reads the bucket's totals, and the next
    // bucket's first barrier comes before anything is written to them again
  }
}

// Count and hash of every hub (of the mask) from its buckets' totals.
__global__ void k_hub_finish(SigArgs a, HubArgs h, uint64_t n_hub) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_hub;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = h.first + i;
    if (!in_mask(a, p)) continue;
    const unsigned long long tot = h.hub_cur[i];
    const uint64_t tsum = ((uint64_t)h.hub_term[2 * i + 1] << 32) | h.hub_term[2 * i];
    a.ucnt[p] = (uint32_t)tot;
    a.hash[p] = node_hash(tsum, a.prev[p], tot, a.seed, a.mask);
  }
}

// --------------------------------------------------------------------------
// Grouping: equal hashes -> smallest original id; exact verification
// --------------------------------------------------------------------------
// Table slots are 64-bit words (hash fingerprint << 32 | smallest original
// id), empty = all ones.  A slot is claimed by CAS and then lowered with
// atomicMin; different hashes that meet in one slot with the same
// fingerprint are merged here and separated again by exact verification.
struct GroupArgs {
  const uint64_t* hash;
  const uint32_t* p2o;
  const uint32_t* o2p;
  unsigned long long* table;
  uint64_t tmask;   // table capacity - 1
  uint32_t* slot;
  uint32_t* rep;
  uint32_t* err;
  const uint8_t* alone;  // nodes alone in their previous block (may be null): heads, not grouped
  int read_first;        // few distinct hashes shared by many nodes (level 0): read a slot before any atomic
};

__device__ __forceinline__ uint32_t table_insert(const GroupArgs& g, uint64_t h, uint32_t minid) {
  const unsigned long long fp = (unsigned long long)(uint32_t)(h >> 32);
  const unsigned long long v = (fp << 32) | minid;
  uint32_t s = (uint32_t)(mix64(h) & g.tmask);
  for (uint64_t t = 0; t <= g.tmask; ++t) {
    // a slot already holding this fingerprint with an id no larger needs no atomic
    if (g.read_first) {
      const unsigned long long seen = *(volatile unsigned long long*)&g.table[s];
      if ((seen >> 32) == fp && seen != kEmpty64 && (uint32_t)seen <= minid) return s;
    }
    const unsigned long long cur = atomicCAS(&g.table[s], (unsigned long long)kEmpty64, v);
    if (cur == kEmpty64) return s;
    if ((cur >> 32) == fp) {
      if ((uint32_t)cur > minid) atomicMin(&g.table[s], v);
      return s;
    }
    s = (uint32_t)((s + 1) & g.tmask);
  }
  atomicOr(g.err, kErrProbe);
  return 0;
}

// A CTA takes 1024 nodes, combines equal hashes in shared memory (smallest
// original id per hash), then inserts each distinct hash once.
constexpr int kInsThreads = 256, kInsItems = 4, kInsChunk = kInsThreads * kInsItems, kInsSlots = 2 * kInsChunk;

__global__ void __launch_bounds__(kInsThreads) k_group_insert(GroupArgs g, const uint32_t* list, uint64_t count) {
  __shared__ unsigned long long skey[kInsSlots];
  __shared__ unsigned int smin[kInsSlots];
  __shared__ unsigned int sglob[kInsSlots];
  __shared__ unsigned short used[kInsChunk];  // slots taken in this chunk (one per distinct hash)
  __shared__ unsigned int n_used;
  const uint32_t lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kInsSlots; i += kInsThreads) {
    skey[i] = kEmpty64;
    smin[i] = kNone32;
  }
  if (threadIdx.x == 0) n_used = 0;
  __syncthreads();
  for (uint64_t base = (uint64_t)blockIdx.x * kInsChunk; base < count; base += (uint64_t)gridDim.x * kInsChunk) {
    // loads of all items first (node ids, then alone flags, then hashes and
    // original ids of the nodes that are grouped), so that they overlap
    uint32_t ls[kInsItems], pp[kInsItems], oo[kInsItems];
    uint64_t hh[kInsItems];
#pragma unroll
    for (int t = 0; t < kInsItems; ++t) {
      const uint64_t i = base + threadIdx.x + (uint64_t)t * kInsThreads;
      pp[t] = i < count ? (list ? list[i] : (uint32_t)i) : kNone32;
    }
#pragma unroll
    for (int t = 0; t < kInsItems; ++t)
      ls[t] = (pp[t] != kNone32 && !(g.alone && g.alone[pp[t]])) ? 0u : kNone32;
#pragma unroll
    for (int t = 0; t < kInsItems; ++t) {
      if (ls[t] != kNone32) {
        hh[t] = g.hash[pp[t]];
        oo[t] = g.p2o[pp[t]];
      }
    }
#pragma unroll
    for (int t = 0; t < kInsItems; ++t) {
      bool took = false;
      if (ls[t] != kNone32) {
        const uint64_t h = hh[t];
        uint32_t s = (uint32_t)(mix64(h) & (kInsSlots - 1));
        for (int q = 0; q < kInsSlots; ++q) {  // at most kInsChunk distinct hashes: always room
          const unsigned long long cur = atomicCAS(&skey[s], (unsigned long long)kEmpty64, (unsigned long long)h);
          if (cur == kEmpty64) { took = true; break; }
          if (cur == h) break;
          s = (s + 1) & (kInsSlots - 1);
        }
        atomicMin(&smin[s], oo[t]);
        ls[t] = s;
      }
      const unsigned tm = __ballot_sync(kFull, took);
      if (tm) {
        uint32_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&n_used, (unsigned)__popc(tm));
        b0 = __shfl_sync(kFull, b0, 0);
        if (took) used[b0 + __popc(tm & lanes_below(lane))] = (unsigned short)ls[t];
      }
    }
    __syncthreads();
    const uint32_t nu = n_used;
    for (uint32_t i = threadIdx.x; i < nu; i += kInsThreads) {
      const uint32_t sl = used[i];
      sglob[sl] = table_insert(g, skey[sl], smin[sl]);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kInsItems; ++t)
      if (ls[t] != kNone32) g.slot[pp[t]] = sglob[ls[t]];
    __syncthreads();
    // only the slots this chunk took are cleared for the next one
    for (uint32_t i = threadIdx.x; i < nu; i += kInsThreads) {
      const uint32_t sl = used[i];
      skey[sl] = kEmpty64;
      smin[sl] = kNone32;
    }
    if (threadIdx.x == 0) n_used = 0;
    __syncthreads();
  }
}

struct VerifyArgs {
  int mode;                 // 0: level 0 (labels), 1: signatures
  int key64;                // signature words are 64-bit
  const uint32_t* nlabel;
  const uint32_t* prev;
  const uint32_t* ucnt;
  const uint64_t* off;
  const void* sigkey;
  uint32_t* out_list;       // unresolved nodes
  unsigned long long* n_out;
  unsigned long long* n_collided;
  uint32_t* long_list;      // (node, candidate) pairs with long signatures
  unsigned long long* n_long;
  uint32_t* hbits;          // head bitmap over original ids (canonical numbering)
  uint8_t* member;          // per internal id: this head has other members
};

constexpr uint32_t kShortSig = 8;

// Set equality of two duplicate-free key lists of the same length n <= kShortSig.
template <typename K>
__device__ __forceinline__ bool same_set_short(const K* a, const K* b, uint32_t n) {
  K bk[kShortSig];
#pragma unroll
  for (uint32_t j = 0; j < kShortSig; ++j) bk[j] = j < n ? b[j] : (K)0;
  for (uint32_t i = 0; i < n; ++i) {
    const K x = a[i];
    bool found = false;
#pragma unroll
    for (uint32_t j = 0; j < kShortSig; ++j) found |= (j < n && bk[j] == x);
    if (!found) return false;
  }
  return true;
}

// Marks for the canonical numbering, set where a node's representative is
// settled: a head sets the bit of its original id; a member sets its head's
// member flag (read first: in a large block most members find it set).
__device__ __forceinline__ void mark_head(const VerifyArgs& v, uint32_t o) {
  atomicOr(&v.hbits[o >> 5], 1u << (o & 31));
}
__device__ __forceinline__ void mark_member(const VerifyArgs& v, uint32_t r) {
  if (!*(volatile uint8_t*)&v.member[r]) v.member[r] = 1;
}

constexpr int kMarkSeen = 256;  // heads a verification CTA remembers as marked

__device__ __forceinline__ void mark_unresolved(const VerifyArgs& v, uint32_t* rep, uint32_t p) {
  rep[p] = kNone32;
  const unsigned long long q = atomicAdd(v.n_out, 1ull);
  v.out_list[q] = p;
  atomicAdd(v.n_collided, 1ull);
}

// Each thread takes kVerItems nodes of a tile at a time, and every step's
// loads for all of them are issued together (node ids; alone flags; original
// ids and table slots; representatives; their fields; the short key lists).
constexpr int kVerNodeThreads = 256, kVerItems = 2, kVerTile = kVerNodeThreads * kVerItems;

__global__ void __launch_bounds__(kVerNodeThreads) k_group_verify(GroupArgs g, VerifyArgs v, const uint32_t* list,
                                                                   uint64_t count) {
  // heads this CTA has marked as having members: a block of millions of
  // nodes (level 0) then costs one global access per CTA, not per member
  __shared__ uint32_t seen[kMarkSeen];
  for (int i = threadIdx.x; i < kMarkSeen; i += kVerNodeThreads) seen[i] = kNone32;
  __syncthreads();
  for (uint64_t base = (uint64_t)blockIdx.x * kVerTile; base < count; base += (uint64_t)gridDim.x * kVerTile) {
    uint32_t p[kVerItems], o[kVerItems], x[kVerItems], r[kVerItems], U[kVerItems];
    bool act[kVerItems], eq[kVerItems];
#pragma unroll
    for (int t = 0; t < kVerItems; ++t) {
      const uint64_t i = base + threadIdx.x + (uint64_t)t * kVerNodeThreads;
      p[t] = i < count ? (list ? list[i] : (uint32_t)i) : kNone32;
    }
#pragma unroll
    for (int t = 0; t < kVerItems; ++t) act[t] = p[t] != kNone32 && !(g.alone && g.alone[p[t]]);
#pragma unroll
    for (int t = 0; t < kVerItems; ++t) {
      if (p[t] != kNone32) o[t] = g.p2o[p[t]];
      if (act[t]) x[t] = g.slot[p[t]];
    }
#pragma unroll
    for (int t = 0; t < kVerItems; ++t)
      if (act[t]) x[t] = (uint32_t)g.table[x[t]];  // smallest original id of the node's hash
    // heads: alone in the previous block, or the smallest id of their hash
#pragma unroll
    for (int t = 0; t < kVerItems; ++t) {
      if (p[t] != kNone32 && (!act[t] || x[t] == o[t])) {
        g.rep[p[t]] = p[t];
        mark_head(v, o[t]);
        act[t] = false;
      }
    }
#pragma unroll
    for (int t = 0; t < kVerItems; ++t)
      if (act[t]) r[t] = g.o2p[x[t]];
    if (v.mode == 0) {
#pragma unroll
      for (int t = 0; t < kVerItems; ++t)
        if (act[t]) eq[t] = v.nlabel[p[t]] == v.nlabel[r[t]];
    } else {
#pragma unroll
      for (int t = 0; t < kVerItems; ++t) {
        if (act[t]) {
          U[t] = v.ucnt[p[t]];
          eq[t] = v.prev[p[t]] == v.prev[r[t]] && U[t] == v.ucnt[r[t]];
        }
      }
#pragma unroll
      for (int t = 0; t < kVerItems; ++t) {
        if (act[t] && eq[t] && U[t] > kShortSig) {  // long signature: compared by a CTA later
          const unsigned long long q = atomicAdd(v.n_long, 1ull);
          v.long_list[2 * q] = p[t];
          v.long_list[2 * q + 1] = r[t];
          act[t] = false;
        }
      }
#pragma unroll
      for (int t = 0; t < kVerItems; ++t) {
        if (act[t] && eq[t]) {
          eq[t] = v.key64 ? same_set_short(static_cast<const uint64_t*>(v.sigkey) + v.off[p[t]],
                                           static_cast<const uint64_t*>(v.sigkey) + v.off[r[t]], U[t])
                          : same_set_short(static_cast<const uint32_t*>(v.sigkey) + v.off[p[t]],
                                           static_cast<const uint32_t*>(v.sigkey) + v.off[r[t]], U[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kVerItems; ++t) {
      if (!act[t]) continue;
      if (eq[t]) {
        g.rep[p[t]] = r[t];
        if (atomicCAS(&seen[r[t] % kMarkSeen], kNone32, r[t]) != r[t]) mark_member(v, r[t]);
      } else {
        mark_unresolved(v, g.rep, p[t]);
      }
    }
  }
}

// One CTA per (node, candidate) pair with a long signature: the candidate's
// keys go into a shared-memory set, chunk by chunk, and the node's keys are
// looked up; the sets are equal iff every one of the node's keys is found
// (both lists are duplicate-free and of equal length).
constexpr int kVerThreads = 256, kVerChunk = 4096;

template <typename K>
__host__ __device__ constexpr size_t verify_ws_bytes() { return team_set_bytes<K>(2 * kVerChunk, 0, kVerThreads); }

template <typename K>
__global__ void __launch_bounds__(kVerThreads) k_verify_long(GroupArgs g, VerifyArgs v, uint64_t count) {
  extern __shared__ __align__(16) char smem[];
  TeamSet<K> ts = carve_set<K>(smem, 2 * kVerChunk, 0);
  const K* keys = static_cast<const K*>(v.sigkey);
  for (uint64_t q = blockIdx.x; q < count; q += gridDim.x) {
    const uint32_t p = v.long_list[2 * q], r = v.long_list[2 * q + 1];
    const uint32_t U = v.ucnt[p];
    const K* ka = keys + v.off[p];
    const K* kb = keys + v.off[r];
    uint32_t found = 0;
    for (uint32_t c0 = 0; c0 < U; c0 += kVerChunk) {
      const uint32_t cn = min((uint32_t)kVerChunk, U - c0);
      const int hcap = set_size_for(cn, 2 * kVerChunk);
      set_clear<kVerThreads>(ts, hcap, threadIdx.x);
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < cn; i += kVerThreads) set_insert(ts, hcap, kb[c0 + i]);
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < U; i += kVerThreads) found += set_find(ts, hcap, ka[i]) ? 1 : 0;
      __syncthreads();
    }
    found = team_sum<kVerThreads>(found, ts.red, threadIdx.x);
    if (threadIdx.x == 0) {
      if (found == U) {
        g.rep[p] = r;
        mark_member(v, r);
      } else {
        mark_unresolved(v, g.rep, p);
      }
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Canonical renumbering: heads are nodes with rep[p] == p (the node with the
// smallest original id in its block); a block's id is the number of heads
// with a smaller original id.  Heads are marked in a bitmap over original ids
// (n/8 bytes, cache resident); an exclusive scan of the per-word head counts
// then gives each head its rank with one more popcount.
// --------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

struct RankArgs {
  uint64_t n, n_alive;
  const uint32_t* rep;
  const uint32_t* p2o;
  const uint32_t* ucnt;    // may be null (level 0)
  uint32_t* hbits;         // [words] head bitmap, original order
  uint64_t* hword;         // [words] head count per word, then heads before the word
  uint8_t* member;         // [n] internal order: the head has other members
  uint8_t* alone;          // [n] internal order: output, node alone in its block
  uint32_t* pid;           // output level, internal order
  unsigned long long* stats;  // [2] key total, [3] max signature, [8] nodes alone in their block
};

__global__ void k_word_counts(const uint32_t* hbits, uint64_t words, uint64_t* hword) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x)
    hword[w] = __popc(hbits[w]);
}

// Exclusive scan of bsum[0..nb) in one CTA; total into *total.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint64_t* bsum, uint64_t nb,
                                                              unsigned long long* total) {
  __shared__ unsigned long long wt[kScanThreads / 32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nb; base += kScanThreads) {
    const uint64_t i = base + threadIdx.x;
    const unsigned long long v = i < nb ? bsum[i] : 0ull;
    unsigned long long x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long t = wt[lane];
      unsigned long long xx = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, xx, o);
        if (lane >= o) xx += y;
      }
      wt[lane] = xx - t;
    }
    __syncthreads();
    const unsigned long long c0 = carry;
    if (i < nb) bsum[i] = c0 + wt[w] + x - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c0 + wt[w] + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Every alive node takes its head's block id; deleted nodes get kDead.  A
// thread takes kFillItems nodes at a time and issues each step's loads for
// all of them together (representatives; their original ids; the bitmap
// words), so the three dependent gathers of a node overlap with the others'.
constexpr int kFillItems = 4;

__global__ void k_pid_fill(RankArgs r) {
  unsigned int n_alone = 0, mx = 0;
  unsigned long long keys = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p0 < r.n; p0 += stride * kFillItems) {
    uint32_t h[kFillItems], o[kFillItems], hb[kFillItems];
    uint64_t hw[kFillItems];
    bool live[kFillItems];
#pragma unroll
    for (int t = 0; t < kFillItems; ++t) {
      const uint64_t p = p0 + (uint64_t)t * stride;
      live[t] = p < r.n_alive;
      if (live[t]) h[t] = r.rep[p];
    }
#pragma unroll
    for (int t = 0; t < kFillItems; ++t)
      if (live[t]) o[t] = r.p2o[h[t]];
#pragma unroll
    for (int t = 0; t < kFillItems; ++t) {
      if (live[t]) {
        hw[t] = r.hword[o[t] >> 5];
        hb[t] = r.hbits[o[t] >> 5];
      }
    }
#pragma unroll
    for (int t = 0; t < kFillItems; ++t) {
      const uint64_t p = p0 + (uint64_t)t * stride;
      if (p >= r.n) break;
      if (live[t]) {
        if (r.ucnt) {
          const uint32_t q = r.ucnt[p];
          keys += q;
          mx = max(mx, q);
        }
        r.pid[p] = (uint32_t)hw[t] + (uint32_t)__popc(hb[t] & ((1u << (o[t] & 31)) - 1u));
        const bool al = h[t] == (uint32_t)p && !r.member[p];
        r.alone[p] = al ? 1 : 0;
        n_alone += al ? 1u : 0u;
      } else {
        r.pid[p] = kDead;
      }
    }
  }
  n_alone = __reduce_add_sync(kFull, n_alone);
  if ((threadIdx.x & 31) == 0 && n_alone) atomicAdd(&r.stats[8], (unsigned long long)n_alone);
  if (r.ucnt) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      keys += __shfl_xor_sync(kFull, keys, o);
      mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&r.stats[2], keys);
      atomicMax(&r.stats[3], (unsigned long long)mx);
    }
  }
}

// Nodes outside the round's mask keep their block: signature (pId_{i-1}(u), {})
// -- a node of a graph that has stopped (batched build) then stays with the
// nodes it was grouped with at the level before.
__global__ void k_freeze(uint64_t n_alive, const uint32_t* mask, const uint32_t* prev, uint32_t* ucnt,
                         uint64_t* hash, uint64_t seed, uint64_t hmask) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n_alive; p += (uint64_t)gridDim.x * blockDim.x) {
    if ((mask[p >> 5] >> (p & 31)) & 1u) continue;
    ucnt[p] = 0;
    hash[p] = node_hash(0, prev[p], 0, seed, hmask);
  }
}

// Checked mode: every a[i] (i < n) must be below `bound`.  The kernels that
// index with an array run only after this check has passed on it.
__global__ void k_check_below(const uint32_t* a, uint64_t n, uint64_t bound, uint32_t* err) {
  bool bad = false;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    bad |= (uint64_t)a[i] >= bound;
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrChecked);
}

// Checked mode: offsets non-decreasing from 0 to m.
__global__ void k_check_offsets_mono(const uint64_t* off, uint64_t n, uint64_t m, uint32_t* err) {
  bool bad = false;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x)
    bad |= off[p] > off[p + 1] || off[p + 1] > m || (p == 0 && off[0] != 0);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrChecked);
}

// Level 0 hash: the node label.
__global__ void k_label_hash(uint64_t n, const uint32_t* nlabel, uint64_t* hash, uint64_t seed, uint64_t mask) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x)
    hash[p] = node_hash(0, nlabel[p], 0, seed, mask);
}

__global__ void k_unpermute(uint64_t n, const uint32_t* o2p, const uint32_t* lvl, uint32_t* out) {
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n;
       o += (uint64_t)gridDim.x * blockDim.x)
    out[o] = lvl[o2p[o]];
}

// --------------------------------------------------------------------------
// Relabelling (once per graph)
// --------------------------------------------------------------------------
__device__ __forceinline__ int degree_class(uint64_t d) { return degree_class_of(d); }

constexpr int kClassTile = 1024;

__device__ __forceinline__ int node_class(uint64_t o, uint64_t n, const uint64_t* off, const uint8_t* alive) {
  if (o >= n) return -1;
  if (alive && !alive[o]) return kClassDead;
  return degree_class(off[o + 1] - off[o]);
}

// Within a degree class, nodes are ordered by popularity as a target (hot
// first), so the identifiers that most edges gather sit in a few dense cache
// lines.  Popularity is the in-degree counted on every 2^kHotSampleShift-th
// edge, put into kHotBuckets buckets; it affects speed only, never results.
constexpr int kHotBuckets = 8;
constexpr int kNumOrder = kNumClasses * kHotBuckets;
constexpr int kHotSampleShift = 8;

__device__ __forceinline__ int hot_bucket(uint32_t c) {
  return c >= 1024 ? 0 : c >= 256 ? 1 : c >= 64 ? 2 : c >= 16 ? 3 : c >= 4 ? 4 : c >= 2 ? 5 : c >= 1 ? 6 : 7;
}

__device__ __forceinline__ int order_class(uint64_t o, uint64_t n, const uint64_t* off, const uint8_t* alive,
                                           const uint32_t* hot) {
  const int c = node_class(o, n, off, alive);
  if (c < 0) return -1;
  return c * kHotBuckets + (c == kClassDead ? 0 : hot_bucket(hot[o]));
}

__global__ void k_hot_sample(uint64_t m, const uint32_t* dst0, uint32_t* hot) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; (i << kHotSampleShift) < m; i += stride)
    atomicAdd(&hot[dst0[i << kHotSampleShift]], 1u);
}

__global__ void __launch_bounds__(kClassTile)
    k_class_tile_count(uint64_t n, const uint64_t* off, const uint8_t* alive, const uint32_t* hot, uint64_t ntiles,
                       unsigned long long* tcnt) {
  __shared__ unsigned int c[kNumOrder];
  for (int i = threadIdx.x; i < kNumOrder; i += kClassTile) c[i] = 0;
  __syncthreads();
  const int cls = order_class((uint64_t)blockIdx.x * kClassTile + threadIdx.x, n, off, alive, hot);
  if (cls >= 0) atomicAdd(&c[cls], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kNumOrder; i += kClassTile) tcnt[(uint64_t)i * ntiles + blockIdx.x] = c[i];
}

// Stable scatter: each tile writes its nodes of order class c in id order at
// the (class, tile) base.
__global__ void __launch_bounds__(kClassTile)
    k_class_tile_scatter(uint64_t n, const uint64_t* off, const uint8_t* alive, const uint32_t* hot, uint64_t ntiles,
                         const unsigned long long* tbase, uint32_t* p2o) {
  __shared__ unsigned int wcnt[kClassTile / 32][kNumOrder];
  for (int i = threadIdx.x; i < (kClassTile / 32) * kNumOrder; i += kClassTile) (&wcnt[0][0])[i] = 0;
  const uint64_t o = (uint64_t)blockIdx.x * kClassTile + threadIdx.x;
  const int cls = order_class(o, n, off, alive, hot);
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned same = __match_any_sync(kFull, cls);
  __syncthreads();
  if (cls >= 0 && lane == (unsigned)__ffs(same) - 1u) wcnt[w][cls] = __popc(same);
  __syncthreads();
  if (cls >= 0) {
    unsigned before = __popc(same & ((1u << lane) - 1u));
    for (unsigned i = 0; i < w; ++i) before += wcnt[i][cls];
    p2o[tbase[(uint64_t)cls * ntiles + blockIdx.x] + before] = (uint32_t)o;
  }
}

__global__ void k_order_starts(const unsigned long long* tbase, uint64_t ntiles, unsigned long long* out) {
  for (int i = threadIdx.x; i < kNumOrder; i += blockDim.x) out[i] = tbase[(uint64_t)i * ntiles];
}

__global__ void k_invert(uint64_t n, const uint32_t* p2o, uint32_t* o2p) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x)
    o2p[p2o[p]] = (uint32_t)p;
}

// deg of internal node p into off[p] (then an exclusive scan makes offsets);
// node labels follow their node.
__global__ void k_relabel_nodes(uint64_t n, const uint32_t* p2o, const uint64_t* off0, const uint32_t* nlab0,
                                unsigned long long* deg, uint32_t* nlab) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t o = p2o[p];
    deg[p] = off0[o + 1] - off0[o];
    nlab[p] = nlab0[o];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) deg[n] = 0;
}

// Copy out-edges to the segment of their source's internal id, relabelling
// targets.  Every lane handles kRelItems edges at a time, all their loads in
// flight together (targets and labels, then the identifier gathers).
constexpr int kRelItems = 4;

// Out-degree <= kSmallMax: one warp per 32 consecutive internal nodes, whose
// edges form one contiguous range of the new table.  Lane k copies edges k,
// k + 32, ... of that range; an edge's node is found by a binary search over
// the 32 new offsets the lanes hold, so reads follow each node's edges in
// order and writes fill the range coalesced.
template <typename TI, typename TO>
__global__ void k_relabel_edges_small(uint64_t n_small, const uint32_t* p2o, const uint32_t* o2p,
                                      const uint64_t* off0, const uint32_t* dst0, const TI* lab0, const uint64_t* off,
                                      uint32_t* dst, TO* lab) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < n_small; w += warps) {
    const uint64_t p = w * 32 + lane;
    const uint64_t base = off[w * 32];
    const uint64_t end = off[min(w * 32 + 32, n_small)];
    // lanes past the last node hold the range's end: an empty node there
    const uint32_t r1 = (uint32_t)((p < n_small ? off[p] : end) - base);
    const uint64_t s0 = p < n_small ? off0[p2o[p]] : 0;
    const uint32_t T = (uint32_t)(end - base);  // at most 32 * kSmallMax
    for (uint32_t k0 = 0; k0 < T; k0 += 32 * kRelItems) {
      uint64_t src[kRelItems];
#pragma unroll
      for (int t = 0; t < kRelItems; ++t) {
        const uint32_t k = min(k0 + lane + 32u * t, T - 1);
        uint32_t j = 0;
#pragma unroll
        for (uint32_t step = 16; step; step >>= 1)
          if (__shfl_sync(kFull, r1, j + step) <= k) j += step;
        src[t] = __shfl_sync(kFull, s0, j) + (k - __shfl_sync(kFull, r1, j));
      }
      uint32_t dv[kRelItems];
      TI lv[kRelItems];
#pragma unroll
      for (int t = 0; t < kRelItems; ++t) {
        if (k0 + lane + 32u * t < T) {
          dv[t] = dst0[src[t]];
          lv[t] = lab0[src[t]];
        }
      }
#pragma unroll
      for (int t = 0; t < kRelItems; ++t)
        if (k0 + lane + 32u * t < T) dv[t] = o2p[dv[t]];
#pragma unroll
      for (int t = 0; t < kRelItems; ++t) {
        const uint32_t k = k0 + lane + 32u * t;
        if (k < T) {
          dst[base + k] = dv[t];
          lab[base + k] = (TO)lv[t];
        }
      }
    }
  }
}

// Deleted nodes (their own class, last): one thread per node; those of
// out-degree <= kSmallMax keep their edges in the new table.
template <typename TI, typename TO>
__global__ void k_relabel_edges_dead(uint64_t p_first, uint64_t p_end, const uint32_t* p2o, const uint32_t* o2p,
                                     const uint64_t* off0, const uint32_t* dst0, const TI* lab0, const uint64_t* off,
                                     uint32_t* dst, TO* lab) {
  for (uint64_t p = p_first + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < p_end;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t o = p2o[p];
    const uint64_t s0 = off0[o], d = off0[o + 1] - s0;
    if (d > (uint64_t)kSmallMax) continue;
    const uint64_t s1 = off[p];
    for (uint64_t i = 0; i < d; ++i) {
      dst[s1 + i] = o2p[dst0[s0 + i]];
      lab[s1 + i] = (TO)lab0[s0 + i];
    }
  }
}

// Copy d edges from src to dst_at in the new table, kRelItems per lane at a
// time, `lane` of `lanes` threads.
template <typename TI, typename TO>
__device__ __forceinline__ void relabel_run(uint64_t src, uint64_t at, uint64_t d, uint32_t lane, uint32_t lanes,
                                            const uint32_t* o2p, const uint32_t* dst0, const TI* lab0, uint32_t* dst,
                                            TO* lab) {
  for (uint64_t i0 = 0; i0 < d; i0 += (uint64_t)lanes * kRelItems) {
    uint32_t dv[kRelItems];
    TI lv[kRelItems];
#pragma unroll
    for (int t = 0; t < kRelItems; ++t) {
      const uint64_t i = i0 + lane + (uint64_t)t * lanes;
      if (i < d) {
        dv[t] = dst0[src + i];
        lv[t] = lab0[src + i];
      }
    }
#pragma unroll
    for (int t = 0; t < kRelItems; ++t)
      if (i0 + lane + (uint64_t)t * lanes < d) dv[t] = o2p[dv[t]];
#pragma unroll
    for (int t = 0; t < kRelItems; ++t) {
      const uint64_t i = i0 + lane + (uint64_t)t * lanes;
      if (i < d) {
        dst[at + i] = dv[t];
        lab[at + i] = (TO)lv[t];
      }
    }
  }
}

// Out-degree 65..4096: one warp per node.
template <typename TI, typename TO>
__global__ void k_relabel_edges_large(uint64_t p_first, uint64_t p_end, const uint32_t* p2o, const uint32_t* o2p,
                                      const uint64_t* off0, const uint32_t* dst0, const TI* lab0, const uint64_t* off,
                                      uint32_t* dst, TO* lab) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t p = p_first + ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5); p < p_end;
       p += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t o = p2o[p];
    const uint64_t s0 = off0[o];
    relabel_run(s0, off[p], off0[o + 1] - s0, lane, 32u, o2p, dst0, lab0, dst, lab);
  }
}

// Hub edges: one CTA per chunk of kHubChunk edges (chunks as in the hub
// signature kernels: hub index, first edge in the new table, length).
template <typename TI, typename TO>
__global__ void k_relabel_edges_hub(uint64_t hub_first, const uint4* chunks, const uint32_t* p2o, const uint32_t* o2p,
                                    const uint64_t* off0, const uint32_t* dst0, const TI* lab0, const uint64_t* off,
                                    uint32_t* dst, TO* lab) {
  const uint4 c = chunks[blockIdx.x];
  const uint64_t p = hub_first + c.x;
  const uint64_t begin = ((uint64_t)c.z << 32) | c.y;
  const uint64_t src = off0[p2o[p]] + (begin - off[p]);
  relabel_run(src, begin, c.w, threadIdx.x, blockDim.x, o2p, dst0, lab0, dst, lab);
}

template <typename TI, typename TO>
void relabel_edges(Store& s, const uint64_t* off0, const uint32_t* dst0, const TI* lab0, TO* lab, int sms) {
  const uint64_t n = s.n;
  const uint32_t* o2p = ptr<uint32_t>(s.o2p);
  const uint64_t* off = ptr<uint64_t>(s.offsets);
  uint32_t* dst = ptr<uint32_t>(s.dst);
  const uint64_t n_small = s.class_start[kClassWarp];
  if (n_small) {
    const unsigned g1 = (unsigned)std::min<uint64_t>(grid_for(n_small, 256), (uint64_t)sms * 32);
    k_relabel_edges_small<TI, TO><<<g1, 256, 0, s.stream>>>(n_small, ptr<uint32_t>(s.p2o), o2p, off0, dst0, lab0, off,
                                                           dst, lab);
  }
  const uint64_t dead = s.class_start[kClassDead];
  if (n > dead)
    k_relabel_edges_dead<TI, TO><<<(unsigned)std::min<uint64_t>(grid_for(n - dead, 256), (uint64_t)sms * 8), 256, 0,
                                   s.stream>>>(dead, n, ptr<uint32_t>(s.p2o), o2p, off0, dst0, lab0, off, dst, lab);
  const uint64_t pf = s.class_start[kClassWarp], pe = s.class_start[kClassHub];
  if (pe > pf) {
    const unsigned g2 = (unsigned)std::min<uint64_t>(grid_for((pe - pf) * 32, 256), (uint64_t)sms * 32);
    k_relabel_edges_large<TI, TO><<<g2, 256, 0, s.stream>>>(pf, pe, ptr<uint32_t>(s.p2o), o2p, off0, dst0, lab0, off,
                                                           dst, lab);
  }
  if (s.n_hub_chunks)
    k_relabel_edges_hub<TI, TO><<<(unsigned)s.n_hub_chunks, 256, 0, s.stream>>>(
        s.class_start[kClassHub], ptr<uint4>(s.hub_chunks), ptr<uint32_t>(s.p2o), o2p, off0, dst0, lab0, off, dst, lab);
}

// Exclusive scan of a uint64 array in place, with an optional copy.
__global__ void __launch_bounds__(kScanThreads) k_tile_sum64(const uint64_t* a, uint64_t n, uint64_t* bsum) {
  __shared__ unsigned long long red[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  unsigned long long c = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    const uint64_t i = base + (uint64_t)t * kScanThreads + threadIdx.x;
    if (i < n) c += a[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) tot += red[w];
    bsum[blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_tile_scan64(uint64_t* a, uint64_t n, const uint64_t* bsum,
                                                                uint64_t* copy) {
  __shared__ unsigned long long wt[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  unsigned long long f[kScanItems];
  unsigned long long c = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    f[t] = base + t < n ? a[base + t] : 0ull;
    c += f[t];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = wt[lane];
    unsigned long long xx = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(kFull, xx, o);
      if (lane >= o) xx += y;
    }
    wt[lane] = xx - t;
  }
  __syncthreads();
  unsigned long long run = bsum[blockIdx.x] + wt[w] + (x - c);
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) {
      a[base + t] = run;
      if (copy) copy[base + t] = run;
    }
    run += f[t];
  }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
Status scan64(Store& s, uint64_t* a, uint64_t n, uint64_t* copy) {
  if (!n) return Status::Ok();
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  Status st = ensure(s, s.bsum, std::max<uint64_t>(tiles, 64) * 8);
  if (!st.ok()) return st;
  uint64_t* bs = ptr<uint64_t>(s.bsum);
  k_tile_sum64<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(a, n, bs);
  k_scan_tiles<<<1, kScanThreads, 0, s.stream>>>(bs, tiles, ptr<unsigned long long>(s.d_scalars) + 15);
  k_tile_scan64<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(a, n, bs, copy);
  return launch_check("scan64");
}

template <int NT, int MIN_DEG, typename LabelT, typename K>
cudaError_t set_chunk_attr() {
  return cudaFuncSetAttribute(k_sig_chunk<NT, MIN_DEG, LabelT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(ChunkSmem<K, NT, MIN_DEG>));
}

template <typename LabelT, typename K>
cudaError_t set_smem_attrs_label() {
  cudaError_t e = set_chunk_attr<kSmallChunkThreads, kChunkMin64, LabelT, K>();
  if (e == cudaSuccess) e = set_chunk_attr<kSmallChunkThreads, kChunkMin1K, LabelT, K>();
  if (e == cudaSuccess) e = set_chunk_attr<kChunkThreads, kChunkMin4K, LabelT, K>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hub_chunk<LabelT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hub_chunk_smem<K>());
  return e;
}

template <typename K>
Status set_smem_attrs_for() {
  cudaError_t e = set_smem_attrs_label<uint8_t, K>();

  if (e == cudaSuccess) e = set_smem_attrs_label<uint32_t, K>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hub_bucket<K, kHubUcaps[0]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BucketSmem<K, kHubUcaps[0]>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hub_bucket<K, kHubUcaps[1]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BucketSmem<K, kHubUcaps[1]>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hub_bucket<K, kHubUcaps[2]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BucketSmem<K, kHubUcaps[2]>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_verify_long<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)verify_ws_bytes<K>());
  return cuda_check(e, "cudaFuncSetAttribute");
}

Status set_smem_attrs(int device) {
  static bool done[64] = {false};
  if (device >= 0 && device < 64 && done[device]) return Status::Ok();
  Status st = set_smem_attrs_for<uint32_t>();
  if (st.ok()) st = set_smem_attrs_for<uint64_t>();
  if (st.ok() && device >= 0 && device < 64) done[device] = true;
  return st;
}

Status read_scalars(Store& s, uint64_t* out) {
  Status st = cuda_check(cudaMemcpyAsync(s.h_scalars.p, s.d_scalars.p, 16 * sizeof(uint64_t),
                                         cudaMemcpyDeviceToHost, s.stream), "read scalars");
  if (!st.ok()) return st;
  st = cuda_check(cudaStreamSynchronize(s.stream), "stream sync");
  if (!st.ok()) return st;
  std::memcpy(out, s.h_scalars.p, 16 * sizeof(uint64_t));
  return Status::Ok();
}

// Checked mode: bring a check kernel's outcome to the host.  Returns CHECKED if
// an index check failed (the kernels that would use the array are not run).
Status checked_outcome(Store& s, const char* what) {
  uint32_t e = 0;
  Status st = launch_check(what);
  if (st.ok()) st = cuda_check(cudaMemcpyAsync(&e, s.d_err.p, 4, cudaMemcpyDeviceToHost, s.stream), what);
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), what);
  if (!st.ok()) return st;
  if (e & kErrChecked) return Status::Err(KBISIM_ERR_CHECKED, std::string("index check failed: ") + what);
  return Status::Ok();
}

Status check_below(Store& s, const uint32_t* a, uint64_t n, uint64_t bound, const char* what) {
  if (!n) return Status::Ok();
  const unsigned g = (unsigned)std::min<uint64_t>(grid_for(n, 256), (uint64_t)sm_count(s.device) * 16);
  k_check_below<<<g, 256, 0, s.stream>>>(a, n, bound, ptr<uint32_t>(s.d_err));
  return checked_outcome(s, what);
}

uint64_t table_capacity(uint64_t n) {
  uint64_t c = 1024;
  while (c < 2 * n) c <<= 1;
  return c;
}

// After a first insert + verify pass (scalars in h): compare the long
// signatures, then regroup the nodes a hash collision left unresolved until
// none is left.  The unresolved nodes hold whole classes; the smallest
// unresolved node of each hash group heads its class, so every pass settles
// at least one class per group (a pass that settles nothing is an error).
Status settle_unresolved(Store& s, const GroupArgs& g, const VerifyArgs& v, bool key64, uint64_t* h, int long_cls) {
  Status st;
  unsigned long long* sc = ptr<unsigned long long>(s.d_scalars);
  const int sms = sm_count(s.device);
  const unsigned ver_grid = resident_blocks(k_group_verify, kVerNodeThreads, 0, sms);
  const unsigned ins_grid = resident_blocks(k_group_insert, kInsThreads, 0, sms);
  if (h[6]) {
    TimedScope ts(s, long_cls, 1);
    const unsigned b = (unsigned)std::min<uint64_t>(h[6], (uint64_t)sms * 8);
    if (key64) k_verify_long<uint64_t><<<b, kVerThreads, verify_ws_bytes<uint64_t>(), s.stream>>>(g, v, h[6]);
    else k_verify_long<uint32_t><<<b, kVerThreads, verify_ws_bytes<uint32_t>(), s.stream>>>(g, v, h[6]);
    if (!(st = launch_check("k_verify_long")).ok()) return st;
    if (!(st = read_scalars(s, h)).ok()) return st;
  }
  uint64_t unresolved_n = h[1];
  int cur = 0;
  while (unresolved_n > 0) {
    const uint64_t cap = table_capacity(unresolved_n);
    GroupArgs g2 = g;
    g2.tmask = cap - 1;
    VerifyArgs v2 = v;
    v2.out_list = ptr<uint32_t>(s.ulist[cur ^ 1]);
    v2.n_out = sc + 5;
    const unsigned b2 = (unsigned)std::min<uint64_t>(grid_for(unresolved_n, kVerTile), ver_grid);
    {
      TimedScope ts(s, KBISIM_KERNEL_OTHER, 2);
      cudaMemsetAsync(s.table.p, 0xFF, cap * 8, s.stream);
      cudaMemsetAsync(sc + 5, 0, 16, s.stream);  // [5] and [6]
      k_group_insert<<<(unsigned)std::min<uint64_t>((unresolved_n + kInsChunk - 1) / kInsChunk, ins_grid),
                       kInsThreads, 0, s.stream>>>(g2, ptr<uint32_t>(s.ulist[cur]), unresolved_n);
      k_group_verify<<<b2, kVerNodeThreads, 0, s.stream>>>(g2, v2, ptr<uint32_t>(s.ulist[cur]), unresolved_n);
    }
    if (!(st = launch_check("collision repair")).ok()) return st;
    if (!(st = read_scalars(s, h)).ok()) return st;
    if (h[6]) {
      TimedScope ts(s, KBISIM_KERNEL_OTHER, 1);
      const unsigned b = (unsigned)std::min<uint64_t>(h[6], (uint64_t)sms * 8);
      if (key64) k_verify_long<uint64_t><<<b, kVerThreads, verify_ws_bytes<uint64_t>(), s.stream>>>(g2, v2, h[6]);
      else k_verify_long<uint32_t><<<b, kVerThreads, verify_ws_bytes<uint32_t>(), s.stream>>>(g2, v2, h[6]);
      if (!(st = launch_check("k_verify_long")).ok()) return st;
      if (!(st = read_scalars(s, h)).ok()) return st;
    }
    if (h[5] >= unresolved_n)
      return Status::Err(KBISIM_ERR_TIMEOUT, "collision repair made no progress");
    unresolved_n = h[5];
    cur ^= 1;
  }
  return Status::Ok();
}

// Scalars used per round (uint64 words of Store::d_scalars):
//  [1] unresolved after the first pass, [2] key total, [3] largest signature,
//  [4] collided nodes, [5] unresolved after a repair pass, [6] long-signature
//  pairs, [7] error flags copy, [8] nodes alone in their block, [15] scan
//  total (after renumbering: the number of blocks).
Status group_and_rank(Store& s, int mode, const uint32_t* prev, bool key64, uint32_t* pid, uint64_t* blocks,
                      uint64_t* collided, bool with_stats, uint64_t* keys, uint64_t* maxsig, bool use_alone) {
  const uint64_t n = s.n, na = s.n_alive;
  Status st;
  unsigned long long* sc = ptr<unsigned long long>(s.d_scalars);
  GroupArgs g;
  g.hash = ptr<uint64_t>(s.hash);
  g.p2o = ptr<uint32_t>(s.p2o);
  g.o2p = ptr<uint32_t>(s.o2p);
  g.table = ptr<unsigned long long>(s.table);
  g.tmask = s.tcap - 1;
  g.slot = ptr<uint32_t>(s.slot);
  g.rep = ptr<uint32_t>(s.rep);
  g.err = ptr<uint32_t>(s.d_err);
  g.alone = use_alone ? ptr<uint8_t>(s.alone) : nullptr;
  g.read_first = mode == 0 ? 1 : 0;
  VerifyArgs v;
  v.mode = mode;
  v.key64 = key64 ? 1 : 0;
  v.nlabel = ptr<uint32_t>(s.nlabel);
  v.prev = prev;
  v.ucnt = ptr<uint32_t>(s.ucnt);
  v.off = ptr<uint64_t>(s.offsets);
  v.sigkey = s.sigkey.p;
  v.n_collided = sc + 4;
  v.long_list = ptr<uint32_t>(s.long_pairs);
  v.n_long = sc + 6;
  v.hbits = ptr<uint32_t>(s.hbits);
  v.member = ptr<uint8_t>(s.member);
  const uint64_t words = (n + 31) / 32;
  const int sms = sm_count(s.device);
  const unsigned ver_grid = resident_blocks(k_group_verify, kVerNodeThreads, 0, sms);
  const unsigned gblocks = (unsigned)std::min<uint64_t>(grid_for(na, kVerTile), ver_grid);
  {
    TimedScope ts(s, KBISIM_KERNEL_OTHER, 0);
    cudaMemsetAsync(s.d_scalars.p, 0, 15 * 8, s.stream);
    // marks of the canonical numbering, set as representatives are settled
    cudaMemsetAsync(s.hbits.p, 0, words * 4, s.stream);
    cudaMemsetAsync(s.member.p, 0, n, s.stream);
  }
  v.out_list = ptr<uint32_t>(s.ulist[0]);
  v.n_out = sc + 1;
  // only nodes not alone in their previous block are inserted
  const uint64_t ins = use_alone ? na - std::min(na, s.n_alone) : na;
  const unsigned ins_grid = resident_blocks(k_group_insert, kInsThreads, 0, sms);
  const uint64_t tcap = std::min<uint64_t>(s.tcap, table_capacity(ins));
  g.tmask = tcap - 1;
  {
    TimedScope ts(s, KBISIM_KERNEL_OTHER, 0);
    cudaMemsetAsync(s.table.p, 0xFF, tcap * 8, s.stream);
  }
  const unsigned iblocks = (unsigned)std::min<uint64_t>((na + kInsChunk - 1) / kInsChunk, ins_grid);
  {
    TimedScope ts(s, KBISIM_KERNEL_GROUP, na ? 1 : 0);
    if (na) k_group_insert<<<iblocks, kInsThreads, 0, s.stream>>>(g, nullptr, na);
  }
  if (!(st = launch_check("k_group_insert")).ok()) return st;
  {
    TimedScope ts(s, KBISIM_KERNEL_VERIFY, 1);
    k_group_verify<<<gblocks, kVerNodeThreads, 0, s.stream>>>(g, v, nullptr, na);
  }
  if (!(st = launch_check("k_group_verify")).ok()) return st;
  uint64_t h[16];
  if (!(st = read_scalars(s, h)).ok()) return st;
  if (!(st = settle_unresolved(s, g, v, key64, h, KBISIM_KERNEL_VERIFY)).ok()) return st;
  *collided = h[4];
  if (s.checked && !(st = check_below(s, g.rep, na, n, "block heads")).ok()) return st;
  // canonical renumbering
  RankArgs r;
  r.n = n;
  r.n_alive = na;
  r.rep = g.rep;
  r.p2o = g.p2o;
  r.ucnt = with_stats ? ptr<uint32_t>(s.ucnt) : nullptr;
  r.hbits = ptr<uint32_t>(s.hbits);
  r.hword = ptr<uint64_t>(s.hword);
  r.member = ptr<uint8_t>(s.member);
  r.alone = ptr<uint8_t>(s.alone);
  r.pid = pid;
  r.stats = sc;
  {
    TimedScope ts(s, KBISIM_KERNEL_RENUMBER, n ? 5 : 0);  // 2 kernels + the 3 of scan64
    if (n) {
      k_word_counts<<<(unsigned)std::min<uint64_t>(grid_for(words, 256), (uint64_t)sms * 16), 256, 0, s.stream>>>(
          r.hbits, words, r.hword);
      if (!(st = scan64(s, r.hword, words, nullptr)).ok()) return st;
      k_pid_fill<<<(unsigned)std::min<uint64_t>(grid_for(n, 256), (uint64_t)sms * 16), 256, 0, s.stream>>>(r);
    }
  }
  if (!(st = launch_check("renumber")).ok()) return st;
  cudaMemcpyAsync(sc + 7, s.d_err.p, 4, cudaMemcpyDeviceToDevice, s.stream);
  if (!(st = read_scalars(s, h)).ok()) return st;
  *blocks = n ? h[15] : 0;  // scan total: heads
  if (s.checked && !(st = check_below(s, pid, na, *blocks, "identifiers")).ok()) return st;
  s.n_alone = h[8];
  if (keys) *keys = h[2];
  if (maxsig) *maxsig = h[3];
  const uint32_t e = (uint32_t)h[7];
  if (e & kErrProbe) return Status::Err(KBISIM_ERR_TIMEOUT, "hash table probe bound exceeded");
  if (e & kErrChecked) return Status::Err(KBISIM_ERR_CHECKED, "device bounds check failed");
  return Status::Ok();
}

// (Re)build the per-hub bucket table for the bucket size s.hub_ucap and the
// current extra bits: hub i has 2^(bits_i + extra) buckets of cap_i key words
// each, bits_i the least with degree <= (hub_ucap / 2) << bits_i, cap_i twice
// the mean bucket load plus a margin (at most hub_ucap).
Status hub_layout(Store& s) {
  Status st;
  std::vector<uint32_t> bits(s.n_hub), cap(s.n_hub);
  std::vector<uint64_t> bbase(s.n_hub + 1, 0), tbase(s.n_hub, 0);
  uint64_t words = 0;
  const uint64_t target = s.hub_ucap / 2;
  for (uint64_t i = 0; i < s.n_hub; ++i) {
    uint32_t db = 0;
    while ((target << db) < s.h_hub_deg[i]) ++db;
    bits[i] = db + s.h_hub_xbits[i];
    const uint64_t nb = 1ull << bits[i];
    bbase[i + 1] = bbase[i] + nb;
    const uint64_t mean = (s.h_hub_deg[i] + nb - 1) / nb;
    cap[i] = (uint32_t)std::min<uint64_t>(s.h_hub_deg[i], std::min<uint64_t>(s.hub_ucap, 2 * mean + 256)
                                                                << s.h_hub_shift[i]);
    tbase[i] = words;
    words += nb * cap[i];
  }
  s.n_hub_buckets = bbase[s.n_hub];
  s.hub_tmp_words = words;
  std::vector<uint32_t> bhub(s.n_hub_buckets);
  for (uint64_t i = 0; i < s.n_hub; ++i)
    for (uint64_t b = bbase[i]; b < bbase[i + 1]; ++b) bhub[b] = (uint32_t)i;
  if (!(st = ensure(s, s.hub_bits, s.n_hub * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_cap, s.n_hub * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_bbase, (s.n_hub + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, s.hub_tbase, s.n_hub * 8)).ok()) return st;
  if (!(st = ensure(s, s.bucket_hub, s.n_hub_buckets * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_cursor, s.n_hub_buckets * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_acc, s.n_hub * 24)).ok()) return st;
  if (!(st = ensure(s, s.hub_mode, s.n_hub)).ok()) return st;
  if (!(st = ensure(s, s.hub_force, s.n_hub)).ok()) return st;
  if (!(st = ensure(s, s.hub_err, s.n_hub * 4)).ok()) return st;
  cudaMemcpyAsync(s.hub_force.p, s.h_hub_force.data(), s.n_hub, cudaMemcpyHostToDevice, s.stream);  cudaMemcpyAsync(s.hub_bits.p, bits.data(), s.n_hub * 4, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.hub_cap.p, cap.data(), s.n_hub * 4, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.hub_bbase.p, bbase.data(), (s.n_hub + 1) * 8, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.hub_tbase.p, tbase.data(), s.n_hub * 8, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.bucket_hub.p, bhub.data(), s.n_hub_buckets * 4, cudaMemcpyHostToDevice, s.stream);
  return cuda_check(cudaStreamSynchronize(s.stream), "hub layout");
}

// The bucket pass with buckets of at most U key words: one resident wave of CTAs.
template <typename K, int U>
void launch_hub_bucket(Store& s, const SigArgs& a, const HubArgs& h, int sms) {
  const unsigned g = (unsigned)std::min<uint64_t>(
      s.n_hub_buckets, resident_blocks(k_hub_bucket<K, U>, kBucketThreads, sizeof(BucketSmem<K, U>), sms));
  k_hub_bucket<K, U><<<g, kBucketThreads, sizeof(BucketSmem<K, U>), s.stream>>>(a, h, s.n_hub_buckets);
}

template <typename LabelT, typename K>
Status run_signatures(Store& s, const SigArgs& a) {
  Status st;
  const int sms = sm_count(s.device);
  // thread-per-node classes: 0..4 (out-degree <= 8) in one launch, 5 and 6
  // (9..16, 17..32) in one launch each, so that each kernel carries only its
  // own unrolled code; class 7 (33..64) runs as 128-thread chunks
  auto small_launch = [&](int first, int last) {
    SmallLaunch L;
    uint32_t b = 0;
    for (int c = 0; c < kSmallClasses; ++c) {
      L.start[c] = s.class_start[c];
      L.count[c] = s.class_start[c + 1] - s.class_start[c];
      L.bstart[c] = b;
      if (c >= first && c <= last) b += (uint32_t)((L.count[c] + kSmallThreads - 1) / kSmallThreads);
    }
    L.bstart[kSmallClasses] = b;
    return L;
  };
  const SmallLaunch L04 = small_launch(0, 4), L5 = small_launch(5, 5), L6 = small_launch(6, 6);
  const uint32_t n04 = L04.bstart[5], n5 = L5.bstart[6] - L5.bstart[5], n6 = L6.bstart[7] - L6.bstart[6];
  {
    TimedScope ts(s, KBISIM_KERNEL_SIG_SMALL, (n04 ? 1 : 0) + (n5 ? 1 : 0) + (n6 ? 1 : 0) + (s.n_mid_chunks[0] ? 1 : 0));
    if (n04) k_sig_small<0, 4, LabelT, K><<<n04, kSmallThreads, 0, s.stream>>>(a, L04);
    if (n5) k_sig_small<5, 5, LabelT, K><<<n5, kSmallThreads, 0, s.stream>>>(a, L5);
    if (n6) k_sig_small<6, 6, LabelT, K><<<n6, kSmallThreads, 0, s.stream>>>(a, L6);
    if (s.n_mid_chunks[0])
      k_sig_chunk<kSmallChunkThreads, kChunkMin64, LabelT, K>
          <<<(unsigned)s.n_mid_chunks[0], kSmallChunkThreads,
             sizeof(ChunkSmem<K, kSmallChunkThreads, kChunkMin64>), s.stream>>>(a, ptr<uint2>(s.mid_chunks));
  }
  if (!(st = launch_check("k_sig_small")).ok()) return st;
  if (s.n_mid_chunks[1] + s.n_mid_chunks[2]) {
    TimedScope ts(s, KBISIM_KERNEL_SIG_MEDIUM, (s.n_mid_chunks[1] ? 1 : 0) + (s.n_mid_chunks[2] ? 1 : 0));
    if (s.n_mid_chunks[1])
      k_sig_chunk<kSmallChunkThreads, kChunkMin1K, LabelT, K>
          <<<(unsigned)s.n_mid_chunks[1], kSmallChunkThreads,
             sizeof(ChunkSmem<K, kSmallChunkThreads, kChunkMin1K>), s.stream>>>(
              a, ptr<uint2>(s.mid_chunks) + s.n_mid_chunks[0]);
    if (s.n_mid_chunks[2])
      k_sig_chunk<kChunkThreads, kChunkMin4K, LabelT, K>
          <<<(unsigned)s.n_mid_chunks[2], kChunkThreads, sizeof(ChunkSmem<K, kChunkThreads, kChunkMin4K>),
             s.stream>>>(a, ptr<uint2>(s.mid_chunks) + s.n_mid_chunks[0] + s.n_mid_chunks[1]);
  }
  if (!(st = launch_check("k_sig_chunk")).ok()) return st;
  if (s.n_hub) {
    auto run_hubs = [&]() -> Status {
      Status st;
      // a repeat after an overflow runs only the hubs that overflowed (the
      // others' signatures are written): a mask over their internal ids
      SigArgs ah = a;
      for (int attempt = 0;; ++attempt) {
        if (!(st = ensure(s, s.hub_tmp, s.hub_tmp_words * sizeof(K))).ok()) return st;
        HubArgs h;
        h.first = s.class_start[kClassHub];
        h.hub_bits = ptr<uint32_t>(s.hub_bits);
        h.hub_bbase = ptr<uint64_t>(s.hub_bbase);
        h.hub_cap = ptr<uint32_t>(s.hub_cap);
        h.hub_tbase = ptr<uint64_t>(s.hub_tbase);
        h.bucket_hub = ptr<uint32_t>(s.bucket_hub);
        h.chunks = ptr<uint4>(s.hub_chunks);
        h.cursor = ptr<uint32_t>(s.hub_cursor);
        h.hub_cur = ptr<unsigned long long>(s.hub_acc);
        h.hub_term = reinterpret_cast<uint32_t*>(h.hub_cur + s.n_hub);
        h.tmp = s.hub_tmp.p;
        h.mode = ptr<uint8_t>(s.hub_mode);
        h.force = ptr<uint8_t>(s.hub_force);
        h.hub_err = ptr<uint32_t>(s.hub_err);
        {
          // each hub's chunks run either the deduplicating pass or the plain
          // scatter, as its key sample says; both kernels cover all chunks and
          // skip those of the other kind
          TimedScope ts(s, KBISIM_KERNEL_SIG_HUB, 5);
          cudaMemsetAsync(h.cursor, 0, s.n_hub_buckets * 4, s.stream);
          cudaMemsetAsync(s.hub_acc.p, 0, s.n_hub * 24, s.stream);
          cudaMemsetAsync(s.hub_err.p, 0, s.n_hub * 4, s.stream);
          k_hub_sample<LabelT, K><<<(unsigned)((s.n_hub + 7) / 8), 256, 0, s.stream>>>(ah, h, s.n_hub);
          k_hub_chunk<LabelT, K><<<(unsigned)s.n_hub_chunks, kChunkThreads, hub_chunk_smem<K>(), s.stream>>>(ah, h);
          k_hub_scatter<LabelT, K><<<(unsigned)s.n_hub_chunks, kChunkThreads, 0, s.stream>>>(ah, h);
          if (s.hub_ucap == (uint32_t)kHubUcaps[1]) launch_hub_bucket<K, kHubUcaps[1]>(s, ah, h, sms);
          else if (s.hub_ucap == (uint32_t)kHubUcaps[2]) launch_hub_bucket<K, kHubUcaps[2]>(s, ah, h, sms);
          else launch_hub_bucket<K, kHubUcaps[0]>(s, ah, h, sms);
          k_hub_finish<<<(unsigned)((s.n_hub + 255) / 256), 256, 0, s.stream>>>(ah, h, s.n_hub);
        }
        if (!(st = launch_check("hub kernels")).ok()) return st;
        uint32_t e = 0;
        st = cuda_check(cudaMemcpyAsync(&e, s.d_err.p, 4, cudaMemcpyDeviceToHost, s.stream), "read err");
        if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
        if (!st.ok()) return st;
        if (!(e & (kErrHubOverflow | kErrHubSet))) return Status::Ok();
        if (attempt >= 40) return Status::Err(KBISIM_ERR_TIMEOUT, "hub bucket overflow persists");
        std::vector<uint32_t> herr(s.n_hub);
        std::vector<uint8_t> hmode(s.n_hub);
        st = cuda_check(cudaMemcpyAsync(herr.data(), s.hub_err.p, s.n_hub * 4, cudaMemcpyDeviceToHost, s.stream),
                        "hub flags");
        if (st.ok())
          st = cuda_check(cudaMemcpyAsync(hmode.data(), s.hub_mode.p, s.n_hub, cudaMemcpyDeviceToHost, s.stream),
                          "hub modes");
        if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
        if (!st.ok()) return st;
        for (uint64_t i = 0; i < s.n_hub; ++i) {
          // a bucket overflowed (a key repeated many times): larger buckets for
          // the hub, up to its degree, or, once the scatter has overflowed
          // buckets kHubScatterShiftMax times larger than the first, the
          // deduplicating pass; too many distinct keys in a bucket: more buckets
          if (herr[i] & kErrHubOverflow) {
            if (hmode[i] && s.h_hub_shift[i] >= kHubScatterShiftMax) s.h_hub_force[i] = 1;
            else s.h_hub_shift[i] += 1;
          }
          if (herr[i] & kErrHubSet) s.h_hub_xbits[i] += 1;
        }
        if (!(st = hub_layout(s)).ok()) return st;
        // the repeat's mask: the words of the hub id range, bits of the failed hubs
        const uint64_t first = s.class_start[kClassHub], w0 = first >> 5, w1 = (first + s.n_hub + 31) >> 5;
        std::vector<uint32_t> bits(w1 - w0, 0u);
        for (uint64_t i = 0; i < s.n_hub; ++i)
          if (herr[i]) bits[((first + i) >> 5) - w0] |= 1u << ((first + i) & 31);
        if (!(st = ensure(s, s.hub_retry, (w1 + 1) * 4)).ok()) return st;
        st = cuda_check(cudaMemcpyAsync(ptr<uint32_t>(s.hub_retry) + w0, bits.data(), bits.size() * 4,
                                        cudaMemcpyHostToDevice, s.stream), "hub repeat mask");
        if (!st.ok()) return st;
        ah.fmask = ptr<uint32_t>(s.hub_retry);
        cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
      }
    };
    if (!s.tune_now) return run_hubs();
    // tuning (once per handle, on a full round from level 2 on): each bucket
    // size runs the hub pass twice, the sizes alternating, each pass timed
    // with the repeats its overflows need (a repeat runs only the hubs that
    // overflowed).  A size's second pass starts from the bucket growth its
    // first pass learned and finds the round's data in L2 as the first passes
    // left it, so the second passes compare the sizes as the later rounds run
    // them; the first size (the default) is kept unless another is faster by
    // more than kHubTuneMargin.  Every pass writes the same signatures, so the
    // round's result is the last pass's.
    constexpr int kSizes = 2;
    constexpr float kHubTuneMargin = 0.05f;
    // bucket growth is learned per size: each starts from the growth before
    // tuning, and the chosen size keeps its own
    const std::vector<uint32_t> x0 = s.h_hub_xbits, sh0 = s.h_hub_shift;
    const std::vector<uint8_t> f0 = s.h_hub_force;
    std::vector<uint32_t> xs[kSizes], shs[kSizes];
    std::vector<uint8_t> fs[kSizes];
    cudaEvent_t ev[2];
    if (!(st = cuda_check(cudaEventCreate(&ev[0]), "event")).ok()) return st;
    if (!(st = cuda_check(cudaEventCreate(&ev[1]), "event")).ok()) {
      cudaEventDestroy(ev[0]);
      return st;
    }
    for (int rep = 0; rep < 2 && st.ok(); ++rep) {
      for (int c = 0; c < kSizes && st.ok(); ++c) {
        s.h_hub_xbits = rep ? xs[c] : x0;
        s.h_hub_shift = rep ? shs[c] : sh0;
        s.h_hub_force = rep ? fs[c] : f0;
        s.hub_ucap = (uint32_t)kHubUcaps[c];
        if (!(st = hub_layout(s)).ok()) break;
        cudaEventRecord(ev[0], s.stream);
        if (!(st = run_hubs()).ok()) break;
        cudaEventRecord(ev[1], s.stream);
        if (!(st = cuda_check(cudaEventSynchronize(ev[1]), "event")).ok()) break;
        cudaEventElapsedTime(&s.hub_tune_ms[c], ev[0], ev[1]);
        xs[c] = s.h_hub_xbits;
        shs[c] = s.h_hub_shift;
        fs[c] = s.h_hub_force;
      }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (!st.ok()) return st;
    s.hub_tune = 2;
    int best = 0;
    for (int c = 1; c < kSizes; ++c)
      if (s.hub_tune_ms[c] < s.hub_tune_ms[best] * (1.0f - kHubTuneMargin)) best = c;
    if (best != kSizes - 1) {
      s.hub_ucap = (uint32_t)kHubUcaps[best];
      s.h_hub_xbits.swap(xs[best]);
      s.h_hub_shift.swap(shs[best]);
      s.h_hub_force.swap(fs[best]);
      if (!(st = hub_layout(s)).ok()) return st;
    }
  }
  return Status::Ok();
}

Status ensure_round_scratch(Store& s) {
  Status st;
  const uint64_t n = std::max<uint64_t>(s.n, 1), m = std::max<uint64_t>(s.m, 1);
  const uint64_t cap = table_capacity(std::max<uint64_t>(s.n_alive, 1));
  if (!(st = ensure(s, s.sigkey, m * 8)).ok()) return st;
  if (!(st = ensure(s, s.ucnt, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.hash, n * 8)).ok()) return st;
  if (!(st = ensure(s, s.table, cap * 8)).ok()) return st;
  s.tcap = cap;
  if (!(st = ensure(s, s.slot, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.rep, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.ulist[0], n * 4)).ok()) return st;
  if (!(st = ensure(s, s.ulist[1], n * 4)).ok()) return st;
  if (!(st = ensure(s, s.hbits, ((n + 31) / 32) * 4 + 16)).ok()) return st;
  if (!(st = ensure(s, s.hword, std::max<uint64_t>((n + 31) / 32, 1) * 8)).ok()) return st;
  if (!(st = ensure(s, s.member, n + 16)).ok()) return st;
  if (!(st = ensure(s, s.alone, n + 16)).ok()) return st;
  if (!(st = ensure(s, s.long_pairs, n * 8)).ok()) return st;
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (!(st = ensure(s, s.bsum, std::max<uint64_t>(tiles, 64) * 8)).ok()) return st;
  return Status::Ok();
}

uint32_t bits_for(uint64_t v) {  // bits needed to represent values 0..v
  uint32_t b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

}  // namespace

// Bucket growth of the hubs, keyed by original node id: a graph laid out
// again after an update, or loaded again into the same handle, keeps what its
// hubs' buckets learned, instead of overflowing and growing them again in the
// next refinement.  Growth only sizes buckets: a wrong carry costs memory or
// a repeat, never a result.
Status save_hub_growth(Store& s, HubGrowth* g) {
  g->orig.clear();
  g->xbits.clear();
  g->shift.clear();
  g->deg.clear();
  g->force.clear();
  if (!s.has_graph || !s.n_hub || s.h_hub_xbits.size() != s.n_hub) return Status::Ok();
  bool any = false;
  for (uint64_t i = 0; i < s.n_hub && !any; ++i) any = s.h_hub_xbits[i] || s.h_hub_shift[i] || s.h_hub_force[i];
  if (!any) return Status::Ok();
  std::vector<uint32_t> p2o(s.n_hub);
  Status st = cuda_check(cudaMemcpyAsync(p2o.data(), ptr<uint32_t>(s.p2o) + s.class_start[kClassHub], s.n_hub * 4,
                                         cudaMemcpyDeviceToHost, s.stream), "hub ids");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  for (uint64_t i = 0; i < s.n_hub; ++i)
    if (s.h_hub_xbits[i] || s.h_hub_shift[i] || s.h_hub_force[i]) {
      g->orig.push_back(p2o[i]);
      g->xbits.push_back(s.h_hub_xbits[i]);
      g->shift.push_back(s.h_hub_shift[i]);
      g->deg.push_back(i < s.h_hub_deg.size() ? s.h_hub_deg[i] : 0);
      g->force.push_back(s.h_hub_force[i]);
    }
  return Status::Ok();
}

Status restore_hub_growth(Store& s, const HubGrowth& g, bool same_degree) {
  if (g.orig.empty() || !s.has_graph || !s.n_hub) return Status::Ok();
  std::vector<uint32_t> p2o(s.n_hub);
  Status st = cuda_check(cudaMemcpyAsync(p2o.data(), ptr<uint32_t>(s.p2o) + s.class_start[kClassHub], s.n_hub * 4,
                                         cudaMemcpyDeviceToHost, s.stream), "hub ids");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  std::unordered_map<uint32_t, size_t> at;
  at.reserve(g.orig.size() * 2);
  for (size_t j = 0; j < g.orig.size(); ++j) at[g.orig[j]] = j;
  s.h_hub_xbits.resize(s.n_hub, 0);
  s.h_hub_shift.resize(s.n_hub, 0);
  s.h_hub_force.resize(s.n_hub, 0);
  bool changed = false;
  for (uint64_t i = 0; i < s.n_hub; ++i) {
    const auto it = at.find(p2o[i]);
    if (it == at.end()) continue;
    if (same_degree && (i >= s.h_hub_deg.size() || s.h_hub_deg[i] != g.deg[it->second])) continue;
    s.h_hub_xbits[i] = std::max(s.h_hub_xbits[i], g.xbits[it->second]);
    s.h_hub_shift[i] = std::max(s.h_hub_shift[i], g.shift[it->second]);
    s.h_hub_force[i] = std::max(s.h_hub_force[i], g.force[it->second]);
    changed = true;
  }
  return changed ? hub_layout(s) : Status::Ok();
}

// ---------------------------------------------------------------------------
// Relabelling and degree classes (once per graph)
// ---------------------------------------------------------------------------
// Work lists made from the offsets of the degree classes: hub chunks and the
// hubs' bucket layout, and the chunks of whole nodes for out-degree 33..4096.
// `fresh`: a new graph (bucket growth learned on the previous one is dropped).
// Offsets of the out-degree 33..4096 nodes, copied to the host for the chunk
// plan, and the class bounds they cover.
struct MidPlan {
  std::vector<uint64_t> moff;
  uint64_t mf = 0, mw = 0, mb = 0, me = 0;
};

// Hub chunk lists and layout, and the copy of the offsets the chunk plan of
// the out-degree 33..4096 nodes needs (made with the hub offsets' copy).
Status chunk_lists_hubs(Store& s, bool fresh, MidPlan* mp) {
  Status st;
  // hubs: a contiguous internal id range; their offsets come in one copy
  s.n_hub = s.class_start[kClassHub + 1] - s.class_start[kClassHub];
  if (fresh || s.h_hub_xbits.size() != s.n_hub) {  // bucket growth learned on this graph is kept otherwise
    s.h_hub_xbits.assign(s.n_hub, 0);
    s.h_hub_shift.assign(s.n_hub, 0);
    s.h_hub_force.assign(s.n_hub, 0);
  }
  s.h_hub_deg.assign(s.n_hub, 0);
  s.hub_edges = 0;
  s.n_hub_chunks = 0;
  s.n_hub_buckets = 0;
  if (s.n_hub) {
    std::vector<uint64_t> hoff(s.n_hub + 1);
    st = cuda_check(cudaMemcpyAsync(hoff.data(), ptr<uint64_t>(s.offsets) + s.class_start[kClassHub],
                                    (s.n_hub + 1) * 8, cudaMemcpyDeviceToHost, s.stream), "hub offsets");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
    if (!st.ok()) return st;
    std::vector<uint4> chunks;
    std::vector<uint32_t> cstart(s.n_hub + 1, 0);
    for (uint64_t i = 0; i < s.n_hub; ++i) {
      cstart[i] = (uint32_t)chunks.size();
      const uint64_t d = hoff[i + 1] - hoff[i];
      s.h_hub_deg[i] = d;
      s.hub_edges += d;
      for (uint64_t b = 0; b < d; b += kHubChunk) {
        const uint64_t e = hoff[i] + b;
        uint4 q;
        q.x = (uint32_t)i;
        q.y = (uint32_t)(e & 0xFFFFFFFFu);
        q.z = (uint32_t)(e >> 32);
        q.w = (uint32_t)std::min<uint64_t>(kHubChunk, d - b);
        chunks.push_back(q);
      }
    }
    s.n_hub_chunks = chunks.size();
    cstart[s.n_hub] = (uint32_t)chunks.size();
    if (!(st = ensure(s, s.hub_chunks, chunks.size() * sizeof(uint4))).ok()) return st;
    if (!(st = ensure(s, s.hub_cstart, (s.n_hub + 1) * 4)).ok()) return st;
    st = cuda_check(cudaMemcpyAsync(s.hub_chunks.p, chunks.data(), chunks.size() * sizeof(uint4),
                                    cudaMemcpyHostToDevice, s.stream), "hub chunks");
    if (st.ok())
      st = cuda_check(cudaMemcpyAsync(s.hub_cstart.p, cstart.data(), (s.n_hub + 1) * 4, cudaMemcpyHostToDevice,
                                      s.stream), "hub chunks");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "hub chunks");
    if (!st.ok()) return st;
    if (!(st = hub_layout(s)).ok()) return st;
  }
  // the out-degree 33..4096 nodes' offsets for their chunk plan
  mp->mf = s.class_start[kSmallClasses - 1];
  mp->mw = s.class_start[kClassWarp];
  mp->mb = s.class_start[kClassBlock];
  mp->me = s.class_start[kClassHub];
  mp->moff.clear();
  if (mp->me > mp->mf) {
    mp->moff.resize(mp->me - mp->mf + 1);
    st = cuda_check(cudaMemcpyAsync(mp->moff.data(), ptr<uint64_t>(s.offsets) + mp->mf,
                                    (mp->me - mp->mf + 1) * 8, cudaMemcpyDeviceToHost, s.stream),
                    "chunk offsets");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
    if (!st.ok()) return st;
  }
  return Status::Ok();
}

// out-degree 33..4096: runs of whole nodes; 33..64 and 65..1024 in chunks
// of at most 1024 edges (128-thread CTAs), 1025..4096 in chunks of at most
// 4096 edges (512-thread CTAs).  A host loop over the nodes' offsets (about
// 2 ms for 640K nodes), so a load runs it while the GPU relabels the edges.
Status chunk_lists_mid(Store& s, const MidPlan& mp) {
  Status st;
  s.n_mid_chunks[0] = s.n_mid_chunks[1] = s.n_mid_chunks[2] = 0;
  const uint64_t mf = mp.mf, mw = mp.mw, mb = mp.mb, me = mp.me;
  if (me > mf) {
    const std::vector<uint64_t>& moff = mp.moff;
    std::vector<uint2> mc;
    mc.reserve((size_t)((moff[me - mf] - moff[0]) / 512 + (me - mf) / 16 + 16));
    auto pack = [&](uint64_t lo, uint64_t hi, uint64_t max_edges, uint64_t max_nodes) {
      for (uint64_t i = lo; i < hi;) {
        uint64_t j = i + 1;
        while (j < hi && j - i < max_nodes && moff[j + 1] - moff[i] <= max_edges) ++j;
        mc.push_back(make_uint2((uint32_t)(mf + i), (uint32_t)(j - i)));
        i = j;
      }
    };
    using S64 = ChunkShape<kSmallChunkThreads, kChunkMin64>;
    using S1K = ChunkShape<kSmallChunkThreads, kChunkMin1K>;
    using S4K = ChunkShape<kChunkThreads, kChunkMin4K>;
    pack(0, mw - mf, S64::kEdges, S64::kMaxNodes);
    s.n_mid_chunks[0] = mc.size();
    pack(mw - mf, mb - mf, S1K::kEdges, S1K::kMaxNodes);
    s.n_mid_chunks[1] = mc.size() - s.n_mid_chunks[0];
    pack(mb - mf, me - mf, S4K::kEdges, S4K::kMaxNodes);
    s.n_mid_chunks[2] = mc.size() - s.n_mid_chunks[0] - s.n_mid_chunks[1];
    if (!(st = ensure(s, s.mid_chunks, mc.size() * sizeof(uint2))).ok()) return st;
    st = cuda_check(cudaMemcpyAsync(s.mid_chunks.p, mc.data(), mc.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                                    s.stream), "medium chunks");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");  // mc is freed on return
    if (!st.ok()) return st;
  }
  return Status::Ok();
}

Status build_chunk_lists(Store& s, bool fresh) {
  MidPlan mp;
  Status st = chunk_lists_hubs(s, fresh, &mp);
  if (st.ok()) st = chunk_lists_mid(s, mp);
  return st;
}


Status scan_u64(Store& s, uint64_t* a, uint64_t n) { return scan64(s, a, n, nullptr); }

Status relabel_graph(Store& s, const uint64_t* off0, const uint32_t* dst0, const void* lab0,
                     const uint32_t* nlab0, const uint8_t* alive0, uint32_t lab_bytes) {
  Status st = set_smem_attrs(s.device);
  if (!st.ok()) return st;
  const uint64_t n = s.n, m = s.m;
  const int sms = sm_count(s.device);
  const uint64_t ntiles = std::max<uint64_t>(1, (n + kClassTile - 1) / kClassTile);
  // temporaries of the relabelling (kept between loads)
  InUse use(s, kCacheRelabel);
  Buf &tcnt = s.rl_tcnt, &hot = s.rl_hot, &ost = s.rl_ost;
  auto fail = [&](Status e) { return e; };
  if (!(st = ensure(s, tcnt, ntiles * kNumOrder * 8)).ok()) return fail(st);
  if (!(st = ensure(s, hot, std::max<uint64_t>(1, n) * 4)).ok()) return fail(st);
  if (!(st = ensure(s, ost, kNumOrder * 8)).ok()) return fail(st);
  cudaMemsetAsync(tcnt.p, 0, ntiles * kNumOrder * 8, s.stream);
  cudaMemsetAsync(hot.p, 0, std::max<uint64_t>(1, n) * 4, s.stream);
  if (m >> kHotSampleShift)
    k_hot_sample<<<(unsigned)std::min<uint64_t>(grid_for(m >> kHotSampleShift, 256), (uint64_t)sms * 32), 256, 0,
                   s.stream>>>(m, dst0, ptr<uint32_t>(hot));
  if (n)
    k_class_tile_count<<<(unsigned)ntiles, kClassTile, 0, s.stream>>>(n, off0, alive0, ptr<uint32_t>(hot), ntiles,
                                                                      ptr<unsigned long long>(tcnt));
  if (!(st = launch_check("k_class_tile_count")).ok()) return fail(st);
  if (!(st = scan64(s, ptr<uint64_t>(tcnt), ntiles * kNumOrder, nullptr)).ok()) return fail(st);
  k_order_starts<<<1, 128, 0, s.stream>>>(ptr<unsigned long long>(tcnt), ntiles, ptr<unsigned long long>(ost));
  std::vector<uint64_t> hs(kNumOrder);
  st = cuda_check(cudaMemcpyAsync(hs.data(), ost.p, kNumOrder * 8, cudaMemcpyDeviceToHost, s.stream), "class starts");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return fail(st);
  for (int c = 0; c < kNumClasses; ++c) s.class_start[c] = hs[(size_t)c * kHotBuckets];
  s.class_start[kNumClasses] = n;
  s.n_alive = s.class_start[kClassDead];
  if (st.ok()) st = ensure(s, s.p2o, std::max<uint64_t>(1, n) * 4);
  if (st.ok()) st = ensure(s, s.o2p, std::max<uint64_t>(1, n) * 4);
  if (st.ok()) st = ensure(s, s.offsets, (n + 1) * 8);
  if (st.ok()) st = ensure(s, s.nlabel, std::max<uint64_t>(1, n) * 4);
  if (st.ok()) st = ensure(s, s.dst, std::max<uint64_t>(1, m) * 4);
  if (!st.ok()) return fail(st);
  const unsigned gb = (unsigned)std::min<uint64_t>(grid_for(n, 256), (uint64_t)sms * 32);
  if (n) {
    k_class_tile_scatter<<<(unsigned)ntiles, kClassTile, 0, s.stream>>>(n, off0, alive0, ptr<uint32_t>(hot), ntiles,
                                                                        ptr<unsigned long long>(tcnt),
                                                                        ptr<uint32_t>(s.p2o));
    k_invert<<<gb, 256, 0, s.stream>>>(n, ptr<uint32_t>(s.p2o), ptr<uint32_t>(s.o2p));
  }
  k_relabel_nodes<<<gb, 256, 0, s.stream>>>(n, ptr<uint32_t>(s.p2o), off0, nlab0,
                                            ptr<unsigned long long>(s.offsets), ptr<uint32_t>(s.nlabel));
  st = launch_check("relabel nodes");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  fail(Status::Ok());  // the class scatter has finished with the tile bases and counts
  if (!st.ok()) return st;
  if (!(st = scan64(s, ptr<uint64_t>(s.offsets), n + 1, nullptr)).ok()) return st;
  s.n_alone = 0;
  MidPlan mp;
  if (!(st = chunk_lists_hubs(s, true, &mp)).ok()) return st;
  // the edge labels (and with them the label width) from here on
  if (s.await_labels && !(st = s.await_labels(s)).ok()) return st;
  if (!(st = ensure(s, s.elabel, std::max<uint64_t>(1, m) * (s.label8 ? 1 : 4))).ok()) return st;
  if (n && m) {
    if (s.label8) {
      uint8_t* lab = ptr<uint8_t>(s.elabel);
      if (lab_bytes == 1) relabel_edges(s, off0, dst0, static_cast<const uint8_t*>(lab0), lab, sms);
      else if (lab_bytes == 2) relabel_edges(s, off0, dst0, static_cast<const uint16_t*>(lab0), lab, sms);
      else relabel_edges(s, off0, dst0, static_cast<const uint32_t*>(lab0), lab, sms);
    } else {
      uint32_t* lab = ptr<uint32_t>(s.elabel);
      if (lab_bytes == 2) relabel_edges(s, off0, dst0, static_cast<const uint16_t*>(lab0), lab, sms);
      else relabel_edges(s, off0, dst0, static_cast<const uint32_t*>(lab0), lab, sms);
    }
  }
  st = launch_check("relabel edges");
  // the medium chunk plan on the host while the GPU relabels the edges
  if (st.ok()) st = chunk_lists_mid(s, mp);
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  return st;
}

// ---- level 0 when few labels occur (Definition 2: pId_0 groups nodes by
// label) ------------------------------------------------------------------
// A table of kL0Slots 64-bit slots (label << 32 | smallest original id) and a
// node count per slot.  Each CTA first gathers the labels of its node range in
// a shared copy, so the global table sees one update per label per CTA.  If a
// shared or the global table fills (more labels than it holds) the general
// path (hash, grouping, exact check, renumbering) computes the level instead.
constexpr int kL0Slots = 4096;        // global table: labels at most kL0Slots / 2
constexpr int kL0SmemSlots = 1024;    // per CTA
constexpr int kL0Threads = 256;
constexpr unsigned long long kL0Empty = ~0ull;  // (0xFFFFFFFF, 0xFFFFFFFF): no original id is 0xFFFFFFFF

__device__ __forceinline__ uint32_t l0_home(uint32_t label, uint32_t mask) {
  return (label * 0x9E3779B1u >> 7) & mask;  // Fibonacci hashing, then the slot bits
}

// Insert (label, id) into a table of 64-bit slots: the slot of the label keeps
// the smallest id; returns the slot, or -1 if the table is full (shared or
// global memory, through generic addressing).
__device__ __forceinline__ int l0_insert(unsigned long long* tab, uint32_t mask, uint32_t label, uint32_t id) {
  const unsigned long long v = ((unsigned long long)label << 32) | id;
  uint32_t at = l0_home(label, mask);
  for (uint32_t t = 0; t <= mask; ++t) {
    const unsigned long long cur = atomicCAS(tab + at, kL0Empty, v);
    if (cur == kL0Empty) return (int)at;
    if ((uint32_t)(cur >> 32) == label) {
      if ((uint32_t)cur > id) atomicMin(tab + at, v);
      return (int)at;
    }
    at = (at + 1) & mask;
  }
  return -1;
}

__global__ void __launch_bounds__(kL0Threads) k_l0_collect(uint64_t n_alive, const uint32_t* nlabel, const uint32_t* p2o,
                                                           unsigned long long* gtab, uint32_t* gcnt, uint32_t* err) {
  __shared__ unsigned long long tab[kL0SmemSlots];
  __shared__ uint32_t cnt[kL0SmemSlots];
  __shared__ uint32_t full;
  for (uint32_t i = threadIdx.x; i < (uint32_t)kL0SmemSlots; i += kL0Threads) {
    tab[i] = kL0Empty;
    cnt[i] = 0;
  }
  if (threadIdx.x == 0) full = 0;
  __syncthreads();
  const uint64_t per = (n_alive + gridDim.x - 1) / gridDim.x;
  const uint64_t lo0 = (uint64_t)blockIdx.x * per;
  const uint64_t lo = lo0 < n_alive ? lo0 : n_alive, hi = lo + per < n_alive ? lo + per : n_alive;
  for (uint64_t p = lo + threadIdx.x; p < hi; p += kL0Threads) {
    const int at = l0_insert(tab, kL0SmemSlots - 1, nlabel[p], p2o[p]);
    if (at < 0) full = 1;
    else atomicAdd(&cnt[at], 1u);
  }
  __syncthreads();
  if (full) {
    if (threadIdx.x == 0) atomicOr(err, 1u);
    return;
  }
  for (uint32_t i = threadIdx.x; i < (uint32_t)kL0SmemSlots; i += kL0Threads) {
    const unsigned long long v = tab[i];
    if (v == kL0Empty) continue;
    const int at = l0_insert(gtab, kL0Slots - 1, (uint32_t)(v >> 32), (uint32_t)v);
    if (at < 0) atomicOr(err, 1u);
    else atomicAdd(&gcnt[at], cnt[i]);
  }
}

// pId_0 of every node from the ranked table: rank[slot] = block id, and the
// node is alone in its block when its label's count is 1.
__global__ void __launch_bounds__(kL0Threads) k_l0_fill(uint64_t n, uint64_t n_alive, const uint32_t* nlabel,
                                                        const unsigned long long* gtab, const uint32_t* rank,
                                                        const uint32_t* gcnt, uint32_t* pid, uint8_t* alone) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
    if (p >= n_alive) {
      pid[p] = kDead;
      continue;
    }
    const uint32_t label = nlabel[p];
    uint32_t at = l0_home(label, kL0Slots - 1);
    for (uint32_t t = 0; t < (uint32_t)kL0Slots; ++t) {  // the label is in the table: the loop ends at its slot
      const unsigned long long v = __ldg(gtab + at);
      if (v != kL0Empty && (uint32_t)(v >> 32) == label) break;
      at = (at + 1) & (kL0Slots - 1);
    }
    pid[p] = __ldg(rank + at);
    alone[p] = __ldg(gcnt + at) == 1u ? 1 : 0;
  }
}

// Level 0 by the label table; *done = false when there are too many labels
// (the general path then runs).
Status level0_few_labels(Store& s, bool* done) {
  *done = false;
  const uint64_t n = s.n, na = s.n_alive;
  if (!na) return Status::Ok();
  Status st;
  // the table, counts and ranks in the grouping table's buffer (sized for n
  // nodes, so large enough whenever there are nodes)
  const size_t bytes = kL0Slots * 8 + kL0Slots * 4 + kL0Slots * 4 + 16;
  if (s.table.cap < bytes) return Status::Ok();
  unsigned long long* gtab = ptr<unsigned long long>(s.table);
  uint32_t* gcnt = reinterpret_cast<uint32_t*>(gtab + kL0Slots);
  uint32_t* grank = gcnt + kL0Slots;
  uint32_t* err = grank + kL0Slots;
  const int sms = sm_count(s.device);
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  {
    TimedScope ts(s, KBISIM_KERNEL_LABEL_GROUP, 1);
    cudaMemsetAsync(gtab, 0xFF, kL0Slots * 8, s.stream);
    cudaMemsetAsync(gcnt, 0, kL0Slots * 4 * 2 + 16, s.stream);
    const unsigned g = (unsigned)std::min<uint64_t>(grid_for(na, 2048), (uint64_t)sms * 8);
    k_l0_collect<<<g, kL0Threads, 0, s.stream>>>(na, ptr<uint32_t>(s.nlabel), ptr<uint32_t>(s.p2o), gtab, gcnt, err);
  }
  if (!(st = launch_check("k_l0_collect")).ok()) return st;
  std::vector<unsigned long long> tab(kL0Slots);
  std::vector<uint32_t> cnt(kL0Slots + 1);
  st = cuda_check(cudaMemcpyAsync(tab.data(), gtab, kL0Slots * 8, cudaMemcpyDeviceToHost, s.stream), "level 0");
  if (st.ok())
    st = cuda_check(cudaMemcpyAsync(cnt.data(), gcnt, kL0Slots * 4, cudaMemcpyDeviceToHost, s.stream), "level 0");
  if (st.ok()) st = cuda_check(cudaMemcpyAsync(&cnt[kL0Slots], err, 4, cudaMemcpyDeviceToHost, s.stream), "level 0");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok() || cnt[kL0Slots]) return st;  // too many labels: the general path
  // blocks ranked by their smallest original id
  std::vector<std::pair<uint32_t, uint32_t>> heads;  // (smallest id, slot)
  uint64_t alone = 0;
  for (uint32_t i = 0; i < (uint32_t)kL0Slots; ++i)
    if (tab[i] != kL0Empty) {
      heads.push_back({(uint32_t)tab[i], i});
      alone += cnt[i] == 1 ? 1 : 0;
    }
  if (heads.size() > (size_t)kL0Slots / 2) return Status::Ok();  // long probe runs: the general path
  std::sort(heads.begin(), heads.end());
  std::vector<uint32_t> rank(kL0Slots, 0);
  for (size_t r = 0; r < heads.size(); ++r) rank[heads[r].second] = (uint32_t)r;
  st = cuda_check(cudaMemcpyAsync(grank, rank.data(), kL0Slots * 4, cudaMemcpyHostToDevice, s.stream), "level 0");
  if (!st.ok()) return st;
  {
    TimedScope ts(s, KBISIM_KERNEL_RENUMBER, 1);
    const unsigned g = (unsigned)std::min<uint64_t>(grid_for(n, kL0Threads), (uint64_t)sms * 16);
    k_l0_fill<<<g, kL0Threads, 0, s.stream>>>(n, na, ptr<uint32_t>(s.nlabel), gtab, grank, gcnt,
                                             ptr<uint32_t>(s.level[0]), ptr<uint8_t>(s.alone));
  }
  if (!(st = launch_check("k_l0_fill")).ok()) return st;
  if (s.checked && !(st = check_below(s, ptr<uint32_t>(s.level[0]), na, heads.size(), "identifiers")).ok())
    return st;
  s.counts[0] = heads.size();
  s.n_alone = alone;
  *done = true;
  return Status::Ok();
}

Status compute_level0(Store& s) {
  Status st = ensure_round_scratch(s);
  if (!st.ok()) return st;
  bool done = false;
  if (!(st = level0_few_labels(s, &done)).ok()) return st;
  if (done) return Status::Ok();
  const int sms = sm_count(s.device);
  const unsigned blocks = (unsigned)std::min<uint64_t>(grid_for(s.n_alive, 256), (uint64_t)sms * 16);
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  {
    TimedScope ts(s, KBISIM_KERNEL_LABEL_GROUP, s.n_alive ? 1 : 0);
    if (s.n_alive)
      k_label_hash<<<blocks, 256, 0, s.stream>>>(s.n_alive, ptr<uint32_t>(s.nlabel), ptr<uint64_t>(s.hash),
                                                 s.seed, s.hash_mask);
  }
  if (!(st = launch_check("k_label_hash")).ok()) return st;
  uint64_t blocks_out = 0, coll = 0;
  st = group_and_rank(s, 0, nullptr, false, ptr<uint32_t>(s.level[0]), &blocks_out, &coll, false, nullptr,
                      nullptr, false);
  if (!st.ok()) return st;
  s.counts[0] = blocks_out;
  return Status::Ok();
}

// Checked mode, before a round: the edge table's offsets and targets and the
// previous level's identifiers (the indices and the packed values of the
// signature kernels).  With the KBISIM_FAULT_CORRUPT_DST test hook one target
// is set to n first (and put back after the check reports it).
Status check_round_inputs(Store& s, uint32_t i) {
  Status st;
  uint32_t saved = 0;
  const uint64_t at = s.m / 2;
  uint32_t* dst = ptr<uint32_t>(s.dst);
  if (s.fault_corrupt_dst && s.m) {
    const uint32_t bad = (uint32_t)s.n;
    st = cuda_check(cudaMemcpyAsync(&saved, dst + at, 4, cudaMemcpyDeviceToHost, s.stream), "corrupt");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "corrupt");
    if (st.ok()) st = cuda_check(cudaMemcpyAsync(dst + at, &bad, 4, cudaMemcpyHostToDevice, s.stream), "corrupt");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "corrupt");
    if (!st.ok()) return st;
  }
  if (s.n) {
    const unsigned g = (unsigned)std::min<uint64_t>(grid_for(s.n, 256), (uint64_t)sm_count(s.device) * 16);
    k_check_offsets_mono<<<g, 256, 0, s.stream>>>(ptr<uint64_t>(s.offsets), s.n, s.m, ptr<uint32_t>(s.d_err));
    st = checked_outcome(s, "edge offsets");
  }
  if (st.ok()) st = check_below(s, dst, s.m, s.n, "edge targets");
  if (s.fault_corrupt_dst && s.m) {
    Status st2 = cuda_check(cudaMemcpyAsync(dst + at, &saved, 4, cudaMemcpyHostToDevice, s.stream), "restore");
    if (st2.ok()) st2 = cuda_check(cudaStreamSynchronize(s.stream), "restore");
    if (!st2.ok()) return st2;
  }
  if (st.ok()) st = check_below(s, ptr<uint32_t>(s.level[i - 1]), s.n_alive, s.counts[i - 1], "previous level");
  return st;
}

Status compute_round(Store& s, uint32_t i) {
  if (s.fault_timeout_round && i == s.fault_timeout_round)
    return Status::Err(KBISIM_ERR_TIMEOUT, "injected timeout (KBISIM_FAULT_TIMEOUT_ROUND)");
  Status st = ensure_round_scratch(s);
  if (!st.ok()) return st;
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  if (s.checked && !(st = check_round_inputs(s, i)).ok()) return st;
  SigArgs a;
  a.off = ptr<uint64_t>(s.offsets);
  a.dst = ptr<uint32_t>(s.dst);
  a.lab = s.elabel.p;
  a.prev = ptr<uint32_t>(s.level[i - 1]);
  a.sigkey = s.sigkey.p;
  a.ucnt = ptr<uint32_t>(s.ucnt);
  a.hash = ptr<uint64_t>(s.hash);
  a.seed = s.seed;
  a.mask = s.hash_mask;
  a.err = ptr<uint32_t>(s.d_err);
  a.fmask = s.round_mask;
  // 32-bit signature words when (label, child id) fits in 32 bits
  const uint32_t pbits = bits_for(s.counts[i - 1] ? s.counts[i - 1] - 1 : 0);
  const bool key64 = pbits + s.label_bits > 32;
  a.pbits = (int)pbits;
  s.tune_now = s.hub_tune == 1 && i >= 2 && !s.round_mask && s.n_hub;
  if (s.label8)
    st = key64 ? run_signatures<uint8_t, uint64_t>(s, a) : run_signatures<uint8_t, uint32_t>(s, a);
  else
    st = key64 ? run_signatures<uint32_t, uint64_t>(s, a) : run_signatures<uint32_t, uint32_t>(s, a);
  s.tune_now = false;
  if (!st.ok()) return st;
  if (s.round_mask && s.n_alive) {
    const int sms = sm_count(s.device);
    k_freeze<<<(unsigned)std::min<uint64_t>(grid_for(s.n_alive, 256), (uint64_t)sms * 16), 256, 0, s.stream>>>(
        s.n_alive, s.round_mask, a.prev, a.ucnt, a.hash, s.seed, s.hash_mask);
    if (!(st = launch_check("k_freeze")).ok()) return st;
  }
  uint64_t blocks = 0, coll = 0, keys = 0, maxsig = 0;
  // nodes alone in their block at level i-1 stay alone (Proposition 1): they
  // are heads of level i without a table lookup
  st = group_and_rank(s, 1, a.prev, key64, ptr<uint32_t>(s.level[i]), &blocks, &coll, true, &keys, &maxsig, true);
  if (!st.ok()) return st;
  s.counts[i] = blocks;
  kbisim_round_stats rs;
  rs.blocks = blocks;
  rs.unique_keys = keys;
  rs.max_signature = maxsig;
  rs.collided_nodes = coll;
  rs.hub_nodes = s.n_hub;
  if (s.stats.size() < i) s.stats.resize(i);
  s.stats[i - 1] = rs;
  return Status::Ok();
}

Status masked_signatures(Store& s, const uint32_t* prev, const uint32_t* fmask) {
  Status st = ensure_round_scratch(s);
  if (!st.ok()) return st;
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  SigArgs a;
  a.off = ptr<uint64_t>(s.offsets);
  a.dst = ptr<uint32_t>(s.dst);
  a.lab = s.elabel.p;
  a.prev = prev;
  a.sigkey = s.sigkey.p;
  a.ucnt = ptr<uint32_t>(s.ucnt);
  a.hash = ptr<uint64_t>(s.hash);
  a.seed = s.seed;
  a.mask = s.hash_mask;
  a.err = ptr<uint32_t>(s.d_err);
  a.fmask = fmask;
  if (s.mt.key32) {  // labels below 2^pbits (the stores' width)
    a.pbits = (int)s.mt.pbits;
    return s.label8 ? run_signatures<uint8_t, uint32_t>(s, a) : run_signatures<uint32_t, uint32_t>(s, a);
  }
  a.pbits = 32;
  return s.label8 ? run_signatures<uint8_t, uint64_t>(s, a) : run_signatures<uint32_t, uint64_t>(s, a);
}

Status group_list(Store& s, const uint32_t* list, uint64_t count, const uint32_t* prev) {
  Status st = ensure_round_scratch(s);
  if (!st.ok() || !count) return st;
  unsigned long long* sc = ptr<unsigned long long>(s.d_scalars);
  GroupArgs g;
  g.hash = ptr<uint64_t>(s.hash);
  g.p2o = ptr<uint32_t>(s.p2o);
  g.o2p = ptr<uint32_t>(s.o2p);
  g.table = ptr<unsigned long long>(s.table);
  g.slot = ptr<uint32_t>(s.slot);
  g.rep = ptr<uint32_t>(s.rep);
  g.err = ptr<uint32_t>(s.d_err);
  g.alone = nullptr;
  g.read_first = 0;
  VerifyArgs v;
  v.mode = 1;
  v.key64 = s.mt.key32 ? 0 : 1;
  v.nlabel = ptr<uint32_t>(s.nlabel);
  v.prev = prev;
  v.ucnt = ptr<uint32_t>(s.ucnt);
  v.off = ptr<uint64_t>(s.offsets);
  v.sigkey = s.sigkey.p;
  v.n_collided = sc + 4;
  v.long_list = ptr<uint32_t>(s.long_pairs);
  v.n_long = sc + 6;
  v.hbits = ptr<uint32_t>(s.hbits);  // marks of the canonical numbering: not used here
  v.member = ptr<uint8_t>(s.member);
  v.out_list = ptr<uint32_t>(s.ulist[0]);
  v.n_out = sc + 1;
  const uint64_t tcap = std::min<uint64_t>(s.tcap, table_capacity(count));
  g.tmask = tcap - 1;
  const int sms = sm_count(s.device);
  cudaMemsetAsync(s.d_scalars.p, 0, 15 * 8, s.stream);
  cudaMemsetAsync(s.table.p, 0xFF, tcap * 8, s.stream);
  {
    TimedScope ts(s, KBISIM_KERNEL_GROUP, 2);
    k_group_insert<<<(unsigned)std::min<uint64_t>((count + kInsChunk - 1) / kInsChunk,
                                                  resident_blocks(k_group_insert, kInsThreads, 0, sms)),
                     kInsThreads, 0, s.stream>>>(g, list, count);
    k_group_verify<<<(unsigned)std::min<uint64_t>(grid_for(count, kVerTile),
                                                  resident_blocks(k_group_verify, kVerNodeThreads, 0, sms)),
                     kVerNodeThreads, 0, s.stream>>>(g, v, list, count);
  }
  if (!(st = launch_check("group list")).ok()) return st;
  uint64_t h[16];
  if (!(st = read_scalars(s, h)).ok()) return st;
  if (!(st = settle_unresolved(s, g, v, true, h, KBISIM_KERNEL_VERIFY)).ok()) return st;
  uint32_t e = 0;
  st = cuda_check(cudaMemcpyAsync(&e, s.d_err.p, 4, cudaMemcpyDeviceToHost, s.stream), "group list");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "group list");
  if (st.ok() && (e & kErrProbe)) return Status::Err(KBISIM_ERR_TIMEOUT, "hash table probe bound exceeded");
  return st;
}

Status unpermute_level(Store& s, uint32_t level, uint32_t* dst) {
  if (!s.n) return Status::Ok();
  const int sms = sm_count(s.device);
  const unsigned gb = (unsigned)std::min<uint64_t>(grid_for(s.n, 256), (uint64_t)sms * 16);
  k_unpermute<<<gb, 256, 0, s.stream>>>(s.n, ptr<uint32_t>(s.o2p), ptr<uint32_t>(s.level[level]), dst);
  return launch_check("k_unpermute");
}

}  // namespace kb
