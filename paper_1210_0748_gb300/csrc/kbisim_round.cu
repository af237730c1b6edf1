// One refinement round of k-bisimulation on the GPU, and level 0.
//
// Round i (Algorithm 1, the k > 0 branch; Definition 3; Proposition 2):
//   (a) gather: for every edge e = (u, l, v) of the source-sorted edge table,
//       the element key (l, pId_{i-1}(v))          -- Algorithm 1 "fill in
//       pId_old(tId)" (the merge join ET x NT), done as a direct gather;
//   (b) per source node: sort the keys and drop duplicates (the sorted,
//       duplicate-free F of Algorithm 1), written at the node's CSR offset;
//   (c) a 64-bit hash of (pId_{i-1}(u), the key set)  -- stands in for the
//       signature store S (Section 3, "Data structures for S");
//   (d) group nodes with equal hash in an open-addressing table that keeps
//       the smallest node id per hash, compare every node's signature with
//       that node's exactly (so a hash collision never merges two blocks),
//       repair collisions, and number blocks by their smallest node id;
//   (e) the caller stops when the block count is unchanged.
// Level 0 groups nodes by label the same way (Algorithm 1, k = 0 branch).
//
// Signature keys are compared through a fixed bijection (elem_key), and each
// node's set is stored in ascending order of that bijection: any fixed order
// is a canonical form for sets (the paper keeps sets as sorted strings,
// Section 3.2); this one spreads values uniformly, which balances the
// bucketed sorts.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kbisim_internal.cuh"

namespace kb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// --------------------------------------------------------------------------
// Kernel timing
// --------------------------------------------------------------------------
}  // namespace

struct KernelTimer {
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> open;
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

Status timer_begin(Store& s, int cls) {
  s.launches[cls] += 1;
  if (!s.timing) return Status::Ok();
  if (!s.timer) s.timer = new KernelTimer();
  KernelTimer::Rec r;
  r.cls = cls;
  r.a = s.timer->get();
  r.b = s.timer->get();
  cudaEventRecord(r.a, s.stream);
  s.timer->open.push_back(r);
  return Status::Ok();
}

Status timer_end(Store& s, int cls) {
  if (!s.timing || !s.timer) return Status::Ok();
  for (size_t i = s.timer->open.size(); i-- > 0;) {
    if (s.timer->open[i].cls == cls) {
      KernelTimer::Rec r = s.timer->open[i];
      cudaEventRecord(r.b, s.stream);
      s.timer->done.push_back(r);
      s.timer->open.erase(s.timer->open.begin() + i);
      break;
    }
  }
  return Status::Ok();
}

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
  for (auto& r : s.timer->open) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto& r : s.timer->done) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  delete s.timer;
  s.timer = nullptr;
}

namespace {

struct TimedScope {
  Store& s;
  int cls;
  TimedScope(Store& st, int c) : s(st), cls(c) { timer_begin(s, c); }
  ~TimedScope() { timer_end(s, cls); }
};

template <typename T>
T* ptr(Buf& b) { return static_cast<T*>(b.p); }

inline unsigned grid_for(uint64_t work, unsigned per_block) {
  uint64_t g = (work + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, 0x7FFFFFFFull));
}

// --------------------------------------------------------------------------
// Team helpers: a "team" is one warp (NT = 32) or one CTA (NT = blockDim).
// --------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void team_sync() {
  if (NT == 32) __syncwarp(); else __syncthreads();
}

// Exclusive prefix sum of a[0..n) in shared memory by a team of NT threads.
// warp_tot: NT/32 words of shared scratch (unused for NT == 32).
template <int NT>
__device__ void team_excl_scan(uint32_t* a, int n, uint32_t* warp_tot, int rank) {
  const int per = (n + NT - 1) / NT;
  const int lo = min(rank * per, n), hi = min(lo + per, n);
  uint32_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += a[i];
  const int lane = rank & 31;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  uint32_t excl = x - sum;
  if (NT > 32) {
    const int w = rank >> 5;
    if (lane == 31) warp_tot[w] = x;
    team_sync<NT>();
    if (w == 0) {
      uint32_t t = lane < NT / 32 ? warp_tot[lane] : 0;
      uint32_t xx = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, xx, o);
        if (lane >= o) xx += y;
      }
      if (lane < NT / 32) warp_tot[lane] = xx - t;
    }
    team_sync<NT>();
    excl += warp_tot[w];
  }
  uint32_t run = excl;
  for (int i = lo; i < hi; ++i) {
    uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  team_sync<NT>();
}

// Shared-memory layout of one team's dedupe-and-sort workspace.
struct TeamWs {
  uint64_t* set;    // [hcap] hash set, reused as the sorted output
  uint64_t* uniq;   // [ucap] distinct keys in arrival order
  uint64_t* bitv;   // [2] OR and AND of the distinct keys
  uint64_t* red;    // [NT/32] reduction scratch
  uint32_t* cnt;    // [ucap/2] bucket counters
  uint32_t* sh;     // [4] distinct count, saw-empty-key flag, overflow flag
  uint32_t* wtot;   // [NT/32]
  int hcap, ucap;
};

__host__ __device__ constexpr size_t team_ws_bytes(int hcap, int ucap, int nt) {
  return ((size_t)hcap * 8 + (size_t)ucap * 8 + 16 + (size_t)(nt / 32) * 8 + (size_t)(ucap / 2) * 4 +
          16 + (size_t)(nt / 32) * 4 + 15) / 16 * 16;
}

__device__ __forceinline__ TeamWs carve(char* base, int hcap, int ucap, int nt) {
  TeamWs ws;
  ws.set = reinterpret_cast<uint64_t*>(base);
  ws.uniq = ws.set + hcap;
  ws.bitv = ws.uniq + ucap;
  ws.red = ws.bitv + 2;
  ws.cnt = reinterpret_cast<uint32_t*>(ws.red + nt / 32);
  ws.sh = ws.cnt + ucap / 2;
  ws.wtot = ws.sh + 4;
  ws.hcap = hcap;
  ws.ucap = ucap;
  return ws;
}

// Smallest power of two >= 2 n, clamped to [64, cap].
__device__ __forceinline__ int set_size_for(uint64_t n, int cap) {
  int h = 64;
  while (h < cap && (uint64_t)h < 2 * n) h <<= 1;
  return h;
}

// Distinct keys of n inputs, sorted ascending into ws.set[0..U).  Returns U,
// or 0xFFFFFFFF if more than ucap distinct keys arrived (overflow).
// Dedupe: open-addressing set of `hcap` slots in shared memory (keys are
// uniformly mixed, so their low bits index it).  Sort: counting sort into
// about U/2 buckets on the highest bits in which the distinct keys differ
// (keys that share a prefix -- e.g. one hub bucket -- still spread out),
// then insertion sort inside each (tiny) bucket.
template <int NT, class GetKey>
__device__ uint32_t team_dedupe_sort(const TeamWs& ws, int hcap, uint64_t n, GetKey get, int rank) {
  for (int i = rank; i < hcap; i += NT) ws.set[i] = kEmpty64;
  if (rank < 4) ws.sh[rank] = 0;
  if (rank == 0) {
    ws.bitv[0] = 0ull;
    ws.bitv[1] = ~0ull;
  }
  team_sync<NT>();
  volatile uint64_t* vset = ws.set;
  const uint32_t hmask = (uint32_t)(hcap - 1);
  for (uint64_t i = rank; i < n; i += NT) {
    const uint64_t k = get(i);
    bool fresh = false;
    if (k == kEmpty64) {
      fresh = atomicExch(&ws.sh[1], 1u) == 0u;
    } else {
      uint32_t s = (uint32_t)k & hmask;
      int t = 0;
      for (; t < hcap; ++t) {
        uint64_t cur = vset[s];
        if (cur == k) break;
        if (cur == kEmpty64) {
          uint64_t old = atomicCAS((unsigned long long*)&ws.set[s], (unsigned long long)kEmpty64,
                                   (unsigned long long)k);
          if (old == kEmpty64) { fresh = true; break; }
          if (old == k) break;
        }
        s = (s + 1) & hmask;
      }
      if (t == hcap) ws.sh[2] = 1u;
    }
    if (fresh) {
      uint32_t idx = atomicAdd(&ws.sh[0], 1u);
      if (idx < (uint32_t)ws.ucap) ws.uniq[idx] = k; else ws.sh[2] = 1u;
      atomicOr((unsigned long long*)&ws.bitv[0], (unsigned long long)k);
      atomicAnd((unsigned long long*)&ws.bitv[1], (unsigned long long)k);
    }
  }
  team_sync<NT>();
  if (ws.sh[2]) return 0xFFFFFFFFu;
  const uint32_t U = ws.sh[0];
  int bits = 0;
  while ((2u << bits) < U) ++bits;  // NB = 2^bits ~ U/2
  if (U <= 2) bits = 0;
  const int NB = 1 << bits;
  const uint64_t diff = ws.bitv[0] ^ ws.bitv[1];
  const int top = diff ? 63 - __clzll((long long)diff) : 0;  // highest differing bit
  const int shift = (top + 1 >= bits) ? top + 1 - bits : 0;
  const uint64_t bmask = (uint64_t)(NB - 1);
  for (int b = rank; b < NB; b += NT) ws.cnt[b] = 0;
  team_sync<NT>();
  for (uint32_t i = rank; i < U; i += NT) atomicAdd(&ws.cnt[(ws.uniq[i] >> shift) & bmask], 1u);
  team_sync<NT>();
  team_excl_scan<NT>(ws.cnt, NB, ws.wtot, rank);
  for (uint32_t i = rank; i < U; i += NT) {
    const uint64_t k = ws.uniq[i];
    const uint32_t p = atomicAdd(&ws.cnt[(k >> shift) & bmask], 1u);
    ws.set[p] = k;
  }
  team_sync<NT>();
  for (int b = rank; b < NB; b += NT) {
    const uint32_t lo = b ? ws.cnt[b - 1] : 0u, hi = ws.cnt[b];
    for (uint32_t i = lo + 1; i < hi; ++i) {
      uint64_t v = ws.set[i];
      uint32_t j = i;
      while (j > lo && ws.set[j - 1] > v) {
        ws.set[j] = ws.set[j - 1];
        --j;
      }
      ws.set[j] = v;
    }
  }
  team_sync<NT>();
  return U;
}

// Sum of elem_term over ws.set[0..U) across the team (result valid in all lanes
// of the team for NT == 32, in rank 0 for NT > 32).
template <int NT>
__device__ uint64_t team_term_sum(const uint64_t* keys, uint32_t U, uint64_t seed,
                                  uint64_t* red, int rank) {
  uint64_t t = 0;
  for (uint32_t i = rank; i < U; i += NT) t += elem_term(keys[i], seed);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
  if (NT == 32) return t;
  if ((rank & 31) == 0) red[rank >> 5] = t;
  __syncthreads();
  uint64_t tot = 0;
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
  uint64_t* sigkey;
  uint32_t* ucnt;
  uint64_t* hash;
  uint64_t seed;
  uint64_t mask;
  uint32_t* err;
};

template <typename LabelT>
__device__ __forceinline__ uint64_t edge_key(const SigArgs& a, uint64_t e) {
  const LabelT* lab = static_cast<const LabelT*>(a.lab);
  return elem_key((uint32_t)lab[e], a.prev[a.dst[e]]);
}

// Out-degree <= 32: P = 2^c lanes per node (32/P nodes per warp).  Keys are
// sorted by a bitonic network across the P lanes, duplicates dropped by
// comparing with the previous lane, survivors compacted with a ballot.
template <int P, typename LabelT>
__device__ void sig_small_body(const SigArgs& a, const uint32_t* nodes, uint64_t count,
                               uint64_t warp_idx) {
  const int lane = threadIdx.x & 31;
  const int g = lane / P, j = lane % P;
  const uint64_t idx = warp_idx * (32 / P) + g;
  const bool active = idx < count;
  uint32_t u = 0;
  uint64_t off = 0;
  uint32_t d = 0;
  if (active) {
    u = nodes[idx];
    off = a.off[u];
    d = (uint32_t)(a.off[u + 1] - off);
  }
  uint64_t key = kEmpty64;
  if (j < (int)d) key = edge_key<LabelT>(a, off + j);
#pragma unroll
  for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
    for (int s = k >> 1; s > 0; s >>= 1) {
      uint64_t other = __shfl_xor_sync(kFull, key, s);
      bool up = (j & k) == 0;
      bool lower = (j & s) == 0;
      key = (lower == up) ? min(key, other) : max(key, other);
    }
  }
  uint64_t prevk = __shfl_up_sync(kFull, key, 1);
  const bool uniq = (j < (int)d) && (j == 0 || key != prevk);
  const unsigned bal = __ballot_sync(kFull, uniq);
  const unsigned gmask = (P == 32) ? bal : ((bal >> (g * P)) & ((1u << (P & 31)) - 1u));
  const int pos = __popc(gmask & ((1u << j) - 1u));
  if (uniq) a.sigkey[off + pos] = key;
  uint64_t t = uniq ? elem_term(key, a.seed) : 0ull;
#pragma unroll
  for (int s = P >> 1; s > 0; s >>= 1) t += __shfl_xor_sync(kFull, t, s);
  if (active && j == 0) {
    const uint32_t U = (uint32_t)__popc(gmask);
    a.ucnt[u] = U;
    a.hash[u] = node_hash(t, a.prev[u], U, a.seed, a.mask);
  }
}

struct SmallLaunch {
  uint64_t start[kSmallClasses];   // first index of class c in the node list
  uint64_t count[kSmallClasses];
  uint32_t bstart[kSmallClasses + 1];  // first block of class c
};

constexpr int kSmallWarps = 8;

template <typename LabelT>
__global__ void __launch_bounds__(256) k_sig_small(SigArgs a, const uint32_t* nodes, SmallLaunch L) {
  int c = 0;
  while (c + 1 < kSmallClasses && blockIdx.x >= L.bstart[c + 1]) ++c;
  const uint64_t warp_idx = (uint64_t)(blockIdx.x - L.bstart[c]) * kSmallWarps + (threadIdx.x >> 5);
  const uint32_t* list = nodes + L.start[c];
  switch (c) {
    case 0: sig_small_body<1, LabelT>(a, list, L.count[0], warp_idx); break;
    case 1: sig_small_body<2, LabelT>(a, list, L.count[1], warp_idx); break;
    case 2: sig_small_body<4, LabelT>(a, list, L.count[2], warp_idx); break;
    case 3: sig_small_body<8, LabelT>(a, list, L.count[3], warp_idx); break;
    case 4: sig_small_body<16, LabelT>(a, list, L.count[4], warp_idx); break;
    default: sig_small_body<32, LabelT>(a, list, L.count[5], warp_idx); break;
  }
}

// Out-degree 33..kWarpMax: one warp per node, shared-memory dedupe + sort.
constexpr int kWarpHcap = 2 * kWarpMax;
constexpr int kWarpUcap = kWarpMax;
constexpr int kWarpsPerBlock = 8;
constexpr size_t kWarpWsBytes = team_ws_bytes(kWarpHcap, kWarpUcap, 32);

template <typename LabelT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_sig_warp(SigArgs a, const uint32_t* nodes, uint64_t count) {
  extern __shared__ __align__(16) char smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TeamWs ws = carve(smem + w * kWarpWsBytes, kWarpHcap, kWarpUcap, 32);
  for (uint64_t idx = (uint64_t)blockIdx.x * kWarpsPerBlock + w; idx < count;
       idx += (uint64_t)gridDim.x * kWarpsPerBlock) {
    const uint32_t u = nodes[idx];
    const uint64_t off = a.off[u];
    const uint64_t d = a.off[u + 1] - off;
    auto get = [&](uint64_t i) { return edge_key<LabelT>(a, off + i); };
    const uint32_t U = team_dedupe_sort<32>(ws, set_size_for(d, kWarpHcap), d, get, lane);
    if (U == 0xFFFFFFFFu) {  // cannot happen: at most d <= ucap distinct keys
      if (lane == 0) atomicOr(a.err, kErrHubOverflow);
      continue;
    }
    for (uint32_t i = lane; i < U; i += 32) a.sigkey[off + i] = ws.set[i];
    const uint64_t t = team_term_sum<32>(ws.set, U, a.seed, nullptr, lane);
    if (lane == 0) {
      a.ucnt[u] = U;
      a.hash[u] = node_hash(t, a.prev[u], U, a.seed, a.mask);
    }
    __syncwarp();
  }
}

// Out-degree kWarpMax+1..kBlockMax (one CTA per node) and hub buckets.
constexpr int kBlkHcap = 2 * kBlockMax;
constexpr int kBlkUcap = kBlockMax;
constexpr size_t kBlkWsBytes = team_ws_bytes(kBlkHcap, kBlkUcap, kBlockThreads);

template <typename LabelT>
__global__ void __launch_bounds__(kBlockThreads)
    k_sig_block(SigArgs a, const uint32_t* nodes, uint64_t count) {
  extern __shared__ __align__(16) char smem[];
  TeamWs ws = carve(smem, kBlkHcap, kBlkUcap, kBlockThreads);
  uint64_t* red = ws.red;
  for (uint64_t idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const uint32_t u = nodes[idx];
    const uint64_t off = a.off[u];
    const uint64_t d = a.off[u + 1] - off;
    auto get = [&](uint64_t i) { return edge_key<LabelT>(a, off + i); };
    const uint32_t U = team_dedupe_sort<kBlockThreads>(ws, set_size_for(d, kBlkHcap), d, get, threadIdx.x);
    if (U == 0xFFFFFFFFu) {
      if (threadIdx.x == 0) atomicOr(a.err, kErrHubOverflow);
      __syncthreads();
      continue;
    }
    for (uint32_t i = threadIdx.x; i < U; i += kBlockThreads) a.sigkey[off + i] = ws.set[i];
    const uint64_t t = team_term_sum<kBlockThreads>(ws.set, U, a.seed, red, threadIdx.x);
    if (threadIdx.x == 0) {
      a.ucnt[u] = U;
      a.hash[u] = node_hash(t, a.prev[u], U, a.seed, a.mask);
    }
    __syncthreads();
  }
}

// ---- hubs: out-degree > kBlockMax ----------------------------------------
// Partition each hub's keys by their top bits into buckets expected to hold
// about kHubBucketTarget distinct keys, dedupe + sort each bucket in shared
// memory, then concatenate the buckets in order (the top bits order them).
struct HubArgs {
  const uint32_t* hub_nodes;
  const uint32_t* hub_bits;
  const uint64_t* hub_bbase;
  const uint4* chunks;
  uint32_t extra_bits;
  uint64_t* hist;     // per bucket: count, then (after the scan) start
  uint64_t* cursor;   // per bucket: fill cursor
  uint32_t* bucnt;    // per bucket: distinct keys
  uint64_t* bhpart;   // per bucket: term sum
  uint64_t* tmp;
  uint64_t* tmp2;
};

constexpr int kHubItems = kHubChunk / kBlockThreads;  // 16
constexpr int kHubSmemBuckets = 4096;

__device__ __forceinline__ uint32_t hub_bucket(uint64_t k, uint32_t bits) {
  return bits ? (uint32_t)(k >> (64 - bits)) : 0u;
}

template <typename LabelT>
__global__ void __launch_bounds__(kBlockThreads) k_hub_hist(SigArgs a, HubArgs h) {
  __shared__ uint32_t hist[kHubSmemBuckets];
  const uint4 c = h.chunks[blockIdx.x];
  const uint32_t hub = c.x;
  const uint64_t begin = ((uint64_t)c.z << 32) | c.y;
  const uint32_t len = c.w;
  const uint32_t bits = h.hub_bits[hub] + h.extra_bits;
  const uint32_t nb = 1u << bits;
  const bool in_smem = nb <= kHubSmemBuckets;
  uint64_t* g = h.hist + h.hub_bbase[hub];
  if (in_smem)
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
    const uint32_t b = hub_bucket(edge_key<LabelT>(a, begin + i), bits);
    if (in_smem) atomicAdd(&hist[b], 1u); else atomicAdd((unsigned long long*)&g[b], 1ull);
  }
  __syncthreads();
  if (in_smem)
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
      if (hist[b]) atomicAdd((unsigned long long*)&g[b], (unsigned long long)hist[b]);
}

template <typename LabelT>
__global__ void __launch_bounds__(kBlockThreads) k_hub_scatter(SigArgs a, HubArgs h) {
  __shared__ uint32_t cnt[kHubSmemBuckets];
  __shared__ unsigned long long base[kHubSmemBuckets];
  const uint4 c = h.chunks[blockIdx.x];
  const uint32_t hub = c.x;
  const uint64_t begin = ((uint64_t)c.z << 32) | c.y;
  const uint32_t len = c.w;
  const uint32_t bits = h.hub_bits[hub] + h.extra_bits;
  const uint32_t nb = 1u << bits;
  const bool in_smem = nb <= kHubSmemBuckets;
  uint64_t* cur = h.cursor + h.hub_bbase[hub];
  uint64_t keys[kHubItems];
#pragma unroll
  for (int t = 0; t < kHubItems; ++t) {
    const uint32_t i = threadIdx.x + t * kBlockThreads;
    keys[t] = i < len ? edge_key<LabelT>(a, begin + i) : 0ull;
  }
  if (!in_smem) {
#pragma unroll
    for (int t = 0; t < kHubItems; ++t) {
      const uint32_t i = threadIdx.x + t * kBlockThreads;
      if (i < len) {
        const uint32_t b = hub_bucket(keys[t], bits);
        const uint64_t p = atomicAdd((unsigned long long*)&cur[b], 1ull);
        h.tmp[p] = keys[t];
      }
    }
    return;
  }
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kHubItems; ++t) {
    const uint32_t i = threadIdx.x + t * kBlockThreads;
    if (i < len) atomicAdd(&cnt[hub_bucket(keys[t], bits)], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    if (cnt[b]) base[b] = atomicAdd((unsigned long long*)&cur[b], (unsigned long long)cnt[b]);
    cnt[b] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kHubItems; ++t) {
    const uint32_t i = threadIdx.x + t * kBlockThreads;
    if (i < len) {
      const uint32_t b = hub_bucket(keys[t], bits);
      const uint32_t p = atomicAdd(&cnt[b], 1u);
      h.tmp[base[b] + p] = keys[t];
    }
  }
}

// One CTA per hub bucket: distinct keys of the bucket, sorted, into tmp2.
__global__ void __launch_bounds__(kBlockThreads)
    k_hub_bucket(HubArgs h, uint64_t n_buckets, uint64_t seed, uint32_t* err) {
  extern __shared__ __align__(16) char smem[];
  TeamWs ws = carve(smem, kBlkHcap, kBlkUcap, kBlockThreads);
  uint64_t* red = ws.red;
  for (uint64_t b = blockIdx.x; b < n_buckets; b += gridDim.x) {
    const uint64_t lo = h.hist[b];
    const uint64_t hi = h.cursor[b];  // after the scatter, cursor = end of bucket
    const uint64_t* src = h.tmp + lo;
    auto get = [&](uint64_t i) { return src[i]; };
    const uint32_t U = team_dedupe_sort<kBlockThreads>(ws, set_size_for(hi - lo, kBlkHcap), hi - lo, get,
                                                       threadIdx.x);
    if (U == 0xFFFFFFFFu) {
      if (threadIdx.x == 0) {
        atomicOr(err, kErrHubOverflow);
        h.bucnt[b] = 0;
        h.bhpart[b] = 0;
      }
      __syncthreads();
      continue;
    }
    for (uint32_t i = threadIdx.x; i < U; i += kBlockThreads) h.tmp2[lo + i] = ws.set[i];
    const uint64_t t = team_term_sum<kBlockThreads>(ws.set, U, seed, red, threadIdx.x);
    if (threadIdx.x == 0) {
      h.bucnt[b] = U;
      h.bhpart[b] = t;
    }
    __syncthreads();
  }
}

// One CTA per hub: concatenate its buckets' sorted keys at the hub's CSR offset.
__global__ void __launch_bounds__(kBlockThreads) k_hub_compact(SigArgs a, HubArgs h) {
  __shared__ uint32_t cnt[kBlockThreads];
  __shared__ uint32_t wtot[kBlockThreads / 32];
  __shared__ uint64_t red[kBlockThreads / 32];
  __shared__ unsigned long long running;
  const uint32_t hub = blockIdx.x;
  const uint32_t u = h.hub_nodes[hub];
  const uint64_t off = a.off[u];
  const uint64_t b0 = h.hub_bbase[hub];
  const uint64_t nb = (uint64_t)1 << (h.hub_bits[hub] + h.extra_bits);
  if (threadIdx.x == 0) running = 0;
  uint64_t term = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nb; base += kBlockThreads) {
    const uint64_t b = base + threadIdx.x;
    const uint32_t myc = b < nb ? h.bucnt[b0 + b] : 0u;
    if (b < nb) term += h.bhpart[b0 + b];
    cnt[threadIdx.x] = myc;
    __syncthreads();
    team_excl_scan<kBlockThreads>(cnt, kBlockThreads, wtot, threadIdx.x);
    const uint64_t run0 = running;
    // copy bucket by bucket; every thread helps with each bucket
    const int nchunk = (int)((nb - base) < (uint64_t)kBlockThreads ? (nb - base) : (uint64_t)kBlockThreads);
    for (int j = 0; j < nchunk; ++j) {
      const uint64_t bj = b0 + base + j;
      const uint32_t U = h.bucnt[bj];
      const uint64_t lo = h.hist[bj];
      const uint64_t dstp = off + run0 + cnt[j];
      for (uint32_t i = threadIdx.x; i < U; i += kBlockThreads) a.sigkey[dstp + i] = h.tmp2[lo + i];
    }
    __syncthreads();
    if (threadIdx.x == kBlockThreads - 1) running = run0 + cnt[kBlockThreads - 1] + myc;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(kFull, term, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t tot = 0;
    for (int w = 0; w < kBlockThreads / 32; ++w) tot += red[w];
    const uint64_t U = running;
    a.ucnt[u] = (uint32_t)U;
    a.hash[u] = node_hash(tot, a.prev[u], U, a.seed, a.mask);
  }
}

// --------------------------------------------------------------------------
// Grouping: equal hashes -> smallest node id; exact verification
// --------------------------------------------------------------------------
struct GroupArgs {
  const uint64_t* hash;
  uint64_t* tkey;
  uint32_t* tmin;
  uint64_t tmask;   // table capacity - 1
  uint32_t* slot;
  uint32_t* rep;
  const uint8_t* alive;  // may be null (all alive)
  uint32_t* err;
};

__device__ __forceinline__ uint32_t table_home(uint64_t h, uint64_t tmask) {
  return (uint32_t)(mix64(h ^ 0x9e3779b97f4a7c15ull) & tmask);
}

__global__ void k_group_insert(GroupArgs g, const uint32_t* list, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t u = list ? list[i] : (uint32_t)i;
    if (!list && g.alive && !g.alive[u]) continue;
    const uint64_t h = g.hash[u];
    uint32_t s = table_home(h, g.tmask);
    volatile uint64_t* vk = g.tkey;
    bool found = false;
    for (uint64_t t = 0; t <= g.tmask; ++t) {
      const uint64_t cur = vk[s];
      if (cur == h) { found = true; break; }
      if (cur == kEmpty64) {
        const uint64_t old = atomicCAS((unsigned long long*)&g.tkey[s], (unsigned long long)kEmpty64,
                                       (unsigned long long)h);
        if (old == kEmpty64 || old == h) { found = true; break; }
      }
      s = (uint32_t)((s + 1) & g.tmask);
    }
    if (!found) {
      atomicOr(g.err, kErrProbe);
      continue;
    }
    atomicMin(&g.tmin[s], u);
    g.slot[u] = s;
  }
}

struct VerifyArgs {
  int mode;                 // 0: level 0 (labels), 1: signatures
  const uint32_t* nlabel;
  const uint32_t* prev;
  const uint32_t* ucnt;
  const uint64_t* off;
  const uint64_t* sigkey;
  uint32_t* out_list;       // unresolved nodes
  unsigned long long* n_out;
  unsigned long long* n_collided;
};

__device__ __forceinline__ bool same_signature(const VerifyArgs& v, uint32_t u, uint32_t r) {
  if (v.mode == 0) return v.nlabel[u] == v.nlabel[r];
  if (v.prev[u] != v.prev[r]) return false;
  const uint32_t U = v.ucnt[u];
  if (U != v.ucnt[r]) return false;
  const uint64_t* ku = v.sigkey + v.off[u];
  const uint64_t* kr = v.sigkey + v.off[r];
  for (uint32_t t = 0; t < U; ++t)
    if (ku[t] != kr[t]) return false;
  return true;
}

__global__ void k_group_verify(GroupArgs g, VerifyArgs v, const uint32_t* list, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t u = list ? list[i] : (uint32_t)i;
    if (!list && g.alive && !g.alive[u]) continue;
    const uint32_t r = g.tmin[g.slot[u]];
    if (r == u) { g.rep[u] = u; continue; }
    if (same_signature(v, u, r)) {
      g.rep[u] = r;
    } else {
      g.rep[u] = kNone32;
      const unsigned long long p = atomicAdd(v.n_out, 1ull);
      v.out_list[p] = u;
      atomicAdd(v.n_collided, 1ull);
    }
  }
}

// --------------------------------------------------------------------------
// Canonical renumbering: heads are nodes with rep[u] == u (the smallest node
// of their block); block id = number of heads before the node.
// --------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

struct RankArgs {
  uint64_t n;
  const uint32_t* rep;
  const uint8_t* alive;
  const uint32_t* ucnt;    // may be null (level 0)
  uint32_t* pid;           // output level
  uint64_t* bsum;          // per tile head count -> exclusive offsets
  unsigned long long* stats;  // [0] heads total, [2] key total, [3] max signature
};

__device__ __forceinline__ bool is_head(const RankArgs& r, uint64_t u) {
  return u < r.n && (!r.alive || r.alive[u]) && r.rep[u] == (uint32_t)u;
}

__global__ void __launch_bounds__(kScanThreads) k_rank_tilesum(RankArgs r) {
  __shared__ unsigned long long red[kScanThreads / 32];
  __shared__ unsigned long long redk[kScanThreads / 32];
  __shared__ unsigned int redm[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  unsigned long long c = 0, keys = 0;
  unsigned int mx = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    const uint64_t u = base + (uint64_t)t * kScanThreads + threadIdx.x;
    c += is_head(r, u) ? 1 : 0;
    if (r.ucnt && u < r.n && (!r.alive || r.alive[u])) {
      const uint32_t q = r.ucnt[u];
      keys += q;
      mx = max(mx, q);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(kFull, c, o);
    keys += __shfl_xor_sync(kFull, keys, o);
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = c;
    redk[threadIdx.x >> 5] = keys;
    redm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0, kt = 0;
    unsigned int m = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
      tot += red[w];
      kt += redk[w];
      m = max(m, redm[w]);
    }
    r.bsum[blockIdx.x] = tot;
    if (r.ucnt) {
      atomicAdd(&r.stats[2], kt);
      atomicMax(&r.stats[3], (unsigned long long)m);
    }
  }
}

// Exclusive scan of bsum[0..nb) in one CTA; total into stats[0].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint64_t* bsum, uint64_t nb,
                                                              unsigned long long* stats) {
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
  if (threadIdx.x == 0) stats[0] = carry;
}

// Heads get their rank (tile offset + rank inside the tile).
__global__ void __launch_bounds__(kScanThreads) k_rank_heads(RankArgs r) {
  __shared__ unsigned int wt[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  unsigned int f[kScanItems];
  unsigned int c = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    f[t] = is_head(r, base + t) ? 1u : 0u;
    c += f[t];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned int t = wt[lane];
    unsigned int xx = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(kFull, xx, o);
      if (lane >= o) xx += y;
    }
    wt[lane] = xx - t;
  }
  __syncthreads();
  uint64_t rank = r.bsum[blockIdx.x] + wt[w] + (x - c);
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (f[t]) r.pid[base + t] = (uint32_t)rank;
    rank += f[t];
  }
}

// Members copy their head's block id; deleted nodes get kDead.
__global__ void k_rank_fill(RankArgs r) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < r.n;
       u += (uint64_t)gridDim.x * blockDim.x) {
    if (r.alive && !r.alive[u]) { r.pid[u] = kDead; continue; }
    const uint32_t h = r.rep[u];
    if (h != (uint32_t)u) r.pid[u] = r.pid[h];
  }
}

// Level 0 hash: the node label.
__global__ void k_label_hash(uint64_t n, const uint32_t* nlabel, uint64_t* hash, uint64_t seed,
                             uint64_t mask) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n;
       u += (uint64_t)gridDim.x * blockDim.x)
    hash[u] = node_hash(0, nlabel[u], 0, seed, mask);
}

// --------------------------------------------------------------------------
// Degree classes (once per graph)
// --------------------------------------------------------------------------
constexpr int kClassWarp = kSmallClasses, kClassBlock = kSmallClasses + 1,
              kClassHub = kSmallClasses + 2, kNumClasses = kSmallClasses + 3;

__device__ __forceinline__ int degree_class(uint64_t d) {
  if (d <= (uint64_t)kSmallMax) {
    int c = 0;
    while ((1ull << c) < d) ++c;
    return c;
  }
  if (d <= (uint64_t)kWarpMax) return kClassWarp;
  if (d <= (uint64_t)kBlockMax) return kClassBlock;
  return kClassHub;
}

// Stable partition of the alive nodes by degree class, in tiles of 1024 nodes:
// per-tile class counts, an exclusive scan over (class, tile) on the host,
// then each tile writes its nodes in id order.
constexpr int kClassTile = 1024;

__global__ void __launch_bounds__(kClassTile)
    k_class_tile_count(uint64_t n, const uint64_t* off, const uint8_t* alive, uint64_t ntiles,
                       unsigned long long* tcnt) {
  __shared__ unsigned int c[kNumClasses];
  if (threadIdx.x < kNumClasses) c[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t u = (uint64_t)blockIdx.x * kClassTile + threadIdx.x;
  if (u < n && (!alive || alive[u])) atomicAdd(&c[degree_class(off[u + 1] - off[u])], 1u);
  __syncthreads();
  if (threadIdx.x < kNumClasses) tcnt[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

__global__ void __launch_bounds__(kClassTile)
    k_class_tile_scatter(uint64_t n, const uint64_t* off, const uint8_t* alive, uint64_t ntiles,
                         const unsigned long long* tbase, uint32_t* out) {
  __shared__ unsigned int wcount[kClassTile / 32];
  const uint64_t u = (uint64_t)blockIdx.x * kClassTile + threadIdx.x;
  const int cls = (u < n && (!alive || alive[u])) ? degree_class(off[u + 1] - off[u]) : -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < kNumClasses; ++c) {
    const unsigned m = __ballot_sync(kFull, cls == c);
    if (lane == 0) wcount[w] = __popc(m);
    __syncthreads();
    unsigned before = 0;
    for (int i = 0; i < w; ++i) before += wcount[i];
    if (cls == c)
      out[tbase[(uint64_t)c * ntiles + blockIdx.x] + before + __popc(m & ((1u << lane) - 1u))] = (uint32_t)u;
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Host helpers
// --------------------------------------------------------------------------
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

Status set_smem_attrs() {
  static bool done = false;
  if (done) return Status::Ok();
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_sig_warp<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kWarpWsBytes * kWarpsPerBlock));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sig_warp<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kWarpWsBytes * kWarpsPerBlock));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sig_block<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBlkWsBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sig_block<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBlkWsBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hub_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBlkWsBytes);
  if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute");
  done = true;
  return Status::Ok();
}

Status read_scalars(Store& s, uint64_t* out, int count) {
  Status st = cuda_check(cudaMemcpyAsync(s.h_scalars.p, s.d_scalars.p, 8 * sizeof(uint64_t),
                                         cudaMemcpyDeviceToHost, s.stream), "read scalars");
  if (!st.ok()) return st;
  st = cuda_check(cudaStreamSynchronize(s.stream), "stream sync");
  if (!st.ok()) return st;
  std::memcpy(out, s.h_scalars.p, count * sizeof(uint64_t));
  return Status::Ok();
}

Status read_err(Store& s, uint32_t* err) {
  uint32_t v = 0;
  Status st = cuda_check(cudaMemcpyAsync(&v, s.d_err.p, 4, cudaMemcpyDeviceToHost, s.stream), "read err");
  if (!st.ok()) return st;
  st = cuda_check(cudaStreamSynchronize(s.stream), "stream sync");
  *err = v;
  return st;
}

uint64_t table_capacity(uint64_t n) {
  uint64_t c = 1024;
  while (c < 2 * n) c <<= 1;
  return c;
}

// Group the nodes of `hash` (all alive nodes), verify exactly, repair
// collisions, then renumber canonically into `pid`.  Returns the block count.
Status group_and_rank(Store& s, int mode, const uint32_t* prev, uint32_t* pid, uint64_t* blocks,
                      uint64_t* collided, bool with_stats, uint64_t* keys, uint64_t* maxsig) {
  const uint64_t n = s.n;
  Status st;
  uint32_t* err = ptr<uint32_t>(s.d_err);
  unsigned long long* sc = ptr<unsigned long long>(s.d_scalars);
  GroupArgs g;
  g.hash = ptr<uint64_t>(s.hash);
  g.tkey = ptr<uint64_t>(s.tkey);
  g.tmin = ptr<uint32_t>(s.tmin);
  g.tmask = s.tcap - 1;
  g.slot = ptr<uint32_t>(s.slot);
  g.rep = ptr<uint32_t>(s.rep);
  g.alive = s.any_dead ? ptr<uint8_t>(s.alive) : nullptr;
  g.err = err;
  VerifyArgs v;
  v.mode = mode;
  v.nlabel = ptr<uint32_t>(s.nlabel);
  v.prev = prev;
  v.ucnt = ptr<uint32_t>(s.ucnt);
  v.off = ptr<uint64_t>(s.offsets);
  v.sigkey = ptr<uint64_t>(s.sigkey);
  v.n_collided = sc + 4;
  const int sms = sm_count(s.device);
  const unsigned gblocks = (unsigned)std::min<uint64_t>(grid_for(n, 256), (uint64_t)sms * 16);
  {
    TimedScope ts(s, KBISIM_KERNEL_OTHER);
    cudaMemsetAsync(s.tkey.p, 0xFF, s.tcap * 8, s.stream);
    cudaMemsetAsync(s.tmin.p, 0xFF, s.tcap * 4, s.stream);
    cudaMemsetAsync(s.d_scalars.p, 0, 8 * 8, s.stream);
  }
  {
    TimedScope ts(s, KBISIM_KERNEL_GROUP);
    k_group_insert<<<gblocks, 256, 0, s.stream>>>(g, nullptr, n);
  }
  if (!(st = launch_check("k_group_insert")).ok()) return st;
  v.out_list = ptr<uint32_t>(s.ulist[0]);
  v.n_out = sc + 1;
  {
    TimedScope ts(s, KBISIM_KERNEL_VERIFY);
    k_group_verify<<<gblocks, 256, 0, s.stream>>>(g, v, nullptr, n);
  }
  if (!(st = launch_check("k_group_verify")).ok()) return st;
  uint64_t h[8];
  if (!(st = read_scalars(s, h, 8)).ok()) return st;
  uint64_t unresolved = h[1];
  // Collision repair: the unresolved nodes hold whole classes; the smallest
  // unresolved node of each hash group heads its class, so every pass
  // settles at least one class per group.
  int cur = 0;
  uint64_t passes = 0;
  while (unresolved > 0) {
    if (++passes > n + 1) return Status::Err(KBISIM_ERR_TIMEOUT, "collision repair did not converge");
    const uint64_t cap = table_capacity(unresolved);
    GroupArgs g2 = g;
    g2.tmask = cap - 1;
    VerifyArgs v2 = v;
    v2.out_list = ptr<uint32_t>(s.ulist[cur ^ 1]);
    v2.n_out = sc + 5;
    const unsigned b2 = grid_for(unresolved, 256);
    {
      TimedScope ts(s, KBISIM_KERNEL_OTHER);
      cudaMemsetAsync(s.tkey.p, 0xFF, cap * 8, s.stream);
      cudaMemsetAsync(s.tmin.p, 0xFF, cap * 4, s.stream);
      cudaMemsetAsync(sc + 5, 0, 8, s.stream);
      k_group_insert<<<b2, 256, 0, s.stream>>>(g2, ptr<uint32_t>(s.ulist[cur]), unresolved);
      k_group_verify<<<b2, 256, 0, s.stream>>>(g2, v2, ptr<uint32_t>(s.ulist[cur]), unresolved);
    }
    if (!(st = launch_check("collision repair")).ok()) return st;
    if (!(st = read_scalars(s, h, 8)).ok()) return st;
    if (h[5] >= unresolved)  // every pass settles the smallest node of each group
      return Status::Err(KBISIM_ERR_TIMEOUT, "collision repair made no progress");
    unresolved = h[5];
    cur ^= 1;
  }
  *collided = h[4];
  // canonical renumbering
  RankArgs r;
  r.n = n;
  r.rep = ptr<uint32_t>(s.rep);
  r.alive = g.alive;
  r.ucnt = with_stats ? ptr<uint32_t>(s.ucnt) : nullptr;
  r.pid = pid;
  r.bsum = ptr<uint64_t>(s.bsum);
  r.stats = sc;
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  {
    TimedScope ts(s, KBISIM_KERNEL_RENUMBER);
    if (tiles) {
      k_rank_tilesum<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(r);
      k_scan_tiles<<<1, kScanThreads, 0, s.stream>>>(r.bsum, tiles, sc);
      k_rank_heads<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(r);
      k_rank_fill<<<gblocks, 256, 0, s.stream>>>(r);
    }
  }
  if (!(st = launch_check("renumber")).ok()) return st;
  if (!(st = read_scalars(s, h, 8)).ok()) return st;
  *blocks = h[0];
  if (keys) *keys = h[2];
  if (maxsig) *maxsig = h[3];
  uint32_t e = 0;
  if (!(st = read_err(s, &e)).ok()) return st;
  if (e & kErrProbe) return Status::Err(KBISIM_ERR_TIMEOUT, "hash table probe bound exceeded");
  if (e & kErrChecked) return Status::Err(KBISIM_ERR_CHECKED, "device bounds check failed");
  return Status::Ok();
}

}  // namespace

// ---------------------------------------------------------------------------
// Degree classes and hub layout (once per graph, after load)
// ---------------------------------------------------------------------------
Status prepare_classes(Store& s) {
  Status st = set_smem_attrs();
  if (!st.ok()) return st;
  const uint64_t n = s.n;
  const uint8_t* alive = s.any_dead ? ptr<uint8_t>(s.alive) : nullptr;
  const uint64_t ntiles = std::max<uint64_t>(1, (n + kClassTile - 1) / kClassTile);
  Buf tcnt;
  if (!(st = ensure(s, tcnt, ntiles * kNumClasses * 8)).ok()) return st;
  cudaMemsetAsync(tcnt.p, 0, ntiles * kNumClasses * 8, s.stream);
  if (n)
    k_class_tile_count<<<(unsigned)ntiles, kClassTile, 0, s.stream>>>(n, ptr<uint64_t>(s.offsets), alive, ntiles,
                                                                      ptr<unsigned long long>(tcnt));
  if (!(st = launch_check("k_class_tile_count")).ok()) { release(s, tcnt); return st; }
  std::vector<uint64_t> h(ntiles * kNumClasses);
  st = cuda_check(cudaMemcpyAsync(h.data(), tcnt.p, h.size() * 8, cudaMemcpyDeviceToHost, s.stream), "class counts");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) { release(s, tcnt); return st; }
  uint64_t run = 0;
  uint64_t cstart[kNumClasses + 1];
  for (int c = 0; c < kNumClasses; ++c) {
    cstart[c] = run;
    for (uint64_t t = 0; t < ntiles; ++t) {
      const uint64_t v = h[(uint64_t)c * ntiles + t];
      h[(uint64_t)c * ntiles + t] = run;
      run += v;
    }
  }
  cstart[kNumClasses] = run;
  st = cuda_check(cudaMemcpyAsync(tcnt.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s.stream), "class bases");
  if (st.ok()) st = ensure(s, s.class_nodes, std::max<uint64_t>(1, run) * 4);
  if (!st.ok()) { release(s, tcnt); return st; }
  if (n)
    k_class_tile_scatter<<<(unsigned)ntiles, kClassTile, 0, s.stream>>>(
        n, ptr<uint64_t>(s.offsets), alive, ntiles, ptr<unsigned long long>(tcnt), ptr<uint32_t>(s.class_nodes));
  st = launch_check("k_class_tile_scatter");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  release(s, tcnt);
  if (!st.ok()) return st;
  for (int c = 0; c <= kNumClasses; ++c) s.class_start[c] = cstart[c];
  for (int k = 0; k < kSmallClasses; ++k) {
    s.small_start[k] = cstart[k];
    s.small_count[k] = cstart[k + 1] - cstart[k];
  }
  s.small_start[kSmallClasses] = cstart[kSmallClasses];
  s.n_warp = cstart[kClassWarp + 1] - cstart[kClassWarp];
  s.n_block = cstart[kClassBlock + 1] - cstart[kClassBlock];
  s.n_hub = cstart[kClassHub + 1] - cstart[kClassHub];
  // hub layout on the host (few nodes, already in id order)
  s.hub_extra_bits = 0;
  s.h_hub_deg.assign(s.n_hub, 0);
  s.h_hub_degbits.assign(s.n_hub, 0);
  s.hub_edges = 0;
  if (s.n_hub) {
    std::vector<uint32_t> hn(s.n_hub);
    const uint32_t* hubs = ptr<uint32_t>(s.class_nodes) + cstart[kClassHub];
    st = cuda_check(cudaMemcpyAsync(hn.data(), hubs, s.n_hub * 4, cudaMemcpyDeviceToHost, s.stream), "hub nodes");
    if (!st.ok()) return st;
    if (!(st = cuda_check(cudaStreamSynchronize(s.stream), "sync")).ok()) return st;
    std::vector<uint64_t> lo(s.n_hub), hi(s.n_hub);
    for (uint64_t i = 0; i < s.n_hub; ++i) {
      cudaMemcpyAsync(&lo[i], ptr<uint64_t>(s.offsets) + hn[i], 8, cudaMemcpyDeviceToHost, s.stream);
      cudaMemcpyAsync(&hi[i], ptr<uint64_t>(s.offsets) + hn[i] + 1, 8, cudaMemcpyDeviceToHost, s.stream);
    }
    if (!(st = cuda_check(cudaStreamSynchronize(s.stream), "hub offsets")).ok()) return st;
    std::vector<uint4> chunks;
    for (uint64_t i = 0; i < s.n_hub; ++i) {
      const uint64_t d = hi[i] - lo[i];
      s.h_hub_deg[i] = d;
      uint32_t bits = 0;
      while (((uint64_t)kHubBucketTarget << bits) < d) ++bits;
      s.h_hub_degbits[i] = bits;
      s.hub_edges += d;
      for (uint64_t b = 0; b < d; b += kHubChunk) {
        const uint64_t e = lo[i] + b;
        uint4 q;
        q.x = (uint32_t)i;
        q.y = (uint32_t)(e & 0xFFFFFFFFu);
        q.z = (uint32_t)(e >> 32);
        q.w = (uint32_t)std::min<uint64_t>(kHubChunk, d - b);
        chunks.push_back(q);
      }
    }
    s.n_hub_chunks = chunks.size();
    if (!(st = ensure(s, s.hub_chunks, chunks.size() * sizeof(uint4))).ok()) return st;
    st = cuda_check(cudaMemcpyAsync(s.hub_chunks.p, chunks.data(), chunks.size() * sizeof(uint4),
                                    cudaMemcpyHostToDevice, s.stream), "hub chunks");
    if (!st.ok()) return st;
    if (!(st = ensure(s, s.hub_tmp, s.hub_edges * 8)).ok()) return st;
    if (!(st = ensure(s, s.hub_tmp2, s.hub_edges * 8)).ok()) return st;
    if (!(st = cuda_check(cudaStreamSynchronize(s.stream), "sync")).ok()) return st;
  }
  return Status::Ok();
}

namespace {

// (Re)build the per-hub bucket table for the current extra bits.
Status hub_layout(Store& s) {
  Status st;
  std::vector<uint32_t> bits(s.n_hub);
  std::vector<uint64_t> bbase(s.n_hub + 1, 0);
  for (uint64_t i = 0; i < s.n_hub; ++i) {
    bits[i] = s.h_hub_degbits[i];
    bbase[i + 1] = bbase[i] + (1ull << (bits[i] + s.hub_extra_bits));
  }
  s.n_hub_buckets = bbase[s.n_hub];
  if (!(st = ensure(s, s.hub_bits, s.n_hub * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_bbase, (s.n_hub + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, s.hub_hist, s.n_hub_buckets * 8)).ok()) return st;
  if (!(st = ensure(s, s.hub_cursor, s.n_hub_buckets * 8)).ok()) return st;
  if (!(st = ensure(s, s.hub_ucnt, s.n_hub_buckets * 4)).ok()) return st;
  if (!(st = ensure(s, s.hub_hpart, s.n_hub_buckets * 8)).ok()) return st;
  cudaMemcpyAsync(s.hub_bits.p, bits.data(), s.n_hub * 4, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.hub_bbase.p, bbase.data(), (s.n_hub + 1) * 8, cudaMemcpyHostToDevice, s.stream);
  return cuda_check(cudaStreamSynchronize(s.stream), "hub layout");
}

// Exclusive scan of a uint64 array in place (reuses the renumber tile scan).
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

Status scan64(Store& s, uint64_t* a, uint64_t n, uint64_t* copy) {
  if (!n) return Status::Ok();
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  Status st = ensure(s, s.bsum, std::max<uint64_t>(tiles, 1) * 8);
  if (!st.ok()) return st;
  uint64_t* bs = ptr<uint64_t>(s.bsum);
  k_tile_sum64<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(a, n, bs);
  k_scan_tiles<<<1, kScanThreads, 0, s.stream>>>(bs, tiles, ptr<unsigned long long>(s.d_scalars) + 7);
  k_tile_scan64<<<(unsigned)tiles, kScanThreads, 0, s.stream>>>(a, n, bs, copy);
  return launch_check("scan64");
}

template <typename LabelT>
Status run_signatures(Store& s, const SigArgs& a) {
  Status st;
  const int sms = sm_count(s.device);
  // small
  SmallLaunch L;
  uint32_t b = 0;
  for (int c = 0; c < kSmallClasses; ++c) {
    L.start[c] = s.small_start[c];
    L.count[c] = s.small_count[c];
    L.bstart[c] = b;
    const uint64_t npw = 32 >> c;
    const uint64_t warps = (s.small_count[c] + npw - 1) / npw;
    b += (uint32_t)((warps + kSmallWarps - 1) / kSmallWarps);
  }
  L.bstart[kSmallClasses] = b;
  if (b) {
    TimedScope ts(s, KBISIM_KERNEL_SIG_SMALL);
    k_sig_small<LabelT><<<b, kSmallWarps * 32, 0, s.stream>>>(a, ptr<uint32_t>(s.class_nodes), L);
  }
  if (!(st = launch_check("k_sig_small")).ok()) return st;
  if (s.n_warp) {
    TimedScope ts(s, KBISIM_KERNEL_SIG_MEDIUM);
    const unsigned g = (unsigned)std::min<uint64_t>((s.n_warp + kWarpsPerBlock - 1) / kWarpsPerBlock,
                                                    (uint64_t)sms * 8);
    k_sig_warp<LabelT><<<g, kWarpsPerBlock * 32, kWarpWsBytes * kWarpsPerBlock, s.stream>>>(
        a, ptr<uint32_t>(s.class_nodes) + s.class_start[kClassWarp], s.n_warp);
  }
  if (!(st = launch_check("k_sig_warp")).ok()) return st;
  if (s.n_block) {
    TimedScope ts(s, KBISIM_KERNEL_SIG_MEDIUM);
    const unsigned g = (unsigned)std::min<uint64_t>(s.n_block, (uint64_t)sms * 4);
    k_sig_block<LabelT><<<g, kBlockThreads, kBlkWsBytes, s.stream>>>(
        a, ptr<uint32_t>(s.class_nodes) + s.class_start[kClassBlock], s.n_block);
  }
  if (!(st = launch_check("k_sig_block")).ok()) return st;
  if (s.n_hub) {
    for (int attempt = 0;; ++attempt) {
      if (!(st = hub_layout(s)).ok()) return st;
      HubArgs h;
      h.hub_nodes = ptr<uint32_t>(s.class_nodes) + s.class_start[kClassHub];
      h.hub_bits = ptr<uint32_t>(s.hub_bits);
      h.hub_bbase = ptr<uint64_t>(s.hub_bbase);
      h.chunks = ptr<uint4>(s.hub_chunks);
      h.extra_bits = s.hub_extra_bits;
      h.hist = ptr<uint64_t>(s.hub_hist);
      h.cursor = ptr<uint64_t>(s.hub_cursor);
      h.bucnt = ptr<uint32_t>(s.hub_ucnt);
      h.bhpart = ptr<uint64_t>(s.hub_hpart);
      h.tmp = ptr<uint64_t>(s.hub_tmp);
      h.tmp2 = ptr<uint64_t>(s.hub_tmp2);
      {
        TimedScope ts(s, KBISIM_KERNEL_SIG_HUB);
        cudaMemsetAsync(h.hist, 0, s.n_hub_buckets * 8, s.stream);
        k_hub_hist<LabelT><<<(unsigned)s.n_hub_chunks, kBlockThreads, 0, s.stream>>>(a, h);
        if (!(st = scan64(s, h.hist, s.n_hub_buckets, h.cursor)).ok()) return st;
        k_hub_scatter<LabelT><<<(unsigned)s.n_hub_chunks, kBlockThreads, 0, s.stream>>>(a, h);
        const unsigned g = (unsigned)std::min<uint64_t>(s.n_hub_buckets, (uint64_t)sms * 4);
        k_hub_bucket<<<g, kBlockThreads, kBlkWsBytes, s.stream>>>(h, s.n_hub_buckets, a.seed, a.err);
        k_hub_compact<<<(unsigned)s.n_hub, kBlockThreads, 0, s.stream>>>(a, h);
      }
      if (!(st = launch_check("hub kernels")).ok()) return st;
      uint32_t e = 0;
      if (!(st = read_err(s, &e)).ok()) return st;
      if (!(e & kErrHubOverflow)) break;
      if (attempt >= 6) return Status::Err(KBISIM_ERR_TIMEOUT, "hub bucket overflow persists");
      s.hub_extra_bits += 2;
      cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
    }
  }
  return Status::Ok();
}

Status ensure_round_scratch(Store& s) {
  Status st;
  const uint64_t n = std::max<uint64_t>(s.n, 1), m = std::max<uint64_t>(s.m, 1);
  const uint64_t cap = table_capacity(n);
  if (!(st = ensure(s, s.sigkey, m * 8)).ok()) return st;
  if (!(st = ensure(s, s.ucnt, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.hash, n * 8)).ok()) return st;
  if (!(st = ensure(s, s.tkey, cap * 8)).ok()) return st;
  if (!(st = ensure(s, s.tmin, cap * 4)).ok()) return st;
  s.tcap = cap;
  if (!(st = ensure(s, s.slot, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.rep, n * 4)).ok()) return st;
  if (!(st = ensure(s, s.ulist[0], n * 4)).ok()) return st;
  if (!(st = ensure(s, s.ulist[1], n * 4)).ok()) return st;
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (!(st = ensure(s, s.bsum, std::max<uint64_t>(tiles, 64) * 8)).ok()) return st;
  return Status::Ok();
}

}  // namespace

Status compute_level0(Store& s) {
  Status st = ensure_round_scratch(s);
  if (!st.ok()) return st;
  const int sms = sm_count(s.device);
  const unsigned blocks = (unsigned)std::min<uint64_t>(grid_for(s.n, 256), (uint64_t)sms * 16);
  {
    TimedScope ts(s, KBISIM_KERNEL_LABEL_GROUP);
    if (s.n)
      k_label_hash<<<blocks, 256, 0, s.stream>>>(s.n, ptr<uint32_t>(s.nlabel), ptr<uint64_t>(s.hash),
                                                 s.seed, s.hash_mask);
  }
  if (!(st = launch_check("k_label_hash")).ok()) return st;
  uint64_t blocks_out = 0, coll = 0;
  st = group_and_rank(s, 0, nullptr, ptr<uint32_t>(s.level[0]), &blocks_out, &coll, false, nullptr,
                      nullptr);
  if (!st.ok()) return st;
  s.counts[0] = blocks_out;
  return Status::Ok();
}

Status compute_round(Store& s, uint32_t i) {
  Status st = ensure_round_scratch(s);
  if (!st.ok()) return st;
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  SigArgs a;
  a.off = ptr<uint64_t>(s.offsets);
  a.dst = ptr<uint32_t>(s.dst);
  a.lab = s.elabel.p;
  a.prev = ptr<uint32_t>(s.level[i - 1]);
  a.sigkey = ptr<uint64_t>(s.sigkey);
  a.ucnt = ptr<uint32_t>(s.ucnt);
  a.hash = ptr<uint64_t>(s.hash);
  a.seed = s.seed;
  a.mask = s.hash_mask;
  a.err = ptr<uint32_t>(s.d_err);
  st = s.label8 ? run_signatures<uint8_t>(s, a) : run_signatures<uint32_t>(s, a);
  if (!st.ok()) return st;
  uint64_t blocks = 0, coll = 0, keys = 0, maxsig = 0;
  st = group_and_rank(s, 1, a.prev, ptr<uint32_t>(s.level[i]), &blocks, &coll, true, &keys, &maxsig);
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

}  // namespace kb
