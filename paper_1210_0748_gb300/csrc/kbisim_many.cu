// Batched build: many independent graphs refined together.
//
// The graphs arrive as one graph whose node ids are grouped by graph (graph j
// owns ids start[j] .. start[j+1]-1) with no edge between two graphs.  The
// library refines this disjoint union with its usual kernels, one launch
// sequence per round for all graphs.  k-bisimilarity of two nodes of one graph
// depends only on that graph (Definition 1 follows out-edges, which stay in
// the graph), so the union's partition at every level, restricted to graph j,
// is graph j's own partition.  After each level, the blocks are renumbered
// per graph: the block of (graph j, union block b) gets the rank of its
// smallest node id within graph j, which is the canonical numbering graph j
// would get alone.  Per-graph block counts give each graph its own early stop.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "kbisim_internal.cuh"

namespace kb {
namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kAggItems = 4, kAggChunk = kThreads * kAggItems, kAggSlots = 2 * kAggChunk;

template <typename T>
T* ptr(const Buf& b) {
  return static_cast<T*>(b.p);
}

unsigned grid_for(uint64_t n, int threads, int cap) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, (uint64_t)cap));
}

// Graph of each original node: the largest j with start[j] <= o.
__global__ void k_many_gid(uint64_t n, const uint64_t* start, uint32_t G, uint32_t* gid) {
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n; o += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = G;  // start[lo] <= o < start[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (start[mid] <= o) lo = mid; else hi = mid;
    }
    gid[o] = lo;
  }
}

// gidp[p] = graph of internal node p; every edge must stay in its graph.
// One warp per node (hubs included).
__global__ void k_many_check(uint64_t n, const uint64_t* off, const uint32_t* dst, const uint32_t* p2o,
                             const uint32_t* gid, uint32_t* gidp, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  bool bad = false;
  for (uint64_t p = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; p < n; p += warps) {
    const uint32_t g = gid[p2o[p]];
    if (lane == 0) gidp[p] = g;
    for (uint64_t e = off[p] + lane; e < off[p + 1]; e += 32) bad |= gid[p2o[dst[e]]] != g;
  }
  if (__any_sync(kFullMask, bad) && lane == 0) atomicOr(err, kErrBadInput);
}

struct ManyArgs {
  uint64_t n_alive;
  const uint32_t* lvl;     // union level, internal order
  const uint8_t* alone;    // union level: node alone in its block
  const uint32_t* p2o;
  const uint32_t* o2p;
  const uint32_t* gid;     // graph of each original node
  const uint32_t* gidp;    // graph of each internal node
  unsigned long long* tkey;  // (graph << 32 | union block), empty = all ones
  uint32_t* tmin;            // smallest original id of the key
  uint64_t tmask;
  uint32_t* slot;          // per internal node: its key's slot
  uint32_t* hbits;         // head bitmap over original ids
  const uint64_t* hword;   // heads before each bitmap word
  uint32_t* err;
};

__device__ __forceinline__ uint32_t many_insert(const ManyArgs& a, unsigned long long key, uint32_t o) {
  uint32_t s = (uint32_t)(mix64(key) & a.tmask);
  for (uint64_t t = 0; t <= a.tmask; ++t) {
    const unsigned long long cur = atomicCAS(&a.tkey[s], (unsigned long long)kEmpty64, key);
    if (cur == kEmpty64 || cur == key) {
      atomicMin(&a.tmin[s], o);
      return s;
    }
    s = (uint32_t)((s + 1) & a.tmask);
  }
  atomicOr(a.err, kErrProbe);
  return 0;
}

// Nodes not alone in their union block: key (graph, block) -> smallest
// original id.  A CTA combines equal keys of its 1024 nodes first.
__global__ void __launch_bounds__(kThreads) k_many_insert(ManyArgs a) {
  __shared__ unsigned long long skey[kAggSlots];
  __shared__ unsigned int smin[kAggSlots];
  __shared__ unsigned int sglob[kAggSlots];
  for (uint64_t base = (uint64_t)blockIdx.x * kAggChunk; base < a.n_alive; base += (uint64_t)gridDim.x * kAggChunk) {
    for (int i = threadIdx.x; i < kAggSlots; i += kThreads) {
      skey[i] = kEmpty64;
      smin[i] = kNone32;
    }
    __syncthreads();
    uint32_t ls[kAggItems];
    uint64_t pp[kAggItems];
#pragma unroll
    for (int t = 0; t < kAggItems; ++t) {
      const uint64_t p = base + threadIdx.x + (uint64_t)t * kThreads;
      ls[t] = kNone32;
      pp[t] = p;
      if (p >= a.n_alive || a.alone[p]) continue;
      const unsigned long long key = ((unsigned long long)a.gidp[p] << 32) | a.lvl[p];
      uint32_t s = (uint32_t)(mix64(key) & (kAggSlots - 1));
      for (int q = 0; q < kAggSlots; ++q) {  // at most kAggChunk distinct keys: always room
        const unsigned long long cur = atomicCAS(&skey[s], (unsigned long long)kEmpty64, key);
        if (cur == kEmpty64 || cur == key) break;
        s = (s + 1) & (kAggSlots - 1);
      }
      atomicMin(&smin[s], a.p2o[p]);
      ls[t] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kAggSlots; i += kThreads)
      if (skey[i] != kEmpty64) sglob[i] = many_insert(a, skey[i], smin[i]);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kAggItems; ++t)
      if (ls[t] != kNone32) a.slot[pp[t]] = sglob[ls[t]];
    __syncthreads();
  }
}

// Heads: nodes alone in their union block, and the smallest node of each key.
__global__ void k_many_heads(ManyArgs a) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < a.n_alive;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t o = a.p2o[p];
    if (a.alone[p] || a.tmin[a.slot[p]] == o) atomicOr(&a.hbits[o >> 5], 1u << (o & 31));
  }
}

__global__ void k_many_word_counts(const uint32_t* hbits, uint64_t words, uint64_t* hword) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x)
    hword[w] = __popc(hbits[w]);
}

__device__ __forceinline__ uint64_t heads_before(const ManyArgs& a, uint64_t x) {
  const uint64_t w = x >> 5;
  return a.hword[w] + (uint64_t)__popc(a.hbits[w] & ((1u << (x & 31)) - 1u));
}

// Per-graph identifier of every node (original order): rank of its head
// among the heads of its graph.
__global__ void k_many_pid(ManyArgs a, uint64_t n, const uint64_t* start, uint32_t* out) {
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n; o += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = a.o2p[o];
    if (p >= a.n_alive) {
      out[o] = kDead;
      continue;
    }
    const uint32_t head = a.alone[p] ? (uint32_t)o : a.tmin[a.slot[p]];
    out[o] = (uint32_t)(heads_before(a, head) - heads_before(a, start[a.gid[o]]));
  }
}

// cnt[j] = heads before start[j] (j <= G).
__global__ void k_many_counts(ManyArgs a, const uint64_t* start, uint32_t G, unsigned long long* cnt) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= G; j += gridDim.x * blockDim.x)
    cnt[j] = heads_before(a, start[j]);
}

// Work list of the next round: nodes of the graphs still refined.
__global__ void k_many_live_mask(uint64_t n_alive, const uint32_t* gidp, const uint8_t* live, uint32_t* mask) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w * 32 < n_alive;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t bits = 0;
    for (uint32_t b = 0; b < 32; ++b) {
      const uint64_t p = w * 32 + b;
      if (p < n_alive && live[gidp[p]]) bits |= 1u << b;
    }
    mask[w] = bits;
  }
}

}  // namespace

// After level l: the graphs that still need a round (l < k_j, and with early
// stop not yet stable) form the next round's work list; the others keep their
// blocks (their nodes are not signed again).  Only set while some graph has
// stopped and others go on.
Status many_work_list(Store& s, uint32_t l) {
  ManyState& m = s.many;
  s.round_mask = nullptr;
  std::vector<uint8_t> live(m.G, 0);
  uint64_t nlive = 0;
  for (uint32_t j = 0; j < m.G; ++j) {
    bool go = l < m.k[j];
    if (go && s.early_stop && l >= 1 && m.counts[l][j] == m.counts[l - 1][j]) go = false;
    live[j] = go ? 1 : 0;
    nlive += go ? 1 : 0;
  }
  m.live_graphs = nlive;
  if (nlive == 0 || nlive == m.G) return Status::Ok();
  Status st;
  const uint64_t words = s.n_alive / 32 + 1;
  if (!(st = ensure(s, m.live, m.G)).ok()) return st;
  if (!(st = ensure(s, m.live_mask, words * 4)).ok()) return st;
  st = cuda_check(cudaMemcpyAsync(m.live.p, live.data(), m.G, cudaMemcpyHostToDevice, s.stream), "live graphs");
  if (!st.ok()) return st;
  k_many_live_mask<<<grid_for(words, kThreads, s.sms * 16), kThreads, 0, s.stream>>>(
      s.n_alive, ptr<uint32_t>(m.gidp), ptr<uint8_t>(m.live), ptr<uint32_t>(m.live_mask));
  st = cuda_check(cudaGetLastError(), "live mask");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "live mask");  // the host vector goes away
  if (st.ok()) s.round_mask = ptr<uint32_t>(m.live_mask);
  return st;
}

// Per-graph renumbering of level l (called right after the union computed it).
Status many_level(Store& s, uint32_t l) {
  ManyState& m = s.many;
  const uint64_t n = s.n, na = s.n_alive;
  const uint64_t words = n / 32 + 1;  // one spare word: heads_before(n) stays in range
  Status st;
  if (m.lvl.size() < (size_t)l + 1) m.lvl.resize(l + 1);
  if (!(st = ensure(s, m.lvl[l], std::max<uint64_t>(n, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, m.hbits, words * 4)).ok()) return st;
  if (!(st = ensure(s, m.hword, words * 8)).ok()) return st;
  if (!(st = ensure(s, m.cnt, (m.G + 1) * 8)).ok()) return st;
  const uint64_t ins = na - std::min(na, s.n_alone);
  uint64_t cap = 1024;
  while (cap < 2 * ins) cap <<= 1;
  if (!(st = ensure(s, m.tkey, cap * 8)).ok()) return st;
  if (!(st = ensure(s, m.tmin, cap * 4)).ok()) return st;
  if (!(st = ensure(s, m.slot, std::max<uint64_t>(na, 1) * 4)).ok()) return st;
  ManyArgs a;
  a.n_alive = na;
  a.lvl = ptr<uint32_t>(s.level[l]);
  a.alone = ptr<uint8_t>(s.alone);
  a.p2o = ptr<uint32_t>(s.p2o);
  a.o2p = ptr<uint32_t>(s.o2p);
  a.gid = ptr<uint32_t>(m.gid);
  a.gidp = ptr<uint32_t>(m.gidp);
  a.tkey = ptr<unsigned long long>(m.tkey);
  a.tmin = ptr<uint32_t>(m.tmin);
  a.tmask = cap - 1;
  a.slot = ptr<uint32_t>(m.slot);
  a.hbits = ptr<uint32_t>(m.hbits);
  a.hword = ptr<uint64_t>(m.hword);
  a.err = ptr<uint32_t>(s.d_err);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device);
  if (sms <= 0) sms = 132;
  cudaMemsetAsync(m.tkey.p, 0xFF, cap * 8, s.stream);
  cudaMemsetAsync(m.tmin.p, 0xFF, cap * 4, s.stream);
  cudaMemsetAsync(m.hbits.p, 0, words * 4, s.stream);
  if (na) {
    k_many_insert<<<grid_for(na, kAggChunk, (int)resident_blocks(k_many_insert, kThreads, 0, sms)), kThreads, 0,
                    s.stream>>>(a);
    k_many_heads<<<grid_for(na, kThreads, sms * 16), kThreads, 0, s.stream>>>(a);
  }
  k_many_word_counts<<<grid_for(words, kThreads, sms * 16), kThreads, 0, s.stream>>>(ptr<uint32_t>(m.hbits), words,
                                                                                      ptr<uint64_t>(m.hword));
  if (!(st = scan_u64(s, ptr<uint64_t>(m.hword), words)).ok()) return st;
  if (n)
    k_many_pid<<<grid_for(n, kThreads, sms * 16), kThreads, 0, s.stream>>>(a, n, ptr<uint64_t>(m.dstart),
                                                                             ptr<uint32_t>(m.lvl[l]));
  k_many_counts<<<grid_for(m.G + 1, kThreads, 64), kThreads, 0, s.stream>>>(a, ptr<uint64_t>(m.dstart), m.G,
                                                                             ptr<unsigned long long>(m.cnt));
  if (!(st = cuda_check(cudaGetLastError(), "per-graph renumbering")).ok()) return st;
  std::vector<uint64_t> c(m.G + 1);
  st = cuda_check(cudaMemcpyAsync(c.data(), m.cnt.p, (m.G + 1) * 8, cudaMemcpyDeviceToHost, s.stream), "counts");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  uint32_t e = 0;
  st = cuda_check(cudaMemcpy(&e, s.d_err.p, 4, cudaMemcpyDeviceToHost), "error flags");
  if (!st.ok()) return st;
  if (e & kErrProbe) return Status::Err(KBISIM_ERR_TIMEOUT, "hash table probe bound exceeded");
  if (m.counts.size() < (size_t)l + 1) m.counts.resize(l + 1);
  m.counts[l].resize(m.G);
  for (uint32_t j = 0; j < m.G; ++j) m.counts[l][j] = c[j + 1] - c[j];
  m.levels = l + 1;
  return many_work_list(s, l);
}

Status many_check_args(const kbisim_graph* g, const uint64_t* start, uint32_t G, const uint32_t* k,
                       uint32_t* kmax_out) {
  if (!g || !start || !k || G == 0) return Status::Err(KBISIM_ERR_INVALID_ARG, "graph, starts and k are required");
  if (start[0] != 0 || start[G] != g->num_nodes)
    return Status::Err(KBISIM_ERR_INVALID_ARG, "graph_start must run from 0 to num_nodes");
  uint32_t kmax = 0;
  for (uint32_t j = 0; j < G; ++j) {
    if (start[j + 1] < start[j]) return Status::Err(KBISIM_ERR_INVALID_ARG, "graph_start must not decrease");
    if (k[j] > KBISIM_MAX_K) return Status::Err(KBISIM_ERR_INVALID_ARG, "k too large");
    kmax = std::max(kmax, k[j]);
  }
  *kmax_out = kmax;
  return Status::Ok();
}

// After the union is loaded: graph of every node, and no edge between graphs.
Status many_setup(Store& s, const uint64_t* start, uint32_t G, const uint32_t* k) {
  ManyState& m = s.many;
  m.valid = false;
  m.levels = 0;
  m.counts.clear();
  m.G = G;
  m.start.assign(start, start + G + 1);
  m.k.assign(k, k + G);
  const uint64_t n = s.n;
  Status st;
  if (!(st = ensure(s, m.dstart, (G + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, m.gid, std::max<uint64_t>(n, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, m.gidp, std::max<uint64_t>(n, 1) * 4)).ok()) return st;
  cudaMemcpyAsync(m.dstart.p, m.start.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s.stream);
  cudaMemsetAsync(s.d_err.p, 0, 4, s.stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device);
  if (sms <= 0) sms = 132;
  if (n) {
    k_many_gid<<<grid_for(n, kThreads, sms * 16), kThreads, 0, s.stream>>>(n, ptr<uint64_t>(m.dstart), G,
                                                                            ptr<uint32_t>(m.gid));
    k_many_check<<<(unsigned)sms * 16, kThreads, 0, s.stream>>>(n, ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst),
                                                                 ptr<uint32_t>(s.p2o), ptr<uint32_t>(m.gid),
                                                                 ptr<uint32_t>(m.gidp), ptr<uint32_t>(s.d_err));
  }
  uint32_t e = 0;
  st = cuda_check(cudaGetLastError(), "graph ids");
  if (st.ok()) st = cuda_check(cudaMemcpyAsync(&e, s.d_err.p, 4, cudaMemcpyDeviceToHost, s.stream), "check");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  if (e) return Status::Err(KBISIM_ERR_INVALID_ARG, "an edge joins two graphs of the batch");
  return Status::Ok();
}

// Per-graph rounds (early stop on the graph's own counts) after the union run.
void many_finish(Store& s) {
  ManyState& m = s.many;
  m.rounds.assign(m.G, 0);
  for (uint32_t j = 0; j < m.G; ++j) {
    uint32_t r = m.k[j];
    if (s.early_stop)
      for (uint32_t i = 1; i <= m.k[j] && i < m.levels; ++i)
        if (m.counts[i][j] == m.counts[i - 1][j]) {
          r = i;
          break;
        }
    m.rounds[j] = r;
  }
  m.valid = true;
}

Status many_pids(Store& s, uint32_t j, uint32_t level, uint32_t* dst, bool dst_on_device) {
  const ManyState& m = s.many;
  if (!m.valid) return Status::Err(KBISIM_ERR_STATE, "no batched result");
  if (j >= m.G || level > m.k[j] || !dst) return Status::Err(KBISIM_ERR_INVALID_ARG, "bad graph or level");
  const uint32_t l = std::min<uint32_t>(std::min(level, m.rounds[j]), m.levels - 1);
  const uint64_t nj = m.start[j + 1] - m.start[j];
  if (!nj) return Status::Ok();
  Status st = cuda_check(cudaMemcpyAsync(dst, ptr<uint32_t>(m.lvl[l]) + m.start[j], nj * 4,
                                         dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                         s.stream), "copy out");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  return st;
}

Status many_info(const Store& s, uint32_t j, uint32_t* rounds_run, uint64_t* counts) {
  const ManyState& m = s.many;
  if (!m.valid) return Status::Err(KBISIM_ERR_STATE, "no batched result");
  if (j >= m.G) return Status::Err(KBISIM_ERR_INVALID_ARG, "bad graph");
  if (rounds_run) *rounds_run = m.rounds[j];
  if (counts)
    for (uint32_t l = 0; l <= m.k[j]; ++l)
      counts[l] = m.counts[std::min<uint32_t>(std::min(l, m.rounds[j]), m.levels - 1)][j];
  return Status::Ok();
}

void many_release(Store& s) {
  ManyState& m = s.many;
  for (Buf& b : m.lvl) release(s, b);
  m.lvl.clear();
  Buf* bufs[] = {&m.dstart, &m.gid, &m.gidp, &m.tkey, &m.tmin, &m.slot, &m.hbits, &m.hword, &m.cnt, &m.live,
                 &m.live_mask};
  for (Buf* b : bufs) release(s, *b);
  m.valid = false;
}

}  // namespace kb
