// C ABI of libkbisim (declared in include/kbisim.h): handles, graph loading
// (CSR build on the device), refinement, extension, copy-out.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kbisim_internal.cuh"

struct kbisim_handle {
  kb::Store s;
  std::string last_error;
};

namespace kb {

Status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return Status::Ok();
  return Status::Err(e == cudaErrorMemoryAllocation ? KBISIM_ERR_OUT_OF_MEMORY : KBISIM_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

// Test hooks, read from the environment at the start of every call that
// computes (the library's own fault injection: nothing here touches a GPU
// setting or makes a kernel fail):
//   KBISIM_FAULT_ALLOC=N          the call's (N+1)-th device allocation fails
//                                 with KBISIM_ERR_OUT_OF_MEMORY;
//   KBISIM_FAULT_TIMEOUT_ROUND=r  round r reports KBISIM_ERR_TIMEOUT, as a
//                                 bounded device loop that gave up would;
//   KBISIM_FAULT_CORRUPT_DST=1    with options.checked only: one stored edge
//                                 target is set to num_nodes (one past the
//                                 last node) before each round, which the
//                                 checked-mode index check must report;
//   KBISIM_FAULT_STORE_ROOM=W     the signature stores of maintenance are
//                                 built with W pool words of room (default
//                                 4M), so that the next updates grow them.
void read_fault_hooks(Store& s) {
  const char* a = std::getenv("KBISIM_FAULT_ALLOC");
  s.fault_alloc = (a && *a) ? std::strtol(a, nullptr, 10) : -1;
  const char* t = std::getenv("KBISIM_FAULT_TIMEOUT_ROUND");
  s.fault_timeout_round = (t && *t) ? (uint32_t)std::strtoul(t, nullptr, 10) : 0u;
  const char* c = std::getenv("KBISIM_FAULT_CORRUPT_DST");
  s.fault_corrupt_dst = s.checked && c && *c == '1';
  const char* r = std::getenv("KBISIM_FAULT_STORE_ROOM");
  s.store_room = (r && *r) ? (uint64_t)std::strtoull(r, nullptr, 10) : (uint64_t)(4u << 20);
}

Status ensure(Store& s, Buf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return Status::Ok();
  size_t want = std::max<size_t>(bytes, 256);
  if (s.budget && s.bytes_held - b.cap + want > s.budget) {
    trim_caches(s);  // may release b too: it is reallocated below
    if (s.bytes_held - b.cap + want > s.budget)
      return Status::Err(KBISIM_ERR_BUDGET, "device memory budget exceeded");
  }
  if (s.fault_alloc >= 0 && s.fault_alloc-- == 0)
    return Status::Err(KBISIM_ERR_OUT_OF_MEMORY, "injected allocation failure (KBISIM_FAULT_ALLOC)");
  if (b.p) {
    cudaStreamSynchronize(s.stream);
    cudaFree(b.p);
    s.bytes_held -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return Status::Err(KBISIM_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(want) + " bytes failed");
  }
  b.p = p;
  b.cap = want;
  s.bytes_held += want;
  return Status::Ok();
}

void release(Store& s, Buf& b) {
  if (b.p) {
    cudaFree(b.p);
    s.bytes_held -= b.cap;
  }
  b.p = nullptr;
  b.cap = 0;
}

void trim_caches(Store& s) {
  const uint32_t u = s.busy;
  if (!(u & kCacheStage))
    for (Buf& b : s.stage) release(s, b);
  if (!(u & kCacheUpd))
    for (Buf& b : s.upd) release(s, b);
  if (!(u & kCacheInplace))
    for (Buf& b : s.inplace) release(s, b);
  if (!(u & kCacheRelabel)) {
    release(s, s.rl_tcnt);
    release(s, s.rl_hot);
    release(s, s.rl_ost);
  }
  if (!(u & kCacheSpare)) {
    for (Buf& b : s.spare_level) release(s, b);
    s.spare_level.clear();
    release(s, s.spare_alone);
  }
  // copies in original order whose results are no longer valid
  for (size_t l = 0; l < s.out_level.size(); ++l)
    if (!(l < s.out_valid.size() && s.out_valid[l])) release(s, s.out_level[l]);
  if (!(u & kCacheMaint)) maint_release(s);
}

namespace {

template <typename T>
T* ptr(Buf& b) { return static_cast<T*>(b.p); }

// Grid of a grid-stride loop over `work` items, `per` per CTA: at most 32
// CTAs per multiprocessor of the handle's device.
unsigned grid(const Store& s, uint64_t work, unsigned per) {
  uint64_t g = (work + per - 1) / per;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)s.sms * 32));
}

// --- load kernels -----------------------------------------------------------
// Every id < n.  Four ids per load when the array is 16-byte aligned.
__global__ void k_check_ids(uint64_t m, uint64_t n, const uint32_t* a, uint32_t* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  bool bad = false;
  uint64_t head = 0;
  if ((reinterpret_cast<uintptr_t>(a) & 15) == 0) {
    const uint64_t m4 = m / 4;
    const uint4* a4 = reinterpret_cast<const uint4*>(a);
    for (uint64_t i = t0; i < m4; i += stride) {
      const uint4 v = a4[i];
      bad |= (v.x >= n) | (v.y >= n) | (v.z >= n) | (v.w >= n);
    }
    head = m4 * 4;
  }
  for (uint64_t e = head + t0; e < m; e += stride) bad |= a[e] >= n;
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrBadInput);
}

__global__ void k_check_offsets(uint64_t n, uint64_t m, const uint64_t* off, uint32_t* err) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = off[u], b = off[u + 1];
    if (b < a || b - a > 0x7FFFFFFFull) atomicOr(err, kErrBadInput);
    if (u == 0 && a != 0) atomicOr(err, kErrBadInput);
    if (u == n - 1 && b != m) atomicOr(err, kErrBadInput);
  }
}

// Largest label.  16 bytes per load when the array is 16-byte aligned (byte
// or half-word maxima by SIMD-in-register max, __vmaxu4 / __vmaxu2).
template <typename T>
__global__ void k_label_max(uint64_t m, const T* lab, unsigned int* mx) {
  unsigned int v = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t head = 0;
  if ((reinterpret_cast<uintptr_t>(lab) & 15) == 0) {
    constexpr uint64_t kPer = 16 / sizeof(T);
    const uint64_t mv = m / kPer;
    const uint4* l4 = reinterpret_cast<const uint4*>(lab);
    unsigned int w = 0;
    for (uint64_t i = t0; i < mv; i += stride) {
      const uint4 q = l4[i];
      if (sizeof(T) == 1) w = __vmaxu4(w, __vmaxu4(__vmaxu4(q.x, q.y), __vmaxu4(q.z, q.w)));
      else if (sizeof(T) == 2) w = __vmaxu2(w, __vmaxu2(__vmaxu2(q.x, q.y), __vmaxu2(q.z, q.w)));
      else w = max(w, max(max(q.x, q.y), max(q.z, q.w)));
    }
    if (sizeof(T) == 1) v = max(max(w & 0xFF, (w >> 8) & 0xFF), max((w >> 16) & 0xFF, w >> 24));
    else if (sizeof(T) == 2) v = max(w & 0xFFFF, w >> 16);
    else v = w;
    head = mv * kPer;
  }
  for (uint64_t e = head + t0; e < m; e += stride)
    v = max(v, (unsigned int)lab[e]);
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, v);
}

__global__ void k_degree_count(uint64_t m, const uint32_t* src, unsigned long long* deg) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[src[e]], 1ull);
}

// Exclusive prefix sum in place: per-tile sums, a one-CTA scan of the tile
// sums, then tile scans.
constexpr int kT = 1024, kI = 4, kTile = kT * kI;

__global__ void __launch_bounds__(kT) k_tsum(const unsigned long long* a, uint64_t n, unsigned long long* bs) {
  __shared__ unsigned long long red[kT / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  unsigned long long c = 0;
  for (int t = 0; t < kI; ++t) {
    const uint64_t i = base + (uint64_t)t * kT + threadIdx.x;
    if (i < n) c += a[i];
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < kT / 32; ++w) tot += red[w];
    bs[blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(kT) k_tscan1(unsigned long long* bs, uint64_t nb) {
  __shared__ unsigned long long wt[kT / 32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nb; base += kT) {
    const uint64_t i = base + threadIdx.x;
    const unsigned long long v = i < nb ? bs[i] : 0ull;
    unsigned long long x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long t = wt[lane], xx = t;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, xx, o);
        if (lane >= o) xx += y;
      }
      wt[lane] = xx - t;
    }
    __syncthreads();
    const unsigned long long c0 = carry;
    if (i < nb) bs[i] = c0 + wt[w] + x - v;
    __syncthreads();
    if (threadIdx.x == kT - 1) carry = c0 + wt[w] + x;
    __syncthreads();
  }
}

// exclusive scan of a[0..n) written in place; optional copy
__global__ void __launch_bounds__(kT) k_tscan2(unsigned long long* a, uint64_t n, const unsigned long long* bs,
                                              unsigned long long* copy) {
  __shared__ unsigned long long wt[kT / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kI;
  unsigned long long f[kI], c = 0;
  for (int t = 0; t < kI; ++t) {
    f[t] = base + t < n ? a[base + t] : 0ull;
    c += f[t];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = c;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = wt[lane], xx = t;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, xx, o);
      if (lane >= o) xx += y;
    }
    wt[lane] = xx - t;
  }
  __syncthreads();
  unsigned long long run = bs[blockIdx.x] + wt[w] + (x - c);
  for (int t = 0; t < kI; ++t) {
    if (base + t < n) {
      a[base + t] = run;
      if (copy) copy[base + t] = run;
    }
    run += f[t];
  }
}

Status exclusive_scan_u64(Store& s, unsigned long long* a, uint64_t n, unsigned long long* copy, Buf& tmp) {
  if (!n) return Status::Ok();
  const uint64_t tiles = (n + kTile - 1) / kTile;
  Status st = ensure(s, tmp, tiles * 8);
  if (!st.ok()) return st;
  unsigned long long* bs = ptr<unsigned long long>(tmp);
  k_tsum<<<(unsigned)tiles, kT, 0, s.stream>>>(a, n, bs);
  k_tscan1<<<1, kT, 0, s.stream>>>(bs, tiles);
  k_tscan2<<<(unsigned)tiles, kT, 0, s.stream>>>(a, n, bs, copy);
  return cuda_check(cudaGetLastError(), "scan");
}

// Drop the graph and its levels.  With keep_buffers (a handle without an HBM
// budget, between loads) the device buffers stay allocated for the next graph.
void free_graph(Store& s, bool keep_buffers) {
  Buf* bufs[] = {&s.offsets, &s.dst, &s.elabel, &s.nlabel, &s.p2o, &s.o2p, &s.mid_chunks, &s.hub_bits,
                 &s.hub_bbase, &s.hub_cap, &s.hub_tbase, &s.hub_chunks, &s.hub_cstart, &s.sigkey, &s.ucnt, &s.hash, &s.table,
                 &s.slot, &s.rep, &s.ulist[0], &s.ulist[1], &s.hbits, &s.member, &s.alone, &s.hword, &s.bsum,
                 &s.long_pairs, &s.hub_cursor, &s.bucket_hub, &s.hub_acc, &s.hub_mode, &s.hub_force, &s.hub_err, &s.hub_retry, &s.hub_tmp, &s.alive_o,
                 &s.rl_tcnt, &s.rl_hot, &s.rl_ost};
  if (!keep_buffers) {
    for (Buf* b : bufs) release(s, *b);
    release(s, s.spare_alone);
    for (Buf& b : s.spare_level) release(s, b);
    s.spare_level.clear();
    for (Buf& b : s.level) release(s, b);
    for (Buf& b : s.out_level) release(s, b);
    for (Buf& b : s.stage) release(s, b);
    for (Buf& b : s.upd) release(s, b);
    for (Buf& b : s.inplace) release(s, b);
    s.level.clear();
    s.out_level.clear();
  }
  for (size_t i = 0; i < s.out_valid.size(); ++i) s.out_valid[i] = false;
  s.counts.clear();
  s.stats.clear();
  s.has_graph = false;
  s.has_levels = false;
  s.stable = false;
  s.any_dead = false;
  s.computed = 0;
  s.n = s.m = s.n_alive = 0;
  s.n_hub = 0;
  kb::maint_release(s);
  s.many.valid = false;
  s.many.levels = 0;
}

Status copy_in(Store& s, void* dstp, const void* srcp, size_t bytes, bool on_device) {
  if (!bytes) return Status::Ok();
  return cuda_check(cudaMemcpyAsync(dstp, srcp, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                                  : cudaMemcpyHostToDevice, s.stream),
                    "copy in");
}

template <typename T>
__global__ void k_place_coo(uint64_t m, const uint32_t* src, const uint32_t* dst_in, const T* lab_in,
                            unsigned long long* cursor, uint32_t* dst_out, T* lab_out) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = atomicAdd(&cursor[src[e]], 1ull);
    dst_out[p] = dst_in[e];
    lab_out[p] = lab_in[e];
  }
}

uint32_t bits_needed(uint64_t v) {  // bits for values 0..v
  uint32_t b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

// Staging buffers of a load (host inputs, COO grouping), kept in the store
// between loads.
struct Temps {
  InUse use;
  Buf* b;
  explicit Temps(Store& st) : use(st, kCacheStage), b(st.stage) {}
};

// The side stream and its two events, made once per handle.
Status ensure_side(Store& s) {
  if (s.side) return Status::Ok();
  Status st = cuda_check(cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking), "side stream");
  if (st.ok()) st = cuda_check(cudaEventCreateWithFlags(&s.ev_copied, cudaEventDisableTiming), "event");
  if (st.ok()) st = cuda_check(cudaEventCreateWithFlags(&s.ev_labels, cudaEventDisableTiming), "event");
  if (!st.ok()) {
    if (s.ev_copied) cudaEventDestroy(s.ev_copied);
    if (s.side) cudaStreamDestroy(s.side);
    s.ev_copied = nullptr;
    s.side = nullptr;
  }
  return st;
}

// The handle's stream waits for the edge labels copied on the side stream;
// their maximum then decides the label width.
Status await_side_labels(Store& s) {
  Status st = cuda_check(cudaStreamWaitEvent(s.stream, s.ev_labels, 0), "wait for labels");
  unsigned int maxlab = 0;
  if (st.ok())
    st = cuda_check(cudaMemcpyAsync(&maxlab, s.lab_max_dev, 4, cudaMemcpyDeviceToHost, s.stream), "label max");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  s.label8 = maxlab < 256;
  s.label_bits = bits_needed(maxlab);
  return Status::Ok();
}

// Load: bring the graph to the device as a CSR in original ids (copying host
// inputs, or grouping COO edges by source with a counting sort), validate it,
// then relabel it into the store's internal layout.
Status load_graph(Store& s, const kbisim_graph* g) {
  if (!g) return Status::Err(KBISIM_ERR_INVALID_ARG, "graph is NULL");
  const uint64_t n = g->num_nodes, m = g->num_edges;
  const uint32_t w = g->edge_label_bytes;
  if (n >= 0xFFFFFFFFull) return Status::Err(KBISIM_ERR_INVALID_ARG, "num_nodes must be < 2^32 - 1");
  if (w != 1 && w != 2 && w != 4) return Status::Err(KBISIM_ERR_INVALID_ARG, "edge_label_bytes must be 1, 2 or 4");
  if (n && !g->node_label) return Status::Err(KBISIM_ERR_INVALID_ARG, "node_label is NULL");
  if (m && (!g->dst || !g->edge_label)) return Status::Err(KBISIM_ERR_INVALID_ARG, "dst/edge_label is NULL");
  if (m && !g->offsets && !g->src) return Status::Err(KBISIM_ERR_INVALID_ARG, "need offsets or src");
  if (m && !n) return Status::Err(KBISIM_ERR_INVALID_ARG, "edges without nodes");
  // the hubs' bucket growth of the graph held now, for hubs of the same
  // original id and out-degree in the new one (a graph loaded again)
  if (s.side) cudaStreamSynchronize(s.side);  // a failed load's label copy may still run
  HubGrowth growth;
  Status gs = save_hub_growth(s, &growth);
  if (!gs.ok()) growth = HubGrowth();
  free_graph(s, s.budget == 0);
  Status st;
  const bool dev = g->on_device != 0;
  if (!(st = ensure(s, s.d_err, 64)).ok()) return st;
  cudaMemsetAsync(s.d_err.p, 0, 64, s.stream);
  uint32_t* err = ptr<uint32_t>(s.d_err);
  Temps t(s);
  Buf &off_b = t.b[0], &dst_b = t.b[1], &lab_b = t.b[2], &nlab_b = t.b[3], &src_b = t.b[4], &cur_b = t.b[5],
      &scan_b = t.b[6];
  // node labels
  const uint32_t* nlab0 = g->node_label;
  if (!dev && n) {
    if (!(st = ensure(s, nlab_b, n * 4)).ok()) return st;
    if (!(st = copy_in(s, nlab_b.p, g->node_label, n * 4, false)).ok()) return st;
    nlab0 = ptr<uint32_t>(nlab_b);
  }
  // edge labels and targets as given
  const void* lab_in = g->edge_label;
  const uint32_t* dst_in = g->dst;
  const uint32_t* src_in = g->src;
  // host CSR input: the edge labels are copied last, on the side stream, so
  // that the copy overlaps the validation and the node phase of the
  // relabelling (which need targets and offsets only)
  const bool overlap = !dev && m && g->offsets && ensure_side(s).ok();
  if (!dev && m) {
    if (!(st = ensure(s, lab_b, m * w)).ok()) return st;
    if (!overlap && !(st = copy_in(s, lab_b.p, g->edge_label, m * w, false)).ok()) return st;
    lab_in = lab_b.p;
    if (!(st = ensure(s, dst_b, m * 4)).ok()) return st;
    if (!(st = copy_in(s, dst_b.p, g->dst, m * 4, false)).ok()) return st;
    dst_in = ptr<uint32_t>(dst_b);
    if (!g->offsets) {
      if (!(st = ensure(s, src_b, m * 4)).ok()) return st;
      if (!(st = copy_in(s, src_b.p, g->src, m * 4, false)).ok()) return st;
      src_in = ptr<uint32_t>(src_b);
    }
  }
  unsigned int* d_max = reinterpret_cast<unsigned int*>(err + 4);
  // offsets in original ids
  const uint64_t* off0 = g->offsets;
  if (g->offsets && !dev) {
    if (!(st = ensure(s, off_b, (n + 1) * 8)).ok()) return st;
    if (!(st = copy_in(s, off_b.p, g->offsets, (n + 1) * 8, false)).ok()) return st;
    off0 = ptr<uint64_t>(off_b);
  }
  auto label_max = [&](cudaStream_t q) {
    const unsigned gb = grid(s, m, 256);
    if (w == 1) k_label_max<uint8_t><<<gb, 256, 0, q>>>(m, static_cast<const uint8_t*>(lab_in), d_max);
    else if (w == 2) k_label_max<uint16_t><<<gb, 256, 0, q>>>(m, static_cast<const uint16_t*>(lab_in), d_max);
    else k_label_max<uint32_t><<<gb, 256, 0, q>>>(m, static_cast<const uint32_t*>(lab_in), d_max);
  };
  if (overlap) {  // after the copies on the handle's stream: labels, then their maximum
    cudaEventRecord(s.ev_copied, s.stream);
    cudaStreamWaitEvent(s.side, s.ev_copied, 0);
    st = cuda_check(cudaMemcpyAsync(lab_b.p, g->edge_label, m * w, cudaMemcpyHostToDevice, s.side), "copy in");
    if (!st.ok()) return st;
    label_max(s.side);
    cudaEventRecord(s.ev_labels, s.side);
  }
  if (m) {
    if (!overlap) label_max(s.stream);
    k_check_ids<<<grid(s, m, 256), 256, 0, s.stream>>>(m, n, dst_in, err);
    if (!g->offsets) k_check_ids<<<grid(s, m, 256), 256, 0, s.stream>>>(m, n, src_in, err);
  }
  if (g->offsets && n) k_check_offsets<<<grid(s, n, 256), 256, 0, s.stream>>>(n, m, off0, err);
  uint32_t hv[8] = {0};
  if (!(st = cuda_check(cudaMemcpyAsync(hv, err, 32, cudaMemcpyDeviceToHost, s.stream), "validate")).ok()) return st;
  if (!(st = cuda_check(cudaStreamSynchronize(s.stream), "sync")).ok()) return st;
  if (hv[0]) return Status::Err(KBISIM_ERR_INVALID_ARG, "invalid graph: node id >= num_nodes or bad offsets");
  const unsigned int maxlab = hv[4];  // (with the side copy: read again by await_side_labels)
  if (!g->offsets) {
    // COO: counting sort by source into temporary CSR buffers
    Buf &csr_dst = t.b[7], &csr_lab = t.b[8];
    if (!(st = ensure(s, off_b, (n + 1) * 8)).ok()) return st;
    if (!(st = ensure(s, cur_b, (n + 1) * 8)).ok()) return st;
    unsigned long long* off = ptr<unsigned long long>(off_b);
    cudaMemsetAsync(off, 0, (n + 1) * 8, s.stream);
    if (m) k_degree_count<<<grid(s, m, 256), 256, 0, s.stream>>>(m, src_in, off);
    if (!(st = exclusive_scan_u64(s, off, n + 1, ptr<unsigned long long>(cur_b), scan_b)).ok()) return st;
    off0 = ptr<uint64_t>(off_b);
    if (m) {
      if (!(st = ensure(s, csr_dst, m * 4)).ok()) return st;
      if (!(st = ensure(s, csr_lab, m * w)).ok()) return st;
      const unsigned gb = grid(s, m, 256);
      unsigned long long* cur = ptr<unsigned long long>(cur_b);
      if (w == 1)
        k_place_coo<uint8_t><<<gb, 256, 0, s.stream>>>(m, src_in, dst_in, static_cast<const uint8_t*>(lab_in), cur,
                                                       ptr<uint32_t>(csr_dst), ptr<uint8_t>(csr_lab));
      else if (w == 2)
        k_place_coo<uint16_t><<<gb, 256, 0, s.stream>>>(m, src_in, dst_in, static_cast<const uint16_t*>(lab_in),
                                                        cur, ptr<uint32_t>(csr_dst), ptr<uint16_t>(csr_lab));
      else
        k_place_coo<uint32_t><<<gb, 256, 0, s.stream>>>(m, src_in, dst_in, static_cast<const uint32_t*>(lab_in),
                                                        cur, ptr<uint32_t>(csr_dst), ptr<uint32_t>(csr_lab));
      st = cuda_check(cudaGetLastError(), "place edges");
      if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
      if (!st.ok()) return st;
      // the grouped copies replace the staged ones
      std::swap(dst_b, csr_dst);
      std::swap(lab_b, csr_lab);
      dst_in = ptr<uint32_t>(dst_b);
      lab_in = lab_b.p;
    }
  }
  s.n = n;
  s.m = m;
  s.label8 = maxlab < 256;
  s.label_bits = bits_needed(maxlab);
  if (overlap) {
    s.await_labels = await_side_labels;
    s.lab_max_dev = d_max;
  }
  st = relabel_graph(s, off0, dst_in, lab_in, nlab0, nullptr, w);
  s.await_labels = nullptr;
  if (overlap) cudaStreamSynchronize(s.side);  // (done already unless the relabelling failed early)
  if (!st.ok()) {
    free_graph(s, s.budget == 0);
    return st;
  }
  s.has_graph = true;
  return restore_hub_growth(s, growth, true);
}

Status ensure_levels(Store& s, uint32_t k) {
  if (s.level.size() < (size_t)k + 1) s.level.resize(k + 1);
  for (uint32_t i = 0; i <= k; ++i) {
    Status st = ensure(s, s.level[i], std::max<uint64_t>(s.n, 1) * 4);
    if (!st.ok()) return st;
  }
  if (s.counts.size() < (size_t)k + 1) s.counts.resize(k + 1, 0);
  return Status::Ok();
}

void invalidate_outputs(Store& s) {
  for (size_t i = 0; i < s.out_valid.size(); ++i) s.out_valid[i] = false;
}

// Original-order copy of level l (kept until the levels change).
Status materialize_level(Store& s, uint32_t l) {
  if (s.out_level.size() < s.level.size()) {
    s.out_level.resize(s.level.size());
    s.out_valid.resize(s.level.size(), false);
  }
  if (s.out_valid[l]) return Status::Ok();
  Status st = ensure(s, s.out_level[l], std::max<uint64_t>(s.n, 1) * 4);
  if (!st.ok()) return st;
  if (!(st = unpermute_level(s, l, ptr<uint32_t>(s.out_level[l]))).ok()) return st;
  s.out_valid[l] = true;
  return Status::Ok();
}

void fill_result(Store& s, uint32_t k, kbisim_result* out) {
  s.k_requested = k;
  if (s.counts.size() < (size_t)k + 1) s.counts.resize(k + 1, 0);
  for (uint32_t j = s.computed + 1; j <= k; ++j) s.counts[j] = s.counts[s.computed];
  if (out) {
    out->k_requested = k;
    out->rounds_run = s.rounds_run;
    out->block_count = s.counts.data();
  }
}

// Run rounds from + 1 .. k (levels up to `from` exist).
Status run_rounds(Store& s, uint32_t from, uint32_t k) {
  Status st;
  for (uint32_t i = from + 1; i <= k; ++i) {
    if (s.early_stop && s.stable) break;
    if (!(st = compute_round(s, i)).ok()) return st;
    s.computed = i;
    s.rounds_run = i;
    if (s.level_hook && !(st = s.level_hook(s, i)).ok()) return st;
    if (s.counts[i] == s.counts[i - 1]) {
      s.stable = true;
      if (s.early_stop) break;
    }
  }
  return Status::Ok();
}

// Host side of a computed result; with the level buffers and the alone flags
// it is what a failed call puts back.
struct LevelSnapshot {
  std::vector<uint64_t> counts;
  std::vector<kbisim_round_stats> stats;
  uint32_t computed, rounds_run, k_requested;
  bool stable, has_levels;
  uint64_t n_alone;
};

LevelSnapshot take_snapshot(const Store& s) {
  return LevelSnapshot{s.counts, s.stats, s.computed, s.rounds_run, s.k_requested, s.stable, s.has_levels,
                       s.n_alone};
}

void put_back(Store& s, LevelSnapshot& p) {
  s.counts.swap(p.counts);
  s.stats.swap(p.stats);
  s.computed = p.computed;
  s.rounds_run = p.rounds_run;
  s.k_requested = p.k_requested;
  s.stable = p.stable;
  s.has_levels = p.has_levels;
  s.n_alone = p.n_alone;
}

// The levels of an incremental update are in place: result and outputs.
Status finish_incremental(Store& s, uint32_t k, kbisim_result* out) {
  invalidate_outputs(s);
  fill_result(s, k, out);
  return timer_collect(s);
}

Status refine_levels(Store& s, uint32_t k) {
  Status st;
  if (!(st = ensure_levels(s, s.early_stop ? std::min<uint32_t>(k, 1) : k)).ok()) return st;
  if (!(st = compute_level0(s)).ok()) return st;
  if (s.level_hook && !(st = s.level_hook(s, 0)).ok()) return st;
  for (uint32_t i = 1; i <= k; ++i) {
    if (s.early_stop && s.stable) break;
    if (!(st = ensure_levels(s, i)).ok()) return st;
    if (!(st = run_rounds(s, i - 1, i)).ok()) return st;
  }
  return Status::Ok();
}

// Levels 0..k of the loaded graph.  The new levels are computed into spare
// buffers; the current result (level buffers, alone flags, counts) is set
// aside and put back if the call fails, so a failed refinement leaves the
// previous result readable.
Status refine(Store& s, uint32_t k, kbisim_result* out) {
  if (!s.has_graph) return Status::Err(KBISIM_ERR_STATE, "no graph loaded");
  if (k > KBISIM_MAX_K) return Status::Err(KBISIM_ERR_INVALID_ARG, "k too large");
  InUse use(s, kCacheSpare);
  LevelSnapshot snap = take_snapshot(s);
  std::swap(s.level, s.spare_level);
  std::swap(s.alone, s.spare_alone);
  s.has_levels = false;
  s.stable = false;
  s.computed = 0;
  s.rounds_run = 0;
  s.stats.clear();
  s.counts.assign(std::max<size_t>(snap.counts.size(), 1), 0);
  Status st = refine_levels(s, k);
  if (!st.ok()) {
    std::swap(s.level, s.spare_level);
    std::swap(s.alone, s.spare_alone);
    put_back(s, snap);
    timer_collect(s);
    return st;
  }
  invalidate_outputs(s);
  s.has_levels = true;
  fill_result(s, k, out);
  return timer_collect(s);
}

// Change k.  Rounds past the computed level write new level buffers only; the
// alone flags and the host side are copied first and restored on failure.
Status extend(Store& s, uint32_t k_new, kbisim_result* out) {
  if (!s.has_levels) return Status::Err(KBISIM_ERR_STATE, "no computed levels");
  if (k_new > KBISIM_MAX_K) return Status::Err(KBISIM_ERR_INVALID_ARG, "k too large");
  InUse use(s, kCacheSpare);
  Status st;
  const bool need = k_new > s.computed && !(s.early_stop && s.stable);
  if (need) {
    if (!(st = ensure(s, s.spare_alone, s.n + 16)).ok()) return st;
    if (!(st = cuda_check(cudaMemcpyAsync(s.spare_alone.p, s.alone.p, s.n + 16, cudaMemcpyDeviceToDevice,
                                          s.stream), "save alone flags")).ok())
      return st;
    LevelSnapshot snap = take_snapshot(s);
    for (uint32_t i = s.computed + 1; i <= k_new && st.ok(); ++i) {
      if (s.early_stop && s.stable) break;
      st = ensure_levels(s, i);
      if (st.ok()) st = run_rounds(s, i - 1, i);
    }
    if (!st.ok()) {
      cudaMemcpyAsync(s.alone.p, s.spare_alone.p, s.n + 16, cudaMemcpyDeviceToDevice, s.stream);
      put_back(s, snap);
      timer_collect(s);
      return st;
    }
    invalidate_outputs(s);
  }
  fill_result(s, k_new, out);
  return timer_collect(s);
}

}  // namespace
}  // namespace kb

using kb::Status;

static int finish(kbisim_handle* h, const Status& st) {
  if (h) {
    h->last_error = st.ok() ? std::string() : st.msg;
    h->s.fault_alloc = -1;  // test hooks apply to one call only
    h->s.fault_timeout_round = 0;
    h->s.fault_corrupt_dst = false;
  }
  return st.code;
}

// Entry of a call that computes: device current, test hooks read.
static void enter(kbisim_handle* h) {
  cudaSetDevice(h->s.device);
  kb::read_fault_hooks(h->s);
}

extern "C" {

void kbisim_default_options(kbisim_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->stream = nullptr;
  opt->device = 0;
  opt->hbm_budget_bytes = 0;
  opt->early_stop = 1;
  opt->hash_seed = 0x12100748ull;
  opt->hash_bits = 64;
  opt->checked = 0;
  opt->collect_timing = 0;
  opt->maintain = 1;
  opt->hub_bucket_keys = 0;
}

int kbisim_create(kbisim_handle** h, const kbisim_options* opt) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  *h = nullptr;
  kbisim_options o;
  if (opt) o = *opt; else kbisim_default_options(&o);
  if (o.hash_bits == 0 || o.hash_bits > 64) return KBISIM_ERR_INVALID_ARG;
  if (o.maintain < 0 || o.maintain > 2) return KBISIM_ERR_INVALID_ARG;
  if (o.hub_bucket_keys != 0 && o.hub_bucket_keys != 2048 && o.hub_bucket_keys != 4096 && o.hub_bucket_keys != 8192)
    return KBISIM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return KBISIM_ERR_CUDA;
  }
  if (o.device < 0 || o.device >= ndev) return KBISIM_ERR_INVALID_ARG;
  if (cudaSetDevice(o.device) != cudaSuccess) return KBISIM_ERR_CUDA;
  kbisim_handle* p = new (std::nothrow) kbisim_handle();
  if (!p) return KBISIM_ERR_OUT_OF_MEMORY;
  kb::Store& s = p->s;
  s.device = o.device;
  if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess || s.sms < 1) {
    cudaGetLastError();
    s.sms = 1;
  }
  s.stream = static_cast<cudaStream_t>(o.stream);
  s.budget = o.hbm_budget_bytes;
  s.early_stop = o.early_stop != 0;
  s.seed = o.hash_seed;
  s.hash_mask = o.hash_bits >= 64 ? ~0ull : ((1ull << o.hash_bits) - 1ull);
  s.checked = o.checked != 0;
  s.timing = o.collect_timing != 0;
  s.maintain = o.maintain;
  if (o.hub_bucket_keys) {
    s.hub_ucap = o.hub_bucket_keys;
    s.hub_tune = 2;
  }
  void* hp = nullptr;
  if (cudaMallocHost(&hp, 16 * 8) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return KBISIM_ERR_CUDA;
  }
  s.h_scalars.p = hp;
  s.h_scalars.cap = 16 * 8;
  Status st = kb::ensure(s, s.d_scalars, 16 * 8);
  if (st.ok()) st = kb::ensure(s, s.d_err, 64);
  if (!st.ok()) {
    cudaFreeHost(hp);
    delete p;
    return st.code;
  }
  *h = p;
  return KBISIM_OK;
}

void kbisim_destroy(kbisim_handle* h) {
  if (!h) return;
  kb::Store& s = h->s;
  cudaSetDevice(s.device);
  cudaStreamSynchronize(s.stream);
  kb::free_graph(s, false);
  kb::many_release(s);
  kb::release(s, s.d_scalars);
  kb::release(s, s.d_err);
  if (s.h_scalars.p) cudaFreeHost(s.h_scalars.p);
  if (s.side) {
    cudaStreamSynchronize(s.side);
    cudaEventDestroy(s.ev_copied);
    cudaEventDestroy(s.ev_labels);
    cudaStreamDestroy(s.side);
  }
  kb::timer_destroy(s);
  delete h;
}

const char* kbisim_last_error(const kbisim_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

int kbisim_load(kbisim_handle* h, const kbisim_graph* g) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  enter(h);
  return finish(h, kb::load_graph(h->s, g));
}

int kbisim_refine(kbisim_handle* h, uint32_t k, kbisim_result* out) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  enter(h);
  return finish(h, kb::refine(h->s, k, out));
}

int kbisim_build_many(kbisim_handle* h, const kbisim_graph* g, const uint64_t* graph_start, uint32_t num_graphs,
                      const uint32_t* k) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  enter(h);
  kb::Store& s = h->s;
  uint32_t kmax = 0;
  Status st = kb::many_check_args(g, graph_start, num_graphs, k, &kmax);
  if (st.ok()) st = kb::load_graph(s, g);
  if (st.ok()) st = kb::many_setup(s, graph_start, num_graphs, k);
  if (st.ok()) {
    kbisim_result r;
    s.level_hook = kb::many_level;
    st = kb::refine(s, kmax, &r);
    s.level_hook = nullptr;
    s.round_mask = nullptr;
    if (st.ok()) kb::many_finish(s);
  }
  if (!st.ok()) s.many.valid = false;
  return finish(h, st);
}

int kbisim_many_pids(kbisim_handle* h, uint32_t graph, uint32_t level, uint32_t* dst, int dst_on_device) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  cudaSetDevice(h->s.device);
  return finish(h, kb::many_pids(h->s, graph, level, dst, dst_on_device != 0));
}

int kbisim_many_info(kbisim_handle* h, uint32_t graph, uint32_t* rounds_run, uint64_t* counts) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  return finish(h, kb::many_info(h->s, graph, rounds_run, counts));
}

int kbisim_build(kbisim_handle* h, const kbisim_graph* g, uint32_t k, kbisim_result* out) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  enter(h);
  Status st = kb::load_graph(h->s, g);
  if (st.ok()) st = kb::refine(h->s, k, out);
  return finish(h, st);
}

int kbisim_extend(kbisim_handle* h, uint32_t k_new, kbisim_result* out) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  enter(h);
  return finish(h, kb::extend(h->s, k_new, out));
}

int kbisim_pids(kbisim_handle* h, uint32_t level, uint32_t* dst, int dst_on_device) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  kb::Store& s = h->s;
  if (!s.has_levels) return finish(h, Status::Err(KBISIM_ERR_STATE, "no computed levels"));
  if (level > s.k_requested) return finish(h, Status::Err(KBISIM_ERR_INVALID_ARG, "level out of range"));
  if (!dst && s.n) return finish(h, Status::Err(KBISIM_ERR_INVALID_ARG, "dst is NULL"));
  cudaSetDevice(s.device);
  const uint32_t l = std::min(level, s.computed);
  Status st;
  if (dst_on_device) {
    st = kb::unpermute_level(s, l, dst);
  } else if (s.budget && s.hash.cap >= s.n * 4) {
    // a budget handle allocates nothing to read a level: the original-order
    // copy goes through the round scratch (the hash array, idle between calls)
    st = kb::unpermute_level(s, l, static_cast<uint32_t*>(s.hash.p));
    if (st.ok())
      st = kb::cuda_check(cudaMemcpyAsync(dst, s.hash.p, s.n * 4, cudaMemcpyDeviceToHost, s.stream), "copy out");
  } else {
    st = kb::materialize_level(s, l);
    if (st.ok())
      st = kb::cuda_check(cudaMemcpyAsync(dst, s.out_level[l].p, s.n * 4, cudaMemcpyDeviceToHost, s.stream),
                          "copy out");
  }
  if (st.ok()) st = kb::cuda_check(cudaStreamSynchronize(s.stream), "sync");
  return finish(h, st);
}

const uint32_t* kbisim_pids_device(kbisim_handle* h, uint32_t level) {
  if (!h || !h->s.has_levels || level > h->s.k_requested) return nullptr;
  kb::Store& s = h->s;
  cudaSetDevice(s.device);
  const uint32_t l = std::min(level, s.computed);
  Status st = kb::materialize_level(s, l);
  if (st.ok()) st = kb::cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) {
    h->last_error = st.msg;
    return nullptr;
  }
  return static_cast<const uint32_t*>(s.out_level[l].p);
}

uint64_t kbisim_num_nodes(const kbisim_handle* h) { return h ? h->s.n : 0; }
uint64_t kbisim_num_edges(const kbisim_handle* h) { return h ? h->s.m : 0; }
uint64_t kbisim_device_bytes(const kbisim_handle* h) { return h ? (uint64_t)h->s.bytes_held : 0; }

uint32_t kbisim_hub_bucket_keys(const kbisim_handle* h) { return h ? h->s.hub_ucap : 0u; }

int kbisim_set_hbm_budget(kbisim_handle* h, uint64_t bytes) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  h->s.budget = bytes;
  return KBISIM_OK;
}

int kbisim_get_update_info(const kbisim_handle* h, kbisim_update_info* out) {
  if (!h || !out) return KBISIM_ERR_INVALID_ARG;
  out->incremental = h->s.mt.incremental;
  out->reason = h->s.mt.reason;
  out->frontier_nodes = h->s.mt.frontier_nodes;
  out->levels = h->s.mt.levels;
  out->in_place = h->s.mt.in_place;
  return KBISIM_OK;
}

int kbisim_get_kernel_times(const kbisim_handle* h, kbisim_kernel_times* out) {
  if (!h || !out) return KBISIM_ERR_INVALID_ARG;
  for (int i = 0; i < KBISIM_KERNEL_COUNT; ++i) {
    out->total_ms[i] = h->s.total_ms[i];
    out->launches[i] = h->s.launches[i];
  }
  return KBISIM_OK;
}

void kbisim_reset_times(kbisim_handle* h) {
  if (!h) return;
  for (int i = 0; i < KBISIM_KERNEL_COUNT; ++i) {
    h->s.total_ms[i] = 0;
    h->s.launches[i] = 0;
  }
}

int kbisim_get_round_stats(const kbisim_handle* h, uint32_t round, kbisim_round_stats* out) {
  if (!h || !out) return KBISIM_ERR_INVALID_ARG;
  if (!h->s.has_levels) return KBISIM_ERR_STATE;
  if (round == 0 || round > h->s.stats.size()) return KBISIM_ERR_INVALID_ARG;
  *out = h->s.stats[round - 1];
  return KBISIM_OK;
}

int kbisim_update(kbisim_handle* h, const kbisim_batch* b, uint32_t k, kbisim_result* out,
                  uint64_t* missing_deletes) {
  if (!h) return KBISIM_ERR_INVALID_ARG;
  if (k > KBISIM_MAX_K) return finish(h, Status::Err(KBISIM_ERR_INVALID_ARG, "k too large"));
  enter(h);
  kb::Store& s = h->s;
  kb::MaintState& m = s.mt;
  kb::InUse use(s, kb::kCacheMaint);
  const auto t0 = std::chrono::steady_clock::now();
  auto ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
  };
  uint64_t missing = 0;
  Status st;
  bool done = false;
  m.incremental = 0;
  m.frontier_nodes = 0;
  m.levels = 0;
  m.in_place = 0;
  const uint64_t batch_edges = b ? b->n_ins + b->n_del : 0;
  const bool suspended = m.suspend_edges && k == m.suspend_k && batch_edges >= m.suspend_edges;
  // timed choice: after one update on each path, the frontier path runs only
  // while it measured cheaper; otherwise the next 16 updates recompute
  bool timed = s.maintain == 1;
  bool cost_off = false;
  if (timed && m.n_inc && m.n_rec && m.ms_inc > m.ms_rec) {
    if (m.cost_skip == 0) m.cost_skip = 16;
    cost_off = --m.cost_skip > 0;
  } else if (timed && m.n_inc && !m.n_rec) {
    cost_off = true;  // one recomputation to compare with
  }
  bool tried = false;  // the frontier path was attempted (its cost is charged to it)
  double entry_build_ms = 0;  // stores built for this update (a one-time cost, not charged)
  if (!s.maintain) {
    m.reason = KBISIM_MAINT_OFF;
  } else if (b && b->n_del_nodes) {
    m.reason = KBISIM_MAINT_DELETES;
  } else if (suspended) {
    // a batch at least this large already switched back at this k: recompute
    m.reason = KBISIM_MAINT_FRONTIER;
    kb::maint_invalidate(s);
  } else if (cost_off) {
    m.reason = KBISIM_MAINT_COST;
    kb::maint_invalidate(s);
  } else {
    // stores made from the current levels when there are none for this k yet
    if ((!m.valid || k > m.k) && s.has_levels && (s.k_requested >= k || s.stable)) {
      const auto tb = std::chrono::steady_clock::now();
      if (!kb::maint_build(s, k).ok()) kb::maint_release(s);
      entry_build_ms = ms_since(tb);
    }
    if (m.valid && k <= m.k) {
      tried = true;
      st = kb::maint_update(s, b, k, &missing, &done);
    } else {
      m.reason = KBISIM_MAINT_NO_STORE;
    }
  }
  if (st.ok() && !done) {
    kb::maint_invalidate(s);  // the graph changes under the stores
    st = kb::apply_batch(s, b, &missing);
  }
  if (st.ok()) st = m.incremental ? kb::finish_incremental(s, k, out) : kb::refine(s, k, out);
  if (m.incremental) {
    m.suspend_edges = 0;
  } else if (m.reason == KBISIM_MAINT_FRONTIER) {
    m.suspend_edges = std::max<uint64_t>(batch_edges, 1);
    m.suspend_k = k;
  }
  // per-update cost of the path taken; building the stores is a one-time
  // cost of the frontier path that later updates reuse, so it is not charged
  const double call_ms = ms_since(t0) - entry_build_ms;
  // after a full recomputation, stores for the next update (not while large
  // batches are known to switch back, nor while recomputation measures
  // cheaper: the update before the next trial of the frontier path makes them)
  const bool next_tries = !(m.reason == KBISIM_MAINT_COST && m.cost_skip > 1);
  if (st.ok() && s.maintain && !m.incremental && s.has_levels && m.reason != KBISIM_MAINT_FRONTIER &&
      next_tries) {
    if (!kb::maint_build(s, k).ok()) kb::maint_release(s);
  }
  if (st.ok() && timed) {
    const double per = 1.0 / std::max<uint32_t>(k, 1);
    auto fold = [](double& avg, uint32_t& n, double x) {
      avg = n ? 0.5 * (avg + x) : x;
      ++n;
    };
    if (tried || m.incremental) {
      // the handle's first frontier update allocates that path's scratch:
      // not a sample of its steady cost
      if (m.inc_warm) fold(m.ms_inc, m.n_inc, call_ms * per);
      m.inc_warm = true;
    }
    else if (m.reason == KBISIM_MAINT_COST || m.reason == KBISIM_MAINT_NO_STORE) fold(m.ms_rec, m.n_rec, call_ms * per);
  }
  if (st.ok() && missing_deletes) *missing_deletes = missing;
  return finish(h, st);
}

}  // extern "C"
