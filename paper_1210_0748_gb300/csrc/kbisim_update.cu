// Maintenance batches (paper Section 4: Add_Nodes, Add_Edges, deletions),
// applied on the device to the stored edge multiset, followed by a rebuild of
// the levels.  Theorem 2 states that the maintained partition is the
// k-bisimulation of the updated graph; recomputing it from the updated graph
// gives exactly that result (the paper's own validation compares Add_Edges
// with Build_Bisim the same way).
//
// Batch order: node additions (ids n, n+1, ... in batch order, isolated),
// edge insertions, edge deletions (one stored copy per listed triple; absent
// triples are counted), node deletions (incident edges removed, node marked
// deleted).  All steps are kernels:
//   1. the stored CSR (internal ids) and the inserted edges become one CSR
//      grouped by original source id (counting sort by source);
//   2. deletions are matched per source node: every source with deletions
//      gets a private open-addressing table of (target, label) -> count, and
//      one warp walks the source's edges claiming one stored copy per count;
//   3. edges on deleted nodes are dropped, the rest compacted per source;
//   4. the result is relabelled like a freshly loaded graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kbisim_internal.cuh"

namespace kb {
namespace {

template <typename T>
T* ptr(Buf& b) { return static_cast<T*>(b.p); }

// Grid of a grid-stride loop over `work` items, `per` per CTA: at most 32
// CTAs per multiprocessor of the handle's device.
unsigned grid(const Store& s, uint64_t work, unsigned per) {
  uint64_t g = (work + per - 1) / per;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)s.sms * 32));
}

#define GRID_STRIDE(i, n) \
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// Flags (bit) written into err[0] by validation kernels.
constexpr uint32_t kBadId = 1u, kDeadEnd = 2u;

__global__ void k_alive_init(uint64_t n0, uint64_t n1, const uint8_t* old_alive, uint8_t* alive) {
  GRID_STRIDE(o, n1) alive[o] = o < n0 ? (old_alive ? old_alive[o] : (uint8_t)1) : (uint8_t)1;
}

__global__ void k_check_inserts(uint64_t k, uint64_t n1, const uint32_t* s, const uint32_t* t, const uint8_t* alive,
                                uint32_t* err) {
  GRID_STRIDE(i, k) {
    if (s[i] >= n1 || t[i] >= n1) atomicOr(err, kBadId);
    else if (!alive[s[i]] || !alive[t[i]]) atomicOr(err, kDeadEnd);
  }
}

__global__ void k_check_ids_only(uint64_t k, uint64_t n1, const uint32_t* a, uint32_t* err) {
  GRID_STRIDE(i, k) if (a[i] >= n1) atomicOr(err, kBadId);
}

__global__ void k_check_node_dels(uint64_t k, uint64_t n1, const uint32_t* u, const uint8_t* alive, uint32_t* err) {
  GRID_STRIDE(i, k) {
    if (u[i] >= n1) atomicOr(err, kBadId);
    else if (!alive[u[i]]) atomicOr(err, kDeadEnd);
  }
}

// Degree of every original node in the stored graph, plus inserted edges.
__global__ void k_count_combined(uint64_t n0, const uint32_t* o2p, const uint64_t* off, uint64_t k,
                                 const uint32_t* ins_s, unsigned long long* cnt) {
  GRID_STRIDE(o, n0) cnt[o] = off[o2p[o] + 1] - off[o2p[o]];
}

__global__ void k_count_inserts(uint64_t k, const uint32_t* ins_s, unsigned long long* cnt) {
  GRID_STRIDE(i, k) atomicAdd(&cnt[ins_s[i]], 1ull);
}

// One warp per original node: copy its stored edges (targets back to
// original ids, labels widened) to the start of its combined segment.
template <typename LabelT>
__global__ void k_copy_stored(uint64_t n0, const uint32_t* o2p, const uint32_t* p2o, const uint64_t* off,
                              const uint32_t* dst, const LabelT* lab, const unsigned long long* coff,
                              unsigned long long* cursor, uint32_t* cdst, uint32_t* clab) {
  const int lane = threadIdx.x & 31;
  for (uint64_t o = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; o < n0;
       o += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t p = o2p[o];
    const uint64_t s0 = off[p], d = off[p + 1] - s0, c0 = coff[o];
    for (uint64_t i = lane; i < d; i += 32) {
      cdst[c0 + i] = p2o[dst[s0 + i]];
      clab[c0 + i] = (uint32_t)lab[s0 + i];
    }
    if (lane == 0) cursor[o] = c0 + d;
  }
}

__global__ void k_place_inserts(uint64_t k, const uint32_t* s, const uint32_t* t, const uint32_t* l,
                                unsigned long long* cursor, uint32_t* cdst, uint32_t* clab) {
  GRID_STRIDE(i, k) {
    const uint64_t q = atomicAdd(&cursor[s[i]], 1ull);
    cdst[q] = t[i];
    clab[q] = l[i];
  }
}

// Per-source deletion tables: region of 2^r >= 2 * (deletes of the source) slots.
// Slots start zeroed: key 0 = empty, stored keys are ((target << 32) | label) + 1
// (never 0 and never overflowing, since target < 2^32 - 1).
struct DelSlot {
  unsigned long long key;
  int count;
  int pad;
};

__global__ void k_count_deletes(uint64_t k, const uint32_t* s, uint64_t n1, unsigned long long* dcnt) {
  GRID_STRIDE(i, k) if (s[i] < n1) atomicAdd(&dcnt[s[i]], 1ull);
}

__global__ void k_region_size(uint64_t n1, const unsigned long long* dcnt, unsigned long long* rsz) {
  GRID_STRIDE(o, n1) {
    const uint64_t c = dcnt[o];
    uint64_t r = 0;
    if (c) {
      r = 4;
      while (r < 2 * c) r <<= 1;
    }
    rsz[o] = r;
  }
}

__global__ void k_insert_deletes(uint64_t k, const uint32_t* s, const uint32_t* t, const uint32_t* l,
                                 const unsigned long long* rbase, const unsigned long long* rsz, DelSlot* tab,
                                 uint32_t* err) {
  GRID_STRIDE(i, k) {
    const uint64_t base = rbase[s[i]], size = rsz[s[i]];
    const unsigned long long key = (((unsigned long long)t[i] << 32) | l[i]) + 1ull;
    uint64_t h = (key * 0x9e3779b97f4a7c15ull) >> 7;
    bool done = false;
    for (uint64_t probe = 0; probe < size && !done; ++probe) {
      DelSlot* sl = &tab[base + ((h + probe) & (size - 1))];
      const unsigned long long cur = atomicCAS(&sl->key, 0ull, key);
      if (cur == 0ull || cur == key) {
        atomicAdd(&sl->count, 1);
        done = true;
      }
    }
    if (!done) atomicOr(err, 4u);
  }
}

// One warp per source with deletions: claim stored copies.
__global__ void k_match_deletes(uint64_t nlist, const uint32_t* list, const unsigned long long* coff,
                                const uint32_t* cdst, const uint32_t* clab, const unsigned long long* rbase,
                                const unsigned long long* rsz, DelSlot* tab, uint8_t* del) {
  const int lane = threadIdx.x & 31;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < nlist;
       w += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t o = list[w];
    const uint64_t base = rbase[o], size = rsz[o];
    for (uint64_t e = coff[o] + lane; e < coff[o + 1]; e += 32) {
      const unsigned long long key = (((unsigned long long)cdst[e] << 32) | clab[e]) + 1ull;
      uint64_t h = (key * 0x9e3779b97f4a7c15ull) >> 7;
      for (uint64_t probe = 0; probe < size; ++probe) {
        DelSlot* sl = &tab[base + ((h + probe) & (size - 1))];
        const unsigned long long cur = sl->key;
        if (cur == 0ull) break;
        if (cur == key) {
          if (atomicSub(&sl->count, 1) > 0) del[e] = 1;
          break;
        }
      }
    }
  }
}

__global__ void k_sources_with_deletes(uint64_t n1, const unsigned long long* dcnt, unsigned long long* nl,
                                       uint32_t* list) {
  GRID_STRIDE(o, n1) if (dcnt[o]) list[atomicAdd(nl, 1ull)] = (uint32_t)o;
}

__global__ void k_missing(uint64_t total, const DelSlot* tab, unsigned long long* missing) {
  unsigned long long m = 0;
  GRID_STRIDE(i, total) if (tab[i].key != 0ull && tab[i].count > 0) m += (unsigned long long)tab[i].count;
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xFFFFFFFFu, m, o);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(missing, m);
}

__global__ void k_mark_dead_nodes(uint64_t k, const uint32_t* u, uint8_t* alive) {
  GRID_STRIDE(i, k) alive[u[i]] = 0;
}

// Kept edges per source (drop deleted copies and edges on deleted nodes).
__global__ void k_count_kept(uint64_t n1, const unsigned long long* coff, const uint32_t* cdst, const uint8_t* del,
                             const uint8_t* alive, unsigned long long* kept) {
  const int lane = threadIdx.x & 31;
  for (uint64_t o = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; o < n1;
       o += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    unsigned long long c = 0;
    if (alive[o])
      for (uint64_t e = coff[o] + lane; e < coff[o + 1]; e += 32) c += (!del[e] && alive[cdst[e]]) ? 1 : 0;
    for (int s = 16; s > 0; s >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, s);
    if (lane == 0) kept[o] = c;
  }
}

__global__ void k_compact(uint64_t n1, const unsigned long long* coff, const uint32_t* cdst, const uint32_t* clab,
                          const uint8_t* del, const uint8_t* alive, const unsigned long long* noff, uint32_t* ndst,
                          uint32_t* nlab) {
  const int lane = threadIdx.x & 31;
  for (uint64_t o = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; o < n1;
       o += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    if (!alive[o]) continue;
    uint64_t w = noff[o];
    for (uint64_t b = coff[o]; b < coff[o + 1]; b += 32) {
      const uint64_t e = b + lane;
      const bool keep = e < coff[o + 1] && !del[e] && alive[cdst[e]];
      const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const uint64_t q = w + __popc(m & ((1u << lane) - 1u));
        ndst[q] = cdst[e];
        nlab[q] = clab[e];
      }
      w += __popc(m);
    }
  }
}

__global__ void k_gather_labels(uint64_t n0, const uint32_t* o2p, const uint32_t* nlabel, uint32_t* out) {
  GRID_STRIDE(o, n0) out[o] = nlabel[o2p[o]];
}

__global__ void k_max32(uint64_t m, const uint32_t* a, unsigned int* mx) {
  unsigned int v = 0;
  GRID_STRIDE(i, m) v = max(v, a[i]);
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, v);
}

__global__ void k_any_dead(uint64_t n, const uint8_t* alive, unsigned int* flag) {
  GRID_STRIDE(o, n) if (!alive[o]) *flag = 1;
}

// Exclusive scan (reduce-then-scan) of u64 in place, with optional copy.
constexpr int kT = 1024, kI = 4, kTile = kT * kI;

__global__ void __launch_bounds__(kT) k_usum(const unsigned long long* a, uint64_t n, unsigned long long* bs) {
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

__global__ void __launch_bounds__(kT) k_uscan1(unsigned long long* bs, uint64_t nb, unsigned long long* total) {
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
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kT) k_uscan2(unsigned long long* a, uint64_t n, const unsigned long long* bs,
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

// Exclusive scan of a[0..n); the grand total into *total_out (host).
Status scan_u64(Store& s, unsigned long long* a, uint64_t n, unsigned long long* copy, Buf& tmp,
                uint64_t* total_out) {
  const uint64_t tiles = std::max<uint64_t>(1, (n + kTile - 1) / kTile);
  Status st = ensure(s, tmp, (tiles + 1) * 8);
  if (!st.ok()) return st;
  unsigned long long* bs = ptr<unsigned long long>(tmp);
  if (n) {
    k_usum<<<(unsigned)tiles, kT, 0, s.stream>>>(a, n, bs);
    k_uscan1<<<1, kT, 0, s.stream>>>(bs, tiles, bs + tiles);
    k_uscan2<<<(unsigned)tiles, kT, 0, s.stream>>>(a, n, bs, copy);
  } else {
    cudaMemsetAsync(bs + tiles, 0, 8, s.stream);
  }
  if (!(st = cuda_check(cudaGetLastError(), "scan")).ok()) return st;
  if (total_out) {
    uint64_t v = 0;
    st = cuda_check(cudaMemcpyAsync(&v, bs + tiles, 8, cudaMemcpyDeviceToHost, s.stream), "scan total");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
    *total_out = v;
  }
  return st;
}

// Temporaries of one batch: the store's update buffers, kept for the next
// batch.
struct Bufs {
  InUse use;
  Buf* b;
  explicit Bufs(Store& st) : use(st, kCacheUpd), b(st.upd) {}
};

// Stage a batch array on the device (copy when it is host memory).
Status stage(Store& s, Buf& b, const uint32_t* src, uint64_t k, bool dev, const uint32_t** out) {
  *out = src;
  if (!k || dev) return Status::Ok();
  Status st = ensure(s, b, k * 4);
  if (!st.ok()) return st;
  *out = ptr<uint32_t>(b);
  return cuda_check(cudaMemcpyAsync(b.p, src, k * 4, cudaMemcpyHostToDevice, s.stream), "stage batch");
}

}  // namespace

// ---------------------------------------------------------------------------
// In-place application of a batch of edge insertions and deletions that keeps
// every node in its degree class (no node additions or deletions): internal
// ids and the class layout stay, only the touched nodes' segments change.
// Deletions claim one stored copy each (a claim bit per edge), the new
// offsets are the old ones shifted by the degree changes, untouched segments
// move as blocks and touched ones are rewritten.  Costs a few passes over the
// edge table instead of the relabelling a general batch needs.
// ---------------------------------------------------------------------------

// Internal ids of the batch's endpoints.
__global__ void k_to_internal_ids(uint64_t k, const uint32_t* o2p, const uint32_t* a, uint32_t* out) {
  GRID_STRIDE(i, k) out[i] = o2p[a[i]];
}

// One warp per deletion: claim the first unclaimed stored copy of (t, l) in
// the segment of s.  Claims are bits over the edge table.
template <typename LabelT>
__global__ void k_claim_deletes(uint64_t k, const uint32_t* ds, const uint32_t* dt, const uint32_t* dl, uint64_t n0,
                                const uint64_t* off, const uint32_t* dst, const LabelT* lab, uint32_t* claimed,
                                int* delta, uint32_t* touched, unsigned long long* missing) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < k; i += warps) {
    const uint32_t p = ds[i], t = dt[i], l = dl[i];
    if (p < n0 && off[p + 1] - off[p] > (uint64_t)kBlockMax) continue;  // hubs: k_claim_deletes_hub
    bool done = false;
    // an added node has no stored edge
    for (uint64_t e0 = p < n0 ? off[p] : 0, e1 = p < n0 ? off[p + 1] : 0; e0 < e1 && !done; e0 += 32) {
      const uint64_t e = e0 + lane;
      unsigned cand = __ballot_sync(0xFFFFFFFFu, e < e1 && dst[e] == t && (uint32_t)lab[e] == l);
      while (cand && !done) {
        const int j = __ffs(cand) - 1;
        cand &= cand - 1;
        uint32_t won = 0;
        if (lane == (uint32_t)j) {
          const uint64_t ej = e0 + j;
          won = (atomicOr(&claimed[ej >> 5], 1u << (ej & 31)) >> (ej & 31)) & 1u ? 0u : 1u;
        }
        done = __shfl_sync(0xFFFFFFFFu, won, j) != 0;
      }
    }
    if (lane == 0) {
      if (done) {
        atomicSub(&delta[p], 1);
        atomicOr(&touched[p >> 5], 1u << (p & 31));
      } else {
        atomicAdd(missing, 1ull);
      }
    }
  }
}

// Deletions whose source is a hub: one CTA per deletion scans the hub's
// segment, kClaimItems blocks of edges at a time with all their loads in
// flight (a hub holds up to millions of edges, and a copy of the triple may
// lie anywhere in it).
constexpr int kClaimItems = 8;

template <typename LabelT>
__global__ void __launch_bounds__(1024) k_claim_deletes_hub(uint64_t k, const uint32_t* ds, const uint32_t* dt,
                                                            const uint32_t* dl, uint64_t n0, const uint64_t* off,
                                                            const uint32_t* dst, const LabelT* lab, uint32_t* claimed,
                                                            int* delta, uint32_t* touched,
                                                            unsigned long long* missing) {
  __shared__ unsigned int done;
  for (uint64_t i = blockIdx.x; i < k; i += gridDim.x) {
    const uint32_t p = ds[i], t = dt[i], l = dl[i];
    if (!(p < n0 && off[p + 1] - off[p] > (uint64_t)kBlockMax)) continue;
    if (threadIdx.x == 0) done = 0;
    __syncthreads();
    const uint64_t e1 = off[p + 1];
    for (uint64_t e0 = off[p]; e0 < e1; e0 += (uint64_t)blockDim.x * kClaimItems) {
      uint32_t tv[kClaimItems], lv[kClaimItems];
#pragma unroll
      for (int r = 0; r < kClaimItems; ++r) {
        const uint64_t e = e0 + (uint64_t)r * blockDim.x + threadIdx.x;
        tv[r] = e < e1 ? dst[e] : 0u;
        lv[r] = e < e1 ? (uint32_t)lab[e] : 0u;
      }
      uint32_t cm = 0;  // bit r: this thread's edge of block r is a copy of the triple
#pragma unroll
      for (int r = 0; r < kClaimItems; ++r) {
        const uint64_t e = e0 + (uint64_t)r * blockDim.x + threadIdx.x;
        if (e < e1 && tv[r] == t && lv[r] == l) cm |= 1u << r;
      }
      // candidates take turns, block by block and in lane order within a
      // block, until one claims (`done` is read after a barrier: uniform)
      if (__syncthreads_or(cm != 0)) {
        for (int r = 0; r < kClaimItems; ++r) {
          if (done) break;
          const bool cand = (cm >> r) & 1u;
          const uint64_t e = e0 + (uint64_t)r * blockDim.x + threadIdx.x;
          if (!__syncthreads_or(cand)) continue;
          for (uint32_t w = 0; w < blockDim.x; w += 32) {
            if (done) break;
            if (threadIdx.x >= w && threadIdx.x < w + 32) {
              unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
              while (m && !done) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                if ((threadIdx.x & 31) == (uint32_t)j) {
                  if (!((atomicOr(&claimed[e >> 5], 1u << (e & 31)) >> (e & 31)) & 1u)) done = 1;
                }
                __syncwarp();
              }
            }
            __syncthreads();
          }
        }
      }
      __syncthreads();
      if (done) break;
    }
    if (threadIdx.x == 0) {
      if (done) {
        atomicSub(&delta[p], 1);
        atomicOr(&touched[p >> 5], 1u << (p & 31));
      } else {
        atomicAdd(missing, 1ull);
      }
    }
    __syncthreads();
  }
}

__global__ void k_count_inserts_internal(uint64_t k, const uint32_t* is, int* delta, uint32_t* touched) {
  GRID_STRIDE(i, k) {
    atomicAdd(&delta[is[i]], 1);
    atomicOr(&touched[is[i] >> 5], 1u << (is[i] & 31));
  }
}

// Touched nodes whose degree class would change (then the batch is applied by
// relabelling), and the new degrees of all nodes.
__global__ void k_new_degrees(uint64_t n0, uint64_t n, const uint64_t* off, const int* delta, unsigned long long* deg,
                              unsigned int* class_moved) {
  GRID_STRIDE(p, n) {
    const uint64_t d0 = p < n0 ? off[p + 1] - off[p] : 0;
    const int dd = delta[p];
    const uint64_t d1 = (uint64_t)((int64_t)d0 + dd);
    deg[p] = d1;
    if (dd && degree_class_of(d0) != degree_class_of(d1)) *class_moved = 1u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) deg[n] = 0;
}

// Untouched segments move to their new offsets.  Out-degree <= 64: one warp
// per 32 consecutive nodes, edges found by a binary search over the 32
// offsets (as in the relabelling); larger: one warp per node.
template <typename LabelT>
__global__ void k_move_small(uint64_t n_small, const uint64_t* off, const uint64_t* noff, const uint32_t* touched,
                             const uint32_t* dst, const LabelT* lab, uint32_t* ndst, LabelT* nlab) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < n_small; w += warps) {
    const uint64_t p = w * 32 + lane;
    const uint64_t base = off[w * 32];
    const uint64_t end = off[min(w * 32 + 32, n_small)];
    const uint32_t r1 = (uint32_t)((p < n_small ? off[p] : end) - base);
    const uint64_t to = p < n_small ? noff[p] : 0;
    const bool skip = p >= n_small || ((touched[p >> 5] >> (p & 31)) & 1u);
    const uint32_t T = (uint32_t)(end - base);
    for (uint32_t k0 = 0; k0 < T; k0 += 32) {
      const uint32_t kk = k0 + lane;
      const uint32_t ks = min(kk, T - 1);
      uint32_t j = 0;
#pragma unroll
      for (uint32_t step = 16; step; step >>= 1)
        if (__shfl_sync(0xFFFFFFFFu, r1, j + step) <= ks) j += step;
      const bool sk = __shfl_sync(0xFFFFFFFFu, skip, j);
      const uint64_t tj = __shfl_sync(0xFFFFFFFFu, to, j);
      const uint32_t rj = __shfl_sync(0xFFFFFFFFu, r1, j);
      if (kk < T && !sk) {
        ndst[tj + (kk - rj)] = dst[base + kk];
        nlab[tj + (kk - rj)] = lab[base + kk];
      }
    }
  }
}

template <typename LabelT>
__global__ void k_move_large(uint64_t p0, uint64_t p1, const uint64_t* off, const uint64_t* noff,
                             const uint32_t* touched, const uint32_t* dst, const LabelT* lab, uint32_t* ndst,
                             LabelT* nlab) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t p = p0 + ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5); p < p1; p += warps) {
    if ((touched[p >> 5] >> (p & 31)) & 1u) continue;
    const uint64_t a = off[p], d = off[p + 1] - a, b = noff[p];
    for (uint64_t i = lane; i < d; i += 32) {
      ndst[b + i] = dst[a + i];
      nlab[b + i] = lab[a + i];
    }
  }
}

// Touched nodes (one warp each): kept edges first, then a cursor for the
// inserted ones.
template <typename LabelT>
__global__ void k_rewrite_touched(const uint32_t* list, uint64_t count, uint64_t n0, const uint64_t* off,
                                  const uint64_t* noff,
                                  const uint32_t* claimed, const uint32_t* dst, const LabelT* lab, uint32_t* ndst,
                                  LabelT* nlab, unsigned long long* cursor) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < count; i += warps) {
    const uint32_t p = list[i];
    if (p < n0 && off[p + 1] - off[p] > (uint64_t)kBlockMax) continue;  // hubs: k_hub_chunk_move
    uint64_t w = noff[p];
    const uint64_t a = p < n0 ? off[p] : 0, b = p < n0 ? off[p + 1] : 0;  // added nodes: no stored edge
    for (uint64_t e0 = a; e0 < b; e0 += 32) {
      const uint64_t e = e0 + lane;
      const bool keep = e < b && !((claimed[e >> 5] >> (e & 31)) & 1u);
      const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const uint64_t q = w + __popc(m & ((1u << lane) - 1u));
        ndst[q] = dst[e];
        nlab[q] = lab[e];
      }
      w += __popc(m);
    }
    if (lane == 0) cursor[p] = w;
  }
}

template <typename LabelT>
__global__ void k_place_inserts_internal(uint64_t k, const uint32_t* is, const uint32_t* it, const uint32_t* il,
                                         unsigned long long* cursor, uint32_t* ndst, LabelT* nlab) {
  GRID_STRIDE(i, k) {
    const uint64_t q = atomicAdd(&cursor[is[i]], 1ull);
    ndst[q] = it[i];
    nlab[q] = (LabelT)il[i];
  }
}

__global__ void k_bits_list(const uint32_t* bits, uint64_t words, uint32_t* list, unsigned long long* count) {
  GRID_STRIDE(w, words) {
    uint32_t m = bits[w];
    if (!m) continue;
    const unsigned long long b = atomicAdd(count, (unsigned long long)__popc(m));
    uint32_t j = 0;
    while (m) {
      const uint32_t x = __ffs(m) - 1;
      m &= m - 1;
      list[b + j++] = (uint32_t)((w << 5) + x);
    }
  }
}

// Hubs, one CTA per chunk of the hub's edges (the chunk list of the current
// layout): claimed copies in the chunk, then per hub a prefix over its chunks
// and the cursor for its inserted edges, then the chunk's kept edges at their
// new places (a block scan of the claim flags).
constexpr int kHubMoveThreads = 256;
constexpr int kHubCntBuf = 14;  // index of the per-chunk claim counts in Store::inplace

__global__ void k_hub_chunk_claims(const uint4* chunks, uint64_t nchunks, const uint32_t* claimed, uint32_t* cnt) {
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint4 q = chunks[c];
    const uint64_t b = ((uint64_t)q.z << 32) | q.y;
    uint32_t tot = 0;
    for (uint32_t i0 = 0; i0 < q.w; i0 += kHubMoveThreads) {
      const uint64_t e = b + i0 + threadIdx.x;
      const bool cl = i0 + threadIdx.x < q.w && ((claimed[e >> 5] >> (e & 31)) & 1u);
      tot += __syncthreads_count(cl);
    }
    if (threadIdx.x == 0) cnt[c] = tot;
  }
}

__global__ void k_hub_chunk_prefix(uint64_t n_hub, uint64_t hub_first, const uint32_t* cstart, const uint4* chunks,
                                   const uint64_t* off, const uint64_t* noff, uint32_t* cnt,
                                   unsigned long long* cursor) {
  for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n_hub; h += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t run = 0;
    for (uint32_t c = cstart[h]; c < cstart[h + 1]; ++c) {
      const uint32_t v = cnt[c];
      cnt[c] = run;
      run += v;
    }
    const uint64_t p = hub_first + h;
    cursor[p] = noff[p] + (off[p + 1] - off[p]) - run;
  }
}

template <typename LabelT>
__global__ void __launch_bounds__(kHubMoveThreads) k_hub_chunk_move(const uint4* chunks, uint64_t nchunks,
                                                                   uint64_t hub_first, const uint64_t* off,
                                                                   const uint64_t* noff, const uint32_t* claimed,
                                                                   const uint32_t* before, const uint32_t* dst,
                                                                   const LabelT* lab, uint32_t* ndst, LabelT* nlab) {
  __shared__ uint32_t wsum[kHubMoveThreads / 32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint4 q = chunks[c];
    const uint64_t p = hub_first + q.x;
    const uint64_t b = ((uint64_t)q.z << 32) | q.y;
    const uint64_t to = noff[p] + (b - off[p]);
    uint32_t run = before[c];  // claims before this chunk in the hub
    for (uint32_t i0 = 0; i0 < q.w; i0 += kHubMoveThreads) {
      const uint32_t i = i0 + threadIdx.x;
      const uint64_t e = b + i;
      const bool valid = i < q.w;
      const bool cl = valid && ((claimed[e >> 5] >> (e & 31)) & 1u);
      const unsigned m = __ballot_sync(0xFFFFFFFFu, cl);
      if (lane == 0) wsum[warp] = __popc(m);
      __syncthreads();
      uint32_t wb = 0, tot = 0;
      for (int w = 0; w < kHubMoveThreads / 32; ++w) {
        if (w < (int)warp) wb += wsum[w];
        tot += wsum[w];
      }
      const uint32_t claims_before = run + wb + __popc(m & ((1u << lane) - 1u));
      if (valid && !cl) {
        ndst[to + i - claims_before] = dst[e];
        nlab[to + i - claims_before] = lab[e];
      }
      run += tot;
      __syncthreads();
    }
  }
}

template <typename LabelT>
Status move_edges(Store& s, const uint64_t* noff, const uint32_t* touched, const uint32_t* claimed,
                  const uint32_t* tlist, uint64_t ntouched, unsigned long long* cursor, const uint32_t* is,
                  const uint32_t* it, const uint32_t* il, uint64_t nins, uint32_t* ndst, LabelT* nlab) {
  const uint64_t* off = ptr<uint64_t>(s.offsets);
  const uint32_t* dst = ptr<uint32_t>(s.dst);
  const LabelT* lab = static_cast<const LabelT*>(s.elabel.p);
  const uint64_t n_small = s.class_start[kClassWarp];
  if (n_small)
    k_move_small<LabelT><<<grid(s, n_small, 256), 256, 0, s.stream>>>(n_small, off, noff, touched, dst, lab, ndst,
                                                                       nlab);
  const uint64_t hub_first = s.class_start[kClassHub];
  if (hub_first > n_small)
    k_move_large<LabelT><<<grid(s, (hub_first - n_small) * 32, 256), 256, 0, s.stream>>>(
        n_small, hub_first, off, noff, touched, dst, lab, ndst, nlab);
  if (s.n_hub_chunks) {
    Status st = ensure(s, s.inplace[kHubCntBuf], s.n_hub_chunks * 4);
    if (!st.ok()) return st;
    uint32_t* cnt = ptr<uint32_t>(s.inplace[kHubCntBuf]);
    const unsigned gc = (unsigned)std::min<uint64_t>(s.n_hub_chunks, (uint64_t)s.sms * 8);
    const uint4* chunks = ptr<uint4>(s.hub_chunks);
    k_hub_chunk_claims<<<gc, kHubMoveThreads, 0, s.stream>>>(chunks, s.n_hub_chunks, claimed, cnt);
    k_hub_chunk_prefix<<<grid(s, s.n_hub, 256), 256, 0, s.stream>>>(s.n_hub, hub_first, ptr<uint32_t>(s.hub_cstart),
                                                                     chunks, off, noff, cnt, cursor);
    k_hub_chunk_move<LabelT><<<gc, kHubMoveThreads, 0, s.stream>>>(chunks, s.n_hub_chunks, hub_first, off, noff,
                                                                    claimed, cnt, dst, lab, ndst, nlab);
  }
  if (ntouched)
    k_rewrite_touched<LabelT><<<grid(s, ntouched * 32, 256), 256, 0, s.stream>>>(tlist, ntouched, s.n, off, noff,
                                                                                 claimed, dst, lab, ndst, nlab, cursor);
  if (nins)
    k_place_inserts_internal<LabelT><<<grid(s, nins, 256), 256, 0, s.stream>>>(nins, is, it, il, cursor, ndst, nlab);
  return cuda_check(cudaGetLastError(), "move edges");
}

// Original-order alive flags grown by the added nodes (alive).
Status ensure_keep_alive(Store& s, uint64_t n0, uint64_t n1) {
  Buf nb;
  Status st = ensure(s, nb, std::max<uint64_t>(n1, 1));
  if (!st.ok()) return st;
  cudaMemcpyAsync(nb.p, s.alive_o.p, n0, cudaMemcpyDeviceToDevice, s.stream);
  cudaMemsetAsync(static_cast<uint8_t*>(nb.p) + n0, 1, n1 - n0, s.stream);
  st = cuda_check(cudaStreamSynchronize(s.stream), "alive flags");
  release(s, s.alive_o);
  s.alive_o = nb;
  return st;
}

// Endpoints of the batch in the current internal ids; a node added by the
// batch (original id >= n0) keeps its original id as its provisional one.
__global__ void k_to_current_ids(uint64_t k, const uint32_t* o2p, uint64_t n0, const uint32_t* a, uint32_t* out) {
  GRID_STRIDE(i, k) out[i] = a[i] < n0 ? o2p[a[i]] : a[i];
}

// Provisional ids -> original ids (the current p2o, extended by the added
// nodes), node labels and alive flags by provisional id, for the relabelling.
__global__ void k_provisional_maps(uint64_t n0, uint64_t n1, uint64_t n_alive0, const uint32_t* p2o,
                                   const uint32_t* nlabel, const uint32_t* add_label, uint32_t* orig, uint32_t* nlab,
                                   uint8_t* alive) {
  GRID_STRIDE(q, n1) {
    orig[q] = q < n0 ? p2o[q] : (uint32_t)q;
    nlab[q] = q < n0 ? nlabel[q] : add_label[q - n0];
    alive[q] = (q < n_alive0 || q >= n0) ? 1 : 0;
  }
}

// After relabelling by provisional ids: p2o[p] = the original id of the
// provisional id the relabelling gave node p; then o2p is its inverse.
__global__ void k_compose_p2o(uint64_t n, const uint32_t* orig, uint32_t* p2o) {
  GRID_STRIDE(p, n) p2o[p] = orig[p2o[p]];
}
__global__ void k_invert_p2o(uint64_t n, const uint32_t* p2o, uint32_t* o2p) {
  GRID_STRIDE(p, n) o2p[p2o[p]] = (uint32_t)p;
}

// The fast path for edge insertions and deletions and node additions (no node
// deletions, every deletion names a stored copy, labels keep their width):
// the new edge table is built in the current internal ids (deletions claim
// stored copies, untouched segments move as blocks, touched ones are
// rewritten).  If every node keeps its degree class and no node is added, the
// table replaces the old one in place; otherwise the new table is laid out
// again from these ids by the usual relabelling, whose order is then mapped
// back to original ids.  *taken = false leaves the graph as it was (the
// general path runs).
Status apply_in_place_body(Store& s, const kbisim_batch* bt, const uint32_t* is, const uint32_t* it,
                           const uint32_t* il, const uint32_t* ds, const uint32_t* dt, const uint32_t* dl,
                           const uint32_t* addl, uint64_t* missing_out, bool* taken);

// With an HBM budget the fast path's buffers (the second edge table, claims,
// degrees) count against it: if they do not fit, the general path runs.
Status apply_in_place(Store& s, const kbisim_batch* bt, const uint32_t* is, const uint32_t* it, const uint32_t* il,
                      const uint32_t* ds, const uint32_t* dt, const uint32_t* dl, const uint32_t* addl,
                      uint64_t* missing_out, bool* taken) {
  Status st;
  {
    InUse use(s, kCacheInplace);
    st = apply_in_place_body(s, bt, is, it, il, ds, dt, dl, addl, missing_out, taken);
  }
  if (s.budget && st.code == KBISIM_ERR_BUDGET && !*taken && s.has_graph) {
    for (Buf& b : s.inplace) release(s, b);  // room for the general path
    return Status::Ok();
  }
  return st;
}

Status apply_in_place_body(Store& s, const kbisim_batch* bt, const uint32_t* is, const uint32_t* it,
                           const uint32_t* il, const uint32_t* ds, const uint32_t* dt, const uint32_t* dl,
                           const uint32_t* addl, uint64_t* missing_out, bool* taken) {
  *taken = false;
  const uint64_t n0 = s.n, m = s.m, ni = bt->n_ins, nd = bt->n_del, na = bt->n_add_nodes;
  const uint64_t n1 = n0 + na;
  if (bt->n_del_nodes || !n0 || !s.has_graph) return Status::Ok();
  if (ni + nd > std::max<uint64_t>(m / 16, 1ull << 16)) return Status::Ok();  // large batches: general path
  Status st;
  Buf* B = s.inplace;
  enum { IDS, DELTA, TOUCH, CLAIM, DEG, CUR, LIST, NDST, NLAB, SC, TMP, ORIG, PNLAB, PALIVE };
  const uint64_t words = n1 / 32 + 1, cwords = m / 32 + 1;
  if (!(st = ensure(s, B[IDS], std::max<uint64_t>(2 * ni + 2 * nd, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, B[DELTA], n1 * 4)).ok()) return st;
  if (!(st = ensure(s, B[TOUCH], words * 4)).ok()) return st;
  if (!(st = ensure(s, B[CLAIM], cwords * 4)).ok()) return st;
  if (!(st = ensure(s, B[DEG], (n1 + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, B[SC], 64)).ok()) return st;
  uint32_t* ids = ptr<uint32_t>(B[IDS]);
  uint32_t *isp = ids, *itp = ids + ni, *dsp = ids + 2 * ni, *dtp = ids + 2 * ni + nd;
  int* delta = ptr<int>(B[DELTA]);
  uint32_t* touched = ptr<uint32_t>(B[TOUCH]);
  uint32_t* claimed = ptr<uint32_t>(B[CLAIM]);
  unsigned long long* deg = ptr<unsigned long long>(B[DEG]);
  unsigned long long* sc = ptr<unsigned long long>(B[SC]);
  cudaMemsetAsync(delta, 0, n1 * 4, s.stream);
  cudaMemsetAsync(touched, 0, words * 4, s.stream);
  cudaMemsetAsync(claimed, 0, cwords * 4, s.stream);
  cudaMemsetAsync(sc, 0, 64, s.stream);
  const uint32_t* o2p = ptr<uint32_t>(s.o2p);
  if (ni) {
    k_to_current_ids<<<grid(s, ni, 256), 256, 0, s.stream>>>(ni, o2p, n0, is, isp);
    k_to_current_ids<<<grid(s, ni, 256), 256, 0, s.stream>>>(ni, o2p, n0, it, itp);
    k_count_inserts_internal<<<grid(s, ni, 256), 256, 0, s.stream>>>(ni, isp, delta, touched);
  }
  if (nd) {
    k_to_current_ids<<<grid(s, nd, 256), 256, 0, s.stream>>>(nd, o2p, n0, ds, dsp);
    k_to_current_ids<<<grid(s, nd, 256), 256, 0, s.stream>>>(nd, o2p, n0, dt, dtp);
    if (s.label8)
      k_claim_deletes<uint8_t><<<grid(s, nd * 32, 256), 256, 0, s.stream>>>(
          nd, dsp, dtp, dl, n0, ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst), ptr<uint8_t>(s.elabel), claimed,
          delta, touched, sc);
    else
      k_claim_deletes<uint32_t><<<grid(s, nd * 32, 256), 256, 0, s.stream>>>(
          nd, dsp, dtp, dl, n0, ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst), ptr<uint32_t>(s.elabel), claimed,
          delta, touched, sc);
    if (s.n_hub) {
      const unsigned gh = (unsigned)std::min<uint64_t>(nd, (uint64_t)s.sms * 2);
      if (s.label8)
        k_claim_deletes_hub<uint8_t><<<gh, 1024, 0, s.stream>>>(nd, dsp, dtp, dl, n0, ptr<uint64_t>(s.offsets),
                                                              ptr<uint32_t>(s.dst), ptr<uint8_t>(s.elabel), claimed,
                                                              delta, touched, sc);
      else
        k_claim_deletes_hub<uint32_t><<<gh, 1024, 0, s.stream>>>(nd, dsp, dtp, dl, n0, ptr<uint64_t>(s.offsets),
                                                               ptr<uint32_t>(s.dst), ptr<uint32_t>(s.elabel), claimed,
                                                               delta, touched, sc);
    }
  }
  unsigned int* moved = reinterpret_cast<unsigned int*>(sc + 1);
  unsigned int* maxlab = moved + 1;
  k_new_degrees<<<grid(s, n1, 256), 256, 0, s.stream>>>(n0, n1, ptr<uint64_t>(s.offsets), delta, deg, moved);
  if (ni) k_max32<<<grid(s, ni, 256), 256, 0, s.stream>>>(ni, il, maxlab);
  uint64_t h[2] = {0, 0};
  st = cuda_check(cudaGetLastError(), "batch");
  if (st.ok()) st = cuda_check(cudaMemcpyAsync(h, sc, 16, cudaMemcpyDeviceToHost, s.stream), "batch");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  const uint32_t moved_v = (uint32_t)h[1], maxlab_v = (uint32_t)(h[1] >> 32);
  if (s.label8 && maxlab_v >= 256) return Status::Ok();  // wider labels: general path
  // a deletion with no stored copy may name an edge inserted by this batch
  // (insertions come first): the general path decides those
  if (h[0]) return Status::Ok();
  const uint64_t m1 = m + ni - nd;
  const bool relabel = moved_v || na;
  // new offsets (current ids), touched list, then the edges
  if (!(st = scan_u64(s, deg, n1 + 1, nullptr, B[TMP], nullptr)).ok()) return st;
  if (!(st = ensure(s, B[CUR], (n1 + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, B[LIST], n1 * 4)).ok()) return st;
  if (!(st = ensure(s, B[NDST], std::max<uint64_t>(m1, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, B[NLAB], std::max<uint64_t>(m1, 1) * (s.label8 ? 1 : 4))).ok()) return st;
  cudaMemsetAsync(sc + 2, 0, 8, s.stream);
  k_bits_list<<<grid(s, words, 256), 256, 0, s.stream>>>(touched, words, ptr<uint32_t>(B[LIST]), sc + 2);
  uint64_t ntouched = 0;
  st = cuda_check(cudaMemcpyAsync(&ntouched, sc + 2, 8, cudaMemcpyDeviceToHost, s.stream), "touched");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  unsigned long long* cur = ptr<unsigned long long>(B[CUR]);
  if (s.label8)
    st = move_edges<uint8_t>(s, reinterpret_cast<const uint64_t*>(deg), touched, claimed, ptr<uint32_t>(B[LIST]),
                             ntouched, cur, isp, itp, il, ni, ptr<uint32_t>(B[NDST]), ptr<uint8_t>(B[NLAB]));
  else
    st = move_edges<uint32_t>(s, reinterpret_cast<const uint64_t*>(deg), touched, claimed, ptr<uint32_t>(B[LIST]),
                              ntouched, cur, isp, itp, il, ni, ptr<uint32_t>(B[NDST]), ptr<uint32_t>(B[NLAB]));
  if (!st.ok()) return st;
  if (maxlab_v) {
    uint32_t lb = 1;
    while (lb < 32 && (maxlab_v >> lb)) ++lb;
    s.label_bits = std::max(s.label_bits, lb);
  }
  for (size_t i = 0; i < s.out_valid.size(); ++i) s.out_valid[i] = false;
  s.has_levels = false;
  s.many.valid = false;
  if (!relabel) {
    // the new table replaces the old one (buffers swap, so both stay allocated)
    std::swap(s.dst, B[NDST]);
    std::swap(s.elabel, B[NLAB]);
    std::swap(s.offsets, B[DEG]);
    s.m = m1;
    if (!(st = build_chunk_lists(s, false)).ok()) return st;
  } else {
    // lay the new table out again; its ids are the current internal ones (and
    // the added nodes'), so the relabelling's order is mapped back to
    // original ids afterwards
    if (!(st = ensure(s, B[ORIG], n1 * 4)).ok()) return st;
    if (!(st = ensure(s, B[PNLAB], n1 * 4)).ok()) return st;
    if (!(st = ensure(s, B[PALIVE], n1)).ok()) return st;
    k_provisional_maps<<<grid(s, n1, 256), 256, 0, s.stream>>>(n0, n1, s.n_alive, ptr<uint32_t>(s.p2o),
                                                               ptr<uint32_t>(s.nlabel), addl, ptr<uint32_t>(B[ORIG]),
                                                               ptr<uint32_t>(B[PNLAB]), ptr<uint8_t>(B[PALIVE]));
    if (!(st = cuda_check(cudaGetLastError(), "provisional ids")).ok()) return st;
    const bool any_dead = s.n_alive < n0;
    s.n = n1;
    s.m = m1;
    if (!(st = relabel_graph(s, reinterpret_cast<const uint64_t*>(deg), ptr<uint32_t>(B[NDST]), B[NLAB].p,
                             ptr<uint32_t>(B[PNLAB]), any_dead ? ptr<uint8_t>(B[PALIVE]) : nullptr,
                             s.label8 ? 1 : 4)).ok()) {
      s.has_graph = false;
      return st;
    }
    k_compose_p2o<<<grid(s, n1, 256), 256, 0, s.stream>>>(n1, ptr<uint32_t>(B[ORIG]), ptr<uint32_t>(s.p2o));
    k_invert_p2o<<<grid(s, n1, 256), 256, 0, s.stream>>>(n1, ptr<uint32_t>(s.p2o), ptr<uint32_t>(s.o2p));
    if (!(st = cuda_check(cudaGetLastError(), "compose ids")).ok()) return st;
    if (s.any_dead && na) {  // alive flags in original order: the added nodes are alive
      if (!(st = ensure_keep_alive(s, n0, n1)).ok()) return st;
    }
  }
  *taken = true;
  s.mt.in_place = relabel ? 0 : 1;
  if (missing_out) *missing_out = 0;
  return cuda_check(cudaStreamSynchronize(s.stream), "batch");
}

Status apply_batch_body(Store& s, const kbisim_batch* bt, uint64_t* missing_out);

// The batch, with the hubs' bucket growth carried over to the new layout.
Status apply_batch(Store& s, const kbisim_batch* bt, uint64_t* missing_out) {
  HubGrowth g;
  Status st = save_hub_growth(s, &g);
  if (st.ok()) st = apply_batch_body(s, bt, missing_out);
  if (st.ok()) st = restore_hub_growth(s, g, false);
  return st;
}

Status apply_batch_body(Store& s, const kbisim_batch* bt, uint64_t* missing_out) {
  if (!bt) return Status::Err(KBISIM_ERR_INVALID_ARG, "batch is NULL");
  if (!s.has_graph) return Status::Err(KBISIM_ERR_STATE, "no graph loaded");
  if ((bt->n_add_nodes && !bt->add_node_label) || (bt->n_ins && (!bt->ins_src || !bt->ins_dst || !bt->ins_label)) ||
      (bt->n_del && (!bt->del_src || !bt->del_dst || !bt->del_label)) || (bt->n_del_nodes && !bt->del_nodes))
    return Status::Err(KBISIM_ERR_INVALID_ARG, "batch array is NULL");
  const uint64_t n0 = s.n, n1 = n0 + bt->n_add_nodes;
  if (n1 >= 0xFFFFFFFFull) return Status::Err(KBISIM_ERR_INVALID_ARG, "too many nodes");
  const bool dev = bt->on_device != 0;
  Status st;
  Bufs t(s);
  enum { ADDL, INS_S, INS_T, INS_L, DEL_S, DEL_T, DEL_L, DEL_N, ALIVE, ERR, CNT, COFF, CUR, CDST, CLAB, DCNT, RSZ,
         RBASE, TAB, LIST, DELF, NOFF, NDST, NLAB };
  const uint32_t *addl, *is, *it, *il, *ds, *dt, *dl, *dn;
  if (!(st = stage(s, t.b[ADDL], bt->add_node_label, bt->n_add_nodes, dev, &addl)).ok()) return st;
  if (!(st = stage(s, t.b[INS_S], bt->ins_src, bt->n_ins, dev, &is)).ok()) return st;
  if (!(st = stage(s, t.b[INS_T], bt->ins_dst, bt->n_ins, dev, &it)).ok()) return st;
  if (!(st = stage(s, t.b[INS_L], bt->ins_label, bt->n_ins, dev, &il)).ok()) return st;
  if (!(st = stage(s, t.b[DEL_S], bt->del_src, bt->n_del, dev, &ds)).ok()) return st;
  if (!(st = stage(s, t.b[DEL_T], bt->del_dst, bt->n_del, dev, &dt)).ok()) return st;
  if (!(st = stage(s, t.b[DEL_L], bt->del_label, bt->n_del, dev, &dl)).ok()) return st;
  if (!(st = stage(s, t.b[DEL_N], bt->del_nodes, bt->n_del_nodes, dev, &dn)).ok()) return st;
  // alive flags (original order) after node additions
  if (!(st = ensure(s, t.b[ALIVE], std::max<uint64_t>(n1, 1))).ok()) return st;
  if (!(st = ensure(s, t.b[ERR], 64)).ok()) return st;
  uint8_t* alive = ptr<uint8_t>(t.b[ALIVE]);
  uint32_t* err = ptr<uint32_t>(t.b[ERR]);
  cudaMemsetAsync(err, 0, 64, s.stream);
  k_alive_init<<<grid(s, n1, 256), 256, 0, s.stream>>>(n0, n1, s.any_dead ? ptr<uint8_t>(s.alive_o) : nullptr, alive);
  if (bt->n_ins) k_check_inserts<<<grid(s, bt->n_ins, 256), 256, 0, s.stream>>>(bt->n_ins, n1, is, it, alive, err);
  if (bt->n_del) {
    k_check_ids_only<<<grid(s, bt->n_del, 256), 256, 0, s.stream>>>(bt->n_del, n1, ds, err);
    k_check_ids_only<<<grid(s, bt->n_del, 256), 256, 0, s.stream>>>(bt->n_del, n1, dt, err);
  }
  if (bt->n_del_nodes)
    k_check_node_dels<<<grid(s, bt->n_del_nodes, 256), 256, 0, s.stream>>>(bt->n_del_nodes, n1, dn, alive, err);
  uint32_t e = 0;
  st = cuda_check(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s.stream), "validate batch");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;
  if (e & kBadId) return Status::Err(KBISIM_ERR_INVALID_ARG, "batch names a node id >= num_nodes");
  if (e & kDeadEnd) return Status::Err(KBISIM_ERR_INVALID_ARG, "batch touches a deleted node");
  {
    bool taken = false;
    s.mt.in_place = 0;
    if (!(st = apply_in_place(s, bt, is, it, il, ds, dt, dl, addl, missing_out, &taken)).ok()) return st;
    if (taken) return Status::Ok();
  }

  // 1. combined CSR by original source: stored edges, then inserted ones
  const uint64_t m0 = s.m, mc = m0 + bt->n_ins;
  if (!(st = ensure(s, t.b[CNT], (n1 + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, t.b[COFF], (n1 + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, t.b[CUR], (n1 + 1) * 8)).ok()) return st;
  if (!(st = ensure(s, t.b[CDST], std::max<uint64_t>(mc, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, t.b[CLAB], std::max<uint64_t>(mc, 1) * 4)).ok()) return st;
  unsigned long long* coff = ptr<unsigned long long>(t.b[COFF]);
  cudaMemsetAsync(coff, 0, (n1 + 1) * 8, s.stream);
  if (n0) k_count_combined<<<grid(s, n0, 256), 256, 0, s.stream>>>(n0, ptr<uint32_t>(s.o2p), ptr<uint64_t>(s.offsets),
                                                               bt->n_ins, is, coff);
  if (bt->n_ins) k_count_inserts<<<grid(s, bt->n_ins, 256), 256, 0, s.stream>>>(bt->n_ins, is, coff);
  uint64_t total = 0;
  if (!(st = scan_u64(s, coff, n1 + 1, nullptr, t.b[CNT], &total)).ok()) return st;
  unsigned long long* cur = ptr<unsigned long long>(t.b[CUR]);
  uint32_t* cdst = ptr<uint32_t>(t.b[CDST]);
  uint32_t* clab = ptr<uint32_t>(t.b[CLAB]);
  if (n0) {
    const unsigned g = grid(s, n0 * 32, 256);
    if (s.label8)
      k_copy_stored<uint8_t><<<g, 256, 0, s.stream>>>(n0, ptr<uint32_t>(s.o2p), ptr<uint32_t>(s.p2o),
                                                      ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst),
                                                      ptr<uint8_t>(s.elabel), coff, cur, cdst, clab);
    else
      k_copy_stored<uint32_t><<<g, 256, 0, s.stream>>>(n0, ptr<uint32_t>(s.o2p), ptr<uint32_t>(s.p2o),
                                                       ptr<uint64_t>(s.offsets), ptr<uint32_t>(s.dst),
                                                       ptr<uint32_t>(s.elabel), coff, cur, cdst, clab);
  }
  if (n1 > n0)  // new nodes start empty
    cudaMemcpyAsync(cur + n0, coff + n0, (n1 - n0) * 8, cudaMemcpyDeviceToDevice, s.stream);
  if (bt->n_ins) k_place_inserts<<<grid(s, bt->n_ins, 256), 256, 0, s.stream>>>(bt->n_ins, is, it, il, cur, cdst, clab);
  if (!(st = cuda_check(cudaGetLastError(), "combine edges")).ok()) return st;

  // 2. deletions, matched per source
  if (!(st = ensure(s, t.b[DELF], std::max<uint64_t>(mc, 1))).ok()) return st;
  uint8_t* delf = ptr<uint8_t>(t.b[DELF]);
  cudaMemsetAsync(delf, 0, std::max<uint64_t>(mc, 1), s.stream);
  uint64_t missing = 0;
  if (bt->n_del) {
    if (!(st = ensure(s, t.b[DCNT], (n1 + 1) * 8)).ok()) return st;
    if (!(st = ensure(s, t.b[RSZ], (n1 + 1) * 8)).ok()) return st;
    if (!(st = ensure(s, t.b[RBASE], (n1 + 1) * 8)).ok()) return st;
    unsigned long long* dcnt = ptr<unsigned long long>(t.b[DCNT]);
    unsigned long long* rsz = ptr<unsigned long long>(t.b[RSZ]);
    unsigned long long* rbase = ptr<unsigned long long>(t.b[RBASE]);
    cudaMemsetAsync(dcnt, 0, (n1 + 1) * 8, s.stream);
    k_count_deletes<<<grid(s, bt->n_del, 256), 256, 0, s.stream>>>(bt->n_del, ds, n1, dcnt);
    k_region_size<<<grid(s, n1 + 1, 256), 256, 0, s.stream>>>(n1 + 1, dcnt, rsz);
    cudaMemcpyAsync(rbase, rsz, (n1 + 1) * 8, cudaMemcpyDeviceToDevice, s.stream);
    uint64_t slots = 0;
    if (!(st = scan_u64(s, rbase, n1 + 1, nullptr, t.b[NOFF], &slots)).ok()) return st;
    if (!(st = ensure(s, t.b[TAB], std::max<uint64_t>(slots, 1) * sizeof(DelSlot))).ok()) return st;
    DelSlot* tab = ptr<DelSlot>(t.b[TAB]);
    cudaMemsetAsync(tab, 0, slots * sizeof(DelSlot), s.stream);
    k_insert_deletes<<<grid(s, bt->n_del, 256), 256, 0, s.stream>>>(bt->n_del, ds, dt, dl, rbase, rsz, tab, err);
    if (!(st = ensure(s, t.b[LIST], std::max<uint64_t>(n1, 1) * 4)).ok()) return st;
    unsigned long long* nl = reinterpret_cast<unsigned long long*>(err + 8);
    cudaMemsetAsync(nl, 0, 8, s.stream);
    k_sources_with_deletes<<<grid(s, n1, 256), 256, 0, s.stream>>>(n1, dcnt, nl, ptr<uint32_t>(t.b[LIST]));
    uint64_t nsrc = 0;
    st = cuda_check(cudaMemcpyAsync(&nsrc, nl, 8, cudaMemcpyDeviceToHost, s.stream), "delete sources");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
    if (!st.ok()) return st;
    if (nsrc)
      k_match_deletes<<<grid(s, nsrc * 32, 256), 256, 0, s.stream>>>(nsrc, ptr<uint32_t>(t.b[LIST]), coff, cdst, clab,
                                                                  rbase, rsz, tab, delf);
    unsigned long long* dmiss = reinterpret_cast<unsigned long long*>(err + 10);
    cudaMemsetAsync(dmiss, 0, 8, s.stream);
    if (slots) k_missing<<<grid(s, slots, 256), 256, 0, s.stream>>>(slots, tab, dmiss);
    st = cuda_check(cudaMemcpyAsync(&missing, dmiss, 8, cudaMemcpyDeviceToHost, s.stream), "missing");
    uint32_t e2 = 0;
    if (st.ok()) st = cuda_check(cudaMemcpyAsync(&e2, err, 4, cudaMemcpyDeviceToHost, s.stream), "err");
    if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
    if (!st.ok()) return st;
    if (e2 & 4u) return Status::Err(KBISIM_ERR_TIMEOUT, "deletion table probe bound exceeded");
  }

  // 3. node deletions; keep the rest
  if (bt->n_del_nodes) k_mark_dead_nodes<<<grid(s, bt->n_del_nodes, 256), 256, 0, s.stream>>>(bt->n_del_nodes, dn, alive);
  if (!(st = ensure(s, t.b[NOFF], (n1 + 1) * 8)).ok()) return st;
  unsigned long long* noff = ptr<unsigned long long>(t.b[NOFF]);
  cudaMemsetAsync(noff, 0, (n1 + 1) * 8, s.stream);
  k_count_kept<<<grid(s, n1 * 32, 256), 256, 0, s.stream>>>(n1, coff, cdst, delf, alive, noff);
  uint64_t m1 = 0;
  if (!(st = scan_u64(s, noff, n1 + 1, nullptr, t.b[CNT], &m1)).ok()) return st;
  if (!(st = ensure(s, t.b[NDST], std::max<uint64_t>(m1, 1) * 4)).ok()) return st;
  if (!(st = ensure(s, t.b[NLAB], std::max<uint64_t>(m1, 1) * 4)).ok()) return st;
  k_compact<<<grid(s, n1 * 32, 256), 256, 0, s.stream>>>(n1, coff, cdst, clab, delf, alive, noff, ptr<uint32_t>(t.b[NDST]),
                                                     ptr<uint32_t>(t.b[NLAB]));
  // node labels in original order (stored ones, then the added ones)
  if (!(st = ensure(s, t.b[CNT], std::max<uint64_t>(n1, 1) * 4)).ok()) return st;
  uint32_t* nlab = ptr<uint32_t>(t.b[CNT]);
  if (n0) k_gather_labels<<<grid(s, n0, 256), 256, 0, s.stream>>>(n0, ptr<uint32_t>(s.o2p), ptr<uint32_t>(s.nlabel), nlab);
  if (n1 > n0) cudaMemcpyAsync(nlab + n0, addl, (n1 - n0) * 4, cudaMemcpyDeviceToDevice, s.stream);
  unsigned int* dmax = reinterpret_cast<unsigned int*>(err + 12);
  cudaMemsetAsync(dmax, 0, 8, s.stream);
  if (m1) k_max32<<<grid(s, m1, 256), 256, 0, s.stream>>>(m1, ptr<uint32_t>(t.b[NLAB]), dmax);
  k_any_dead<<<grid(s, n1, 256), 256, 0, s.stream>>>(n1, alive, dmax + 1);
  uint32_t hv[2] = {0, 0};
  st = cuda_check(cudaGetLastError(), "compact");
  if (st.ok()) st = cuda_check(cudaMemcpyAsync(hv, dmax, 8, cudaMemcpyDeviceToHost, s.stream), "label max");
  if (st.ok()) st = cuda_check(cudaStreamSynchronize(s.stream), "sync");
  if (!st.ok()) return st;

  // 4. the updated graph replaces the stored one (level buffers are reused)
  for (size_t i = 0; i < s.out_valid.size(); ++i) s.out_valid[i] = false;
  s.has_levels = false;
  s.n = n1;
  s.m = m1;
  s.label8 = hv[0] < 256;
  uint32_t lb = 1;
  while (lb < 32 && (hv[0] >> lb)) ++lb;
  s.label_bits = lb;
  s.any_dead = hv[1] != 0;
  if (!(st = relabel_graph(s, reinterpret_cast<const uint64_t*>(noff), ptr<uint32_t>(t.b[NDST]), t.b[NLAB].p, nlab,
                           s.any_dead ? alive : nullptr, 4)).ok()) {
    s.has_graph = false;
    return st;
  }
  if (s.any_dead) {
    if (!(st = ensure(s, s.alive_o, std::max<uint64_t>(n1, 1))).ok()) return st;
    cudaMemcpyAsync(s.alive_o.p, alive, n1, cudaMemcpyDeviceToDevice, s.stream);
  }
  if (missing_out) *missing_out = missing;
  return cuda_check(cudaStreamSynchronize(s.stream), "update");
}

}  // namespace kb
