// Label partition (identifier level 0) without any device allocation.
//
// Some callers cannot allocate device memory when they need this result:
// a serving loop whose device memory is fully reserved up front by another
// allocator (a framework's caching pool, a fixed arena), or code that must
// not risk the implicit device-wide synchronisation that cudaMalloc and
// cudaFree may perform.  For them, kbisim_label_partition_noalloc computes
// the same level 0 as kbisim_refine (blocks of equal node labels, numbered by
// their smallest node id) using only the caller's input and output buffers
// and a fixed scratch area that lives in this library's static device memory.
//
// The scratch area below is allocated when the library is loaded onto a
// device and stays there until the process exits (every GPU that loads the
// library holds it).  It bounds the input size: num_nodes <= kMaxNodes.
// All calls share it and it keeps the last call's contents, so each call
// clears what must start empty, and calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on it.
//
// Host code only ever sees a host-side stand-in for the array's name, so the
// device address is looked up with cudaGetSymbolAddress once per device (with
// that device current) on the first call, which should therefore come before
// any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kbisim.h"

namespace {

constexpr uint64_t kMaxNodes = 1ull << 18;          // 262,144 nodes
constexpr uint64_t kSlots = 2 * kMaxNodes;          // hash table slots (power of two)
constexpr int kThreads = 1024;                      // rank kernels: one node per thread
constexpr uint64_t kTiles = kMaxNodes / kThreads;   // 256
constexpr unsigned long long kEmptySlot = ~0ull;

struct Scratch {
  unsigned long long table[kSlots];  // (label << 32) | smallest node id with that label
  uint32_t rank[kMaxNodes];          // head flag, then the head's block id
  uint32_t tile[kTiles + 1];         // heads per tile, then exclusive offsets; [kTiles] = total
};

static __device__ __align__(256) Scratch g_scratch;

constexpr int kMaxDevices = 64;
Scratch* g_dev_ptr[kMaxDevices] = {nullptr};
std::mutex g_mu;

__device__ __forceinline__ uint32_t home_slot(uint32_t label, uint64_t mask) {
  uint32_t x = label;  // MurmurHash3 32-bit finalizer spreads labels over the table
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return (uint32_t)(x & mask);
}

// The slot of `label`, inserting (label, u) on the way when `insert` is set.
// An empty slot reads as label 0xFFFFFFFF, which a node with that label then
// claims with the same atomicMin; probing is bounded by the table size.
__device__ __forceinline__ int64_t find_slot(Scratch* sc, uint32_t label, uint32_t u, uint64_t mask, bool insert) {
  uint64_t s = home_slot(label, mask);
  const unsigned long long v = ((unsigned long long)label << 32) | u;
  for (uint64_t t = 0; t <= mask; ++t) {
    unsigned long long cur = *(volatile unsigned long long*)&sc->table[s];
    if (cur == kEmptySlot && insert) {
      cur = atomicCAS(&sc->table[s], kEmptySlot, v);
      if (cur == kEmptySlot) return (int64_t)s;
    }
    if ((uint32_t)(cur >> 32) == label) {
      if (insert && (uint32_t)cur > u) atomicMin(&sc->table[s], v);
      return (int64_t)s;
    }
    s = (s + 1) & mask;
  }
  return -1;
}

__global__ void k_na_clear(Scratch* sc, uint64_t slots) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < slots; i += (uint64_t)gridDim.x * blockDim.x)
    sc->table[i] = kEmptySlot;
}

__global__ void k_na_insert(Scratch* sc, const uint32_t* label, uint64_t n, uint64_t mask) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x)
    find_slot(sc, label[u], (uint32_t)u, mask, true);
}

// rank[u] = 1 if u is the smallest node with its label; per-tile head counts.
__global__ void __launch_bounds__(kThreads) k_na_heads(Scratch* sc, const uint32_t* label, uint64_t n, uint64_t mask) {
  __shared__ uint32_t warp_sum[kThreads / 32];
  const uint64_t u = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
  uint32_t head = 0;
  if (u < n) {
    const int64_t s = find_slot(sc, label[u], (uint32_t)u, mask, false);
    head = (s >= 0 && (uint32_t)sc->table[s] == (uint32_t)u) ? 1u : 0u;
    sc->rank[u] = head;
  }
  uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, head));
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += warp_sum[w];
    sc->tile[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile counts (one CTA, at most kTiles tiles).
__global__ void __launch_bounds__(kTiles) k_na_scan(Scratch* sc, uint64_t ntiles, uint32_t* count_out) {
  __shared__ uint32_t v[kTiles];
  const uint32_t i = threadIdx.x;
  v[i] = i < ntiles ? sc->tile[i] : 0u;
  __syncthreads();
  for (uint32_t o = 1; o < kTiles; o <<= 1) {
    const uint32_t add = i >= o ? v[i - o] : 0u;
    __syncthreads();
    v[i] += add;
    __syncthreads();
  }
  if (i < ntiles) sc->tile[i] = v[i] - (i < ntiles ? sc->tile[i] : 0u);
  __syncthreads();
  if (i == 0) {
    sc->tile[kTiles] = v[kTiles - 1];
    if (count_out) *count_out = v[kTiles - 1];
  }
}

// Heads get their block id: tile offset + heads before them in the tile.
__global__ void __launch_bounds__(kThreads) k_na_rank(Scratch* sc, uint64_t n) {
  __shared__ uint32_t warp_sum[kThreads / 32];
  const uint64_t u = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
  const uint32_t head = u < n ? sc->rank[u] : 0u;
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, head);
  if (lane == 0) warp_sum[w] = __popc(bal);
  __syncthreads();
  uint32_t before = sc->tile[blockIdx.x];
  for (unsigned i = 0; i < w; ++i) before += warp_sum[i];
  before += __popc(bal & ((1u << lane) - 1u));
  if (head) sc->rank[u] = before;
}

__global__ void k_na_assign(Scratch* sc, const uint32_t* label, uint64_t n, uint64_t mask, uint32_t* pid0) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t s = find_slot(sc, label[u], (uint32_t)u, mask, false);
    pid0[u] = s >= 0 ? sc->rank[(uint32_t)sc->table[s]] : KBISIM_DELETED;
  }
}

}  // namespace

extern "C" int kbisim_label_partition_noalloc(const uint32_t* node_label, uint64_t num_nodes, uint32_t* pid0,
                                              uint32_t* block_count, void* stream) {
  if (num_nodes > kMaxNodes) return KBISIM_ERR_INVALID_ARG;
  if (num_nodes && (!node_label || !pid0)) return KBISIM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KBISIM_ERR_CUDA;
  }
  Scratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KBISIM_ERR_CUDA;
      }
      g_dev_ptr[dev] = static_cast<Scratch*>(p);
    }
    sc = g_dev_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (num_nodes == 0) {
    if (block_count && cudaMemsetAsync(block_count, 0, sizeof(uint32_t), st) != cudaSuccess) return KBISIM_ERR_CUDA;
    return KBISIM_OK;
  }
  uint64_t slots = 1024;
  while (slots < 2 * num_nodes) slots <<= 1;
  const uint64_t mask = slots - 1;
  const uint64_t ntiles = (num_nodes + kThreads - 1) / kThreads;
  const unsigned g = (unsigned)((num_nodes + 255) / 256);
  k_na_clear<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(sc, slots);
  k_na_insert<<<g, 256, 0, st>>>(sc, node_label, num_nodes, mask);
  k_na_heads<<<(unsigned)ntiles, kThreads, 0, st>>>(sc, node_label, num_nodes, mask);
  k_na_scan<<<1, (unsigned)kTiles, 0, st>>>(sc, ntiles, block_count);
  k_na_rank<<<(unsigned)ntiles, kThreads, 0, st>>>(sc, num_nodes);
  k_na_assign<<<g, 256, 0, st>>>(sc, node_label, num_nodes, mask, pid0);
  return cudaGetLastError() == cudaSuccess ? KBISIM_OK : KBISIM_ERR_CUDA;
}
