// Proposition 2 checker for large results (TEST INFRASTRUCTURE ONLY).
//
// For graphs too large for the oracle (Algorithm 1 with ordered maps runs on
// one core), this checks a candidate level against its definition instead of
// recomputing it.  Given the previous level prev (already checked: level 0
// against the oracle, then each level in turn) and a candidate level cur,
// cur is the canonical level i iff
//   (a) its ids appear in node order as 0, 1, 2, ... (canonical numbering:
//       blocks ranked by their smallest node id, Section 3 "Numbering schemes");
//   (b) every node has the signature of its block's head, the block's smallest
//       node (no two nodes with different signatures share an id);
//   (c) the heads of different blocks have different signatures (no two
//       nodes with equal signatures get different ids);
// where sig_i(u) = (prev(u), the set of (edge label, prev(v)) over the
// out-edges (u, v)) -- Definition 3 with Proposition 2.
//
// Signatures are built exactly (sorted, duplicates removed) and compared
// through a 122-bit fingerprint: two polynomial hashes modulo the Mersenne
// prime 2^61 - 1 over the signature's words, with fixed bases.  (c) never
// accepts a wrong result (equal signatures have equal fingerprints); (b) could
// only accept one if two different signatures of at most L words collided in
// both hashes, probability at most (L / 2^61)^2 per pair -- below 2^-50 over
// a 256M-node graph with signatures of up to 2M words.  The fingerprint is
// unrelated to the signature hash of the CUDA path, and nothing here is shared
// with it.  Nodes are processed in parallel by std::thread workers.
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

const uint64_t kP = (1ull << 61) - 1;
const uint64_t kBaseA = 0x1f2e3d4c5b6a7988ull % kP;
const uint64_t kBaseB = 0x0a1b2c3d4e5f6071ull % kP;
const uint32_t kDead = 0xFFFFFFFFu;

uint64_t mulmod(uint64_t a, uint64_t b) {
  const unsigned __int128 z = (unsigned __int128)a * b;
  uint64_t lo = (uint64_t)(z & kP), hi = (uint64_t)(z >> 61);
  uint64_t r = lo + hi;
  if (r >= kP) r -= kP;
  return r;
}

struct Fp {
  uint64_t a, b;
  bool operator==(const Fp& o) const { return a == o.a && b == o.b; }
  bool operator<(const Fp& o) const { return a != o.a ? a < o.a : b < o.b; }
};

struct Hasher {
  uint64_t a = 0, b = 0;
  void add(uint32_t w) {  // one 32-bit word (< p)
    a = mulmod(a, kBaseA) + w;
    if (a >= kP) a -= kP;
    b = mulmod(b, kBaseB) + w;
    if (b >= kP) b -= kP;
  }
};

template <typename LabelT>
Fp signature_fp(uint64_t u, const uint64_t* off, const uint32_t* dst, const LabelT* lab, const uint32_t* prev,
                std::vector<uint64_t>& buf) {
  buf.clear();
  for (uint64_t e = off[u]; e < off[u + 1]; ++e) buf.push_back(((uint64_t)lab[e] << 32) | prev[dst[e]]);
  std::sort(buf.begin(), buf.end());
  buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
  Hasher h;
  h.add(prev[u]);
  h.add((uint32_t)buf.size());
  h.add((uint32_t)(buf.size() >> 32));
  for (uint64_t x : buf) {
    h.add((uint32_t)(x >> 32));
    h.add((uint32_t)x);
  }
  return Fp{h.a, h.b};
}

template <typename LabelT>
int check(uint64_t n, const uint64_t* off, const uint32_t* dst, const LabelT* lab, const uint32_t* prev,
          const uint32_t* cur, int threads, uint64_t* count, uint64_t* bad) {
  // (a) canonical numbering; heads
  std::vector<uint64_t> head;
  for (uint64_t u = 0; u < n; ++u) {
    if (prev[u] == kDead) {
      if (cur[u] != kDead) { *bad = u; return 1; }
      continue;
    }
    if (cur[u] == head.size()) head.push_back(u);
    else if (cur[u] > head.size()) { *bad = u; return 1; }
  }
  *count = head.size();
  // fingerprints of all signatures
  std::vector<Fp> fp(n);
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  const uint64_t chunk = 1 << 16;
  std::vector<uint64_t> next_chunk(1, 0);
  for (int t = 0; t < threads; ++t) {
    pool.emplace_back([&, t]() {
      std::vector<uint64_t> buf;
      for (uint64_t c = (uint64_t)t; c * chunk < n; c += (uint64_t)threads)
        for (uint64_t u = c * chunk; u < std::min(n, (c + 1) * chunk); ++u)
          if (prev[u] != kDead) fp[u] = signature_fp(u, off, dst, lab, prev, buf);
    });
  }
  for (auto& th : pool) th.join();
  // (b) every node carries its head's signature
  for (uint64_t u = 0; u < n; ++u)
    if (prev[u] != kDead && !(fp[u] == fp[head[cur[u]]])) { *bad = u; return 2; }
  // (c) heads of different blocks differ
  std::vector<std::pair<Fp, uint64_t>> hf(head.size());
  for (uint64_t b = 0; b < head.size(); ++b) hf[b] = std::make_pair(fp[head[b]], head[b]);
  std::sort(hf.begin(), hf.end());
  for (uint64_t b = 1; b < hf.size(); ++b)
    if (hf[b].first == hf[b - 1].first) { *bad = std::max(hf[b].second, hf[b - 1].second); return 3; }
  return 0;
}

}  // namespace

extern "C" {

// Check level cur against prev on a CSR graph (labels of label_bytes = 1 or 4
// bytes).  Returns 0 if cur is the canonical level, else 1 (not canonical),
// 2 (a node's signature differs from its head's) or 3 (two blocks have equal
// signatures), with the offending node in *bad.  *count receives the number
// of blocks of cur.
int oracle_check_level(uint64_t n, const uint64_t* off, const uint32_t* dst, const void* lab, int label_bytes,
                       const uint32_t* prev, const uint32_t* cur, int threads, uint64_t* count, uint64_t* bad) {
  *bad = 0;
  *count = 0;
  if (label_bytes == 1)
    return check(n, off, dst, static_cast<const uint8_t*>(lab), prev, cur, threads, count, bad);
  return check(n, off, dst, static_cast<const uint32_t*>(lab), prev, cur, threads, count, bad);
}

}  // extern "C"
