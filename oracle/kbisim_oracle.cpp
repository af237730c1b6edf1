// Plain CPU oracle for k-bisimulation partition identifiers.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
// reference that the CUDA path is checked against.  Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark may load it; the
// product library never links, loads or calls it, and the two share no code.
//
// What it computes (paper, Section 2 and Section 3):
//   * Definition 2: a k-partition identifier pId_0..pId_k with
//     pId_i(u) == pId_i(v)  <=>  u and v are i-bisimilar (Definition 1).
//   * Definition 3 + Proposition 2: pId_i is a one-to-one function of the
//     signature sig_i(u) = (first(u), { (lambda_E(u,u'), pId_{i-1}(u')) :
//     (u,u') in E }), where first(u) is pId_{i-1}(u) (the default; equivalent
//     by Proposition 1 and the Kaushik-definition equivalence in the appendix)
//     or pId_0(u) (Definition 3 as printed).
//   * Algorithm 1 (Build_Bisim): level 0 from node labels, then one
//     signature-to-identifier pass per level, with the signature storage S a
//     fresh ordered map per level whose counter starts at 0 and is filled in
//     node-id order.  That numbering ranks the blocks of each level by their
//     smallest node id (the canonical numbering; the paper allows any
//     numbering, Section 3.3 "Numbering schemes").
//   * Early stop (Section 3.3, proofs in the appendix "Partition splitting
//     stop condition"): after computing level i, if it has as many blocks as
//     level i-1, the partition is stable and levels i+1..k are copies.
//   * Full bisimulation (appendix, "Connection between localized bisimulation
//     and full bisimulation"): computed independently by naive splitting of
//     the label partition until it is stable with respect to itself
//     (the Paige-Tarjan style definition in the appendix).
//
// Edges are a multiset of (source, label, target) triples; signatures are
// sets, so repeated triples do not matter.  Nodes flagged dead (deleted)
// get the identifier 0xFFFFFFFF on every level, are not counted, and must
// have no incident edges.
//
// Single-threaded, std::map / std::vector only.  No blocking, no hashing, no
// reordering beyond what the algorithm states.

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace {

const uint32_t kDead = 0xFFFFFFFFu;

typedef std::pair<uint32_t, uint32_t> LabelPid;          // (edge label, child pId)
typedef std::pair<uint32_t, std::vector<LabelPid> > Sig;  // (first component, set as sorted vector)

struct Csr {
  std::vector<uint64_t> off;
  std::vector<uint32_t> dst;
  std::vector<uint32_t> lab;
};

// Group the edge list by source (counting sort).  Edge order inside a source
// is irrelevant: the signature sorts and deduplicates it.
Csr group_by_source(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                    const uint32_t* lab) {
  Csr g;
  g.off.assign(n + 1, 0);
  for (uint64_t e = 0; e < m; ++e) g.off[src[e] + 1]++;
  for (uint64_t u = 0; u < n; ++u) g.off[u + 1] += g.off[u];
  g.dst.resize(m);
  g.lab.resize(m);
  std::vector<uint64_t> cur(g.off.begin(), g.off.end() - 1);
  for (uint64_t e = 0; e < m; ++e) {
    uint64_t p = cur[src[e]]++;
    g.dst[p] = dst[e];
    g.lab[p] = lab[e];
  }
  return g;
}

bool valid_input(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 const uint8_t* alive) {
  for (uint64_t e = 0; e < m; ++e) {
    if (src[e] >= n || dst[e] >= n) return false;
    if (alive && (!alive[src[e]] || !alive[dst[e]])) return false;
  }
  return true;
}

}  // namespace

extern "C" {

// Level 0 (Algorithm 1, k = 0 branch): one identifier per distinct node label,
// handed out by a counter in node-id order.  Returns the number of blocks.
uint64_t oracle_level0(uint64_t n, const uint32_t* node_label, const uint8_t* alive,
                       uint32_t* pid0) {
  std::map<uint32_t, uint32_t> S;
  for (uint64_t u = 0; u < n; ++u) {
    if (alive && !alive[u]) { pid0[u] = kDead; continue; }
    std::map<uint32_t, uint32_t>::iterator it = S.find(node_label[u]);
    if (it == S.end()) it = S.insert(std::make_pair(node_label[u], (uint32_t)S.size())).first;
    pid0[u] = it->second;
  }
  return S.size();
}

// Algorithm 1 (Build_Bisim) in memory.
//   pids:   (k+1)*n identifiers, level-major (pids[i*n + u] = pId_i(u)).
//   counts: k+1 block counts.
//   first_component: 0 -> pId_{i-1}(u), 1 -> pId_0(u) as in Definition 3.
//   round_seconds (may be null): wall time of each computed round.
// Returns 0, or -1 on invalid input (an id >= n or an edge touching a dead node).
int oracle_kbisim(uint64_t n, const uint32_t* node_label, const uint8_t* alive, uint64_t m,
                  const uint32_t* src, const uint32_t* dst, const uint32_t* edge_label,
                  uint32_t k, int early_stop, int first_component, uint32_t* pids,
                  uint64_t* counts, uint32_t* rounds_run, double* round_seconds) {
  if (!valid_input(n, m, src, dst, alive)) return -1;
  Csr g = group_by_source(n, m, src, dst, edge_label);
  counts[0] = oracle_level0(n, node_label, alive, pids);
  *rounds_run = 0;
  for (uint32_t i = 1; i <= k; ++i) {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    const uint32_t* prev = pids + (uint64_t)(i - 1) * n;
    uint32_t* cur = pids + (uint64_t)i * n;
    std::map<Sig, uint32_t> S;  // fresh signature storage per level
    for (uint64_t u = 0; u < n; ++u) {
      if (alive && !alive[u]) { cur[u] = kDead; continue; }
      Sig s;
      s.first = first_component ? pids[u] : prev[u];
      for (uint64_t e = g.off[u]; e < g.off[u + 1]; ++e)
        s.second.push_back(LabelPid(g.lab[e], prev[g.dst[e]]));
      std::sort(s.second.begin(), s.second.end());
      s.second.erase(std::unique(s.second.begin(), s.second.end()), s.second.end());
      std::map<Sig, uint32_t>::iterator it = S.find(s);
      if (it == S.end()) it = S.insert(std::make_pair(s, (uint32_t)S.size())).first;
      cur[u] = it->second;
    }
    counts[i] = S.size();
    *rounds_run = i;
    if (round_seconds)
      round_seconds[i - 1] =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (early_stop && counts[i] == counts[i - 1]) {
      for (uint32_t j = i + 1; j <= k; ++j) {
        for (uint64_t u = 0; u < n; ++u) pids[(uint64_t)j * n + u] = cur[u];
        counts[j] = counts[i];
      }
      break;
    }
  }
  return 0;
}

// Full bisimulation by naive splitting (appendix: the coarsest partition that
// refines the label partition and is stable with respect to itself).
// Repeatedly, for every block B and edge label l, split every block C into
// C intersect parents_l(B) and C minus parents_l(B), until nothing splits.
// Output: canonical identifiers (blocks ranked by smallest node id) and the
// block count.  Cost is high; meant for small graphs.
int oracle_full_bisim(uint64_t n, const uint32_t* node_label, uint64_t m, const uint32_t* src,
                      const uint32_t* dst, const uint32_t* edge_label, uint32_t* block,
                      uint64_t* count) {
  if (!valid_input(n, m, src, dst, 0)) return -1;
  // in-edges grouped by target: parents of x with their labels
  Csr rev = group_by_source(n, m, dst, src, edge_label);
  std::vector<uint32_t> labels;
  {
    std::map<uint32_t, int> seen;
    for (uint64_t e = 0; e < m; ++e) seen[edge_label[e]] = 1;
    for (std::map<uint32_t, int>::iterator it = seen.begin(); it != seen.end(); ++it)
      labels.push_back(it->first);
  }
  uint64_t nb = oracle_level0(n, node_label, 0, block);
  std::vector<uint8_t> mark(n);
  bool changed = true;
  while (changed) {
    changed = false;
    for (uint64_t b = 0; b < nb; ++b) {
      for (size_t li = 0; li < labels.size(); ++li) {
        std::fill(mark.begin(), mark.end(), 0);
        for (uint64_t x = 0; x < n; ++x) {
          if (block[x] != b) continue;
          for (uint64_t e = rev.off[x]; e < rev.off[x + 1]; ++e)
            if (rev.lab[e] == labels[li]) mark[rev.dst[e]] = 1;
        }
        // split every block by the mark: (old block, mark) -> new block
        std::map<std::pair<uint32_t, int>, uint32_t> ids;
        std::vector<uint32_t> nxt(n);
        for (uint64_t u = 0; u < n; ++u) {
          std::pair<uint32_t, int> key(block[u], mark[u]);
          std::map<std::pair<uint32_t, int>, uint32_t>::iterator it = ids.find(key);
          if (it == ids.end()) it = ids.insert(std::make_pair(key, (uint32_t)ids.size())).first;
          nxt[u] = it->second;
        }
        if (ids.size() != nb) {
          changed = true;
          nb = ids.size();
        }
        for (uint64_t u = 0; u < n; ++u) block[u] = nxt[u];
      }
    }
  }
  *count = nb;
  return 0;
}

}  // extern "C"
