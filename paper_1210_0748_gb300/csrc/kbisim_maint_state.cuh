// Incremental maintenance state, held by every handle's Store.  Included by
// kbisim_internal.cuh after Buf (kept apart so that maintenance state and the
// round kernels' sources change independently).
#pragma once

#include <stdint.h>

#include <vector>

namespace kb {

// Incremental maintenance state (kbisim_maint.cu).  Level j of the
// maintained partition gives every node a stable label L_j: level 0 the node
// label itself, level j > 0 the label its signature
//   sig_j(u) = (L_{j-1}(u), { (edge label, L_{j-1}(v)) : (u, v) in E })
// has in the signature store S_j (the paper's S, one per level): a hash
// table from signature hash to label plus, per label, the signature itself
// (first component, element count, element words in a pool).  A label keeps
// its meaning across updates, so a node whose signature does not change keeps
// its label, and only changed labels propagate to parents (Algorithm 3).  A
// block all of whose members take one new signature that no label holds keeps
// its label too (the partition of the level is unchanged): the label is
// pointed at the new signature, and the old entry no longer matches anything.
struct MaintLevel {
  Buf lab;                  // uint32 [n] label of each node, original order (kDead: deleted)
  Buf tkey;                 // uint64 [tcap] signature hash of each slot (all ones: empty)
  Buf tval;                 // uint32 [tcap] label of each slot (kNone32 while being written)
  Buf sfirst, scount;       // uint32 [lcap] first component and element count of each label's signature
  Buf soff;                 // uint64 [lcap] first element word of each label in pool
  Buf pool;                 // uint64 [pcap] element words of the stored signatures
  Buf cnt;                  // uint32 [lcap] nodes holding each label
  Buf ctr;                  // uint64 [2] labels handed out, pool words used
  uint64_t tcap = 0, lcap = 0, pcap = 0;
  uint64_t entries = 0;     // table slots taken (those of re-pointed labels included)
};

struct MaintState {
  bool valid = false;
  uint32_t k = 0;                   // levels 1..k are maintained
  std::vector<MaintLevel> lv;       // [k + 1]; level 0 keeps only lab
  Buf fmask, fnext, changed, seeds; // bitmaps over internal ids
  Buf list, pend;                   // uint32 frontier list; pending head lookups
  Buf prev_int;                     // uint32 [n] labels of the level below, internal order
  Buf newlab;                       // uint32 [n] label found for each frontier head (internal id)
  Buf minid;                        // uint32 [lcap] smallest original id of each label
  Buf src;                          // uint32 staged sources of the batch's edges
  Buf misc;                         // uint64 scalars
  Buf woff;                         // uint64 [n + 1] pool offsets of the heads' signatures (build)
  Buf cmp;                          // hash set comparing one long signature with a stored one
  Buf cmp_info;                     // uint64 x 3 per pending comparison
  Buf big;                          // uint2 (node, label): long signatures copied by their own CTA
  Buf huge;                         // uint2 (node, label): the longest, copied by every CTA of a grid
  Buf coarse;                       // bit w: word w of the changed bitmap is non-zero
  Buf gold, gsize;                  // uint32 [n] per frontier group head: its members' old label,
                                    // member count (top bit: members of several old labels)
  Buf hit;                          // bitmap over labels: matched by a head in this level's lookups
  // last update
  int incremental = 0;              // 1 = frontier path, 0 = full recomputation
  int reason = 0;                   // why the last update recomputed everything (KBISIM_MAINT_*)
  uint64_t frontier_nodes = 0;      // nodes signed over all levels
  uint64_t levels = 0;              // levels processed
  int in_place = 0;                 // the batch was applied to the edge table in place
  // after a switch back for a large frontier: batches of at least this many
  // edges (same k) recompute at once, without stores (0 = none)
  uint64_t suspend_edges = 0;
  uint32_t suspend_k = 0;
  // measured cost of the two paths (host ms per maintained level, averaged
  // with weight 1/2 on the newest sample) and how many more updates
  // recompute because the frontier path measured dearer
  double ms_inc = 0, ms_rec = 0;
  uint32_t n_inc = 0, n_rec = 0;
  uint32_t cost_skip = 0;
  bool inc_warm = false;  // a frontier update has run on this handle (later ones are timed)
  // width of the element words the stores are built from: 32-bit when edge
  // label bits + pbits fit (pbits covers the node labels, which are the level-0
  // labels, and twice the node count, which bounds every later label)
  bool key32 = false;
  uint32_t pbits = 32;
};

}  // namespace kb
