// Host-side grid description: patches, node classes and interface tables.
//
// A patch is one refinement box of one level (level 0 is the whole domain).
// Its nodes are stored densely over a storage box (the bounding box of the
// nodes it owns), x padded to a multiple of 32, populations as 27 planes.
//
// Node classes (one byte per stored node) decide which kernel writes a node:
//   T_BULK  fluid, all 27 pull sources are plain stored nodes (fast path)
//   T_BC    fluid, some source lies beyond a wall / in a solid (bounce-back)
//           or beyond the outlet (clamped): generic pull
//   T_D1    child interface node at depth 1 (Sec. III, reconstruction or twin
//           layer): written by the explode kernel when the parent advances in
//           the same instant, by the generic stream-collide otherwise
//   T_D0    child interface node at depth 0: written by explode only
//   T_CF    parent twin node x_t,cf: written by the coalesce kernel
//   T_INLET fixed equilibrium inlet node, never written after init
//   T_SOLID solid node; T_SKIP no node (hole of a child, padding)
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

enum NodeType : uint8_t { T_SKIP = 0, T_BULK = 1, T_BC = 2, T_D1 = 3, T_D0 = 4, T_CF = 5, T_INLET = 6, T_SOLID = 7 };

// Reconstruction sample sources: a parent node (non-equilibrium rescaled to the
// child scale) or a child node (inside the parent hole, or under a parent twin).
enum SampleKind : uint8_t { S_PARENT = 0, S_CHILD = 1 };

struct HostPatch {
  int level = 0, parent = -1;
  std::vector<int> kids;
  int64_t blo[3]{}, bhi[3]{};  // box in parent coordinates (level >= 1)
  bool span[3]{};              // spans a periodic axis completely
  bool flo[3]{}, fhi[3]{};     // box faces that are interfaces toward the parent
  int64_t rlo[3]{}, rhi[3]{};  // region in this level's coordinates (inclusive)
  int64_t org[3]{}, dim[3]{};  // storage box
  int64_t nxp = 0, plane = 0;  // padded row length, nodes per population plane
  double beta = 0, beta1 = 0;
  std::vector<uint8_t> type;  // [z][y][nxp]
  int64_t n_fluid = 0;
  double n_bulk = 0, n_d1 = 0;  // BULK+BC nodes and D1 nodes (written by stream_collide)
  double n_bc = 0;              // BC nodes

  // stream-collide work lists: tiles of 128 nodes along x, id = (z*ny + y)*ntx + tx
  int64_t ntx = 0;
  // TMA path ([0] even, [1] odd substeps): x-tile | y<<16 | z<<32 | bounce mask<<48 | flags<<57
  std::vector<uint64_t> tiles_pure[2];
  // the same tiles as halves of 64 nodes (x-tile in units of 64; a half that
  // starts beyond the row is left out), for the 64-node tile variant
  std::vector<uint64_t> tiles_half[2];
  std::vector<uint32_t> tiles_mixed[2];  // other tiles with nodes to update: [0] even, [1] odd steps
  std::vector<uint32_t> tiles_all[2];    // every tile with nodes to update (thermal model, node by node)
  std::vector<uint32_t> fix_nodes[2];    // nodes of TMA tiles recomputed node by node after the tile pass
  double n_tma[2] = {0, 0};              // updated nodes the TMA pass gives (per parity)
  alignas(64) unsigned char tmap[2][128];   // TMA load descriptors of the two population buffers
  alignas(64) unsigned char tmapo[2][128];  // TMA store descriptors
  alignas(64) unsigned char tmapw[2][128];  // TMA 16-byte wrap descriptors
  alignas(64) unsigned char tmap64[2][128];  // TMA load descriptors of 64-node tiles
  alignas(64) unsigned char tmapg[2][128];   // the same three for the thermal g buffers
  alignas(64) unsigned char tmapgo[2][128];
  alignas(64) unsigned char tmapgw[2][128];

  // interface toward the parent (level >= 1).  Reconstruction values live in
  // a point space [0, n_points()): samples, then stage-1 points (off-lattice
  // along one axis), then stage-2 points (two axes), [value][point] in the
  // sample buffer.
  std::vector<uint32_t> ex_node;    // explode targets (nodes of this patch)
  std::vector<uint32_t> ex_src;     // 4 point ids per target (one-source targets use the first)
  uint32_t ex_one = 0;              // targets [0, ex_one) read one point, the rest interpolate four
  std::vector<uint32_t> pt_src;     // 4 point ids per intermediate point (stage 1, then stage 2)
  uint32_t n_pt[2] = {0, 0};        // intermediate points per stage
  // the transpose of ex_src and pt_src, for the adjoint: for each point
  // column j, use_ent[use_ptr[j] .. use_ptr[j + 1]) lists the consumers that
  // read it, each a target or a point id (bit 31 set: point) with its weight
  // (bit 30 set: weight 1, a one-point target; else bits 28-29 the source slot
  // of the four-point rule), in target order, then point order
  std::vector<uint32_t> use_ptr, use_ent;
  std::vector<uint32_t> smp_node;   // per sample: node index in parent or child
  std::vector<uint8_t> smp_kind;    // per sample: S_PARENT / S_CHILD
  std::vector<uint32_t> cf_parent;  // coalesce: parent twin node
  std::vector<uint32_t> cf_child;   // coalesce: coinciding child node
  // momentum exchange: fluid nodes next to a solid node, bit j set when x + c_j is solid
  std::vector<uint32_t> drag_node, drag_mask;
  // curved solid surface: per drag node k, wq[27 k + j] the fraction of the
  // link along c_j at which the wall lies (1/2 on other links); wq_idx over
  // the storage box gives k, -1 for nodes without solid links.  Empty without
  // an analytic surface.
  std::vector<double> wq;
  std::vector<int32_t> wq_idx;

  // device placement (byte offsets into the bound buffer)
  size_t off_f[2]{}, off_g[2]{}, off_type = 0;
  size_t off_tiles_pure[2]{}, off_tiles_half[2]{}, off_tiles_mixed[2]{}, off_tiles_all[2]{}, off_fix_nodes[2]{};
  size_t off_ex_node = 0, off_ex_src = 0, off_pt_src = 0, off_use_ptr = 0, off_use_ent = 0;
  size_t off_smp_node = 0, off_smp_kind = 0, off_smp_val = 0, off_cf_parent = 0, off_cf_child = 0;
  size_t off_drag_node = 0, off_drag_mask = 0, off_wq = 0, off_wq_idx = 0;
  int cur = 0;  // which population buffer holds the current state
  size_t n_points() const { return smp_node.size() + n_pt[0] + n_pt[1]; }
};

struct HostGrid {
  lbm_desc desc{};
  std::vector<lbm_box> boxes;
  std::vector<uint8_t> solid;
  std::vector<HostPatch> P;
  int nlev = 1;
  bool thermal = false;
  bool pr_gt1 = false;  // thermal model in the Pr > 1 regime (Table I)
  size_t pop_bytes = 4;   // bytes per stored population value
  size_t real_bytes = 4;  // bytes of the compute type (samples, outputs)

  bool periodic(int a) const { return (desc.periodic >> a) & 1u; }
  bool wall(int a, int side) const { return (desc.walls >> (2 * a + side)) & 1u; }
  int64_t period(int lev, int a) const { return (int64_t)desc.n[a] << lev; }
  int64_t maxc(int lev, int a) const { return (int64_t)(desc.n[a] - 1) << lev; }
};

// Builds patches, node classes and interface tables; validates the layout.
// Returns an empty string on success, else the reason.
std::string build_layout(HostGrid& g);

// Assigns byte offsets of every device array; returns the total size.
size_t plan_memory(HostGrid& g);

}  // namespace lbm
