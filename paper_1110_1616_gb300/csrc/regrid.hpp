// Regrid host logic (regrid.cpp): block clustering and transfer maps.
#pragma once
#include <array>
#include <cstdint>
#include <vector>

#include "hierarchy.hpp"

namespace amrmhd {

// New level-(l+1) boxes (level, lo[3], hi[3] in level-(l+1) cells) from the
// flagged level-l cells (x, y, z triples, global level-l indices): buffer the
// flags by 2 cells inside the level-l region, mark the aligned 4^dim blocks of
// level-l cells holding a buffered flag whose 3-cell surroundings lie in the
// region, merge them greedily in z,y,x order (x runs, then y, then z, at most 4
// blocks per side) and refine by 2.
std::vector<std::array<int, 7>> regrid_boxes(const Hierarchy& H, int l, const std::vector<int32_t>& flags);

// The clustering's frame on level l: the dense arrays cover n[3] cells from
// off[3] (the level region's bounding box aligned to the 4-cell blocks and
// widened by 2 blocks, or the whole extent where that does not fit, full[d]);
// nb[3] blocks per dimension.
struct ClusterFrame {
  int off[3], n[3], full[3], nb[3];
};
ClusterFrame cluster_frame(const Hierarchy& H, int l);

// The greedy z,y,x merge of the marked blocks (ok, nb[0] x nb[1] x nb[2]
// bytes; cleared as blocks are taken) into level-(l+1) boxes.
std::vector<std::array<int, 7>> merge_blocks(const Hierarchy& H, int l, const ClusterFrame& fr, uint8_t* ok);

struct TransferMaps {
  // boxes of the new patches' own cells (d = -1) and d-faces, GHOST_BOX_W ints
  // (dst, d, kind, src, lo[3], n[3], aux[3]), lo in dst's local coordinates:
  // kind 0 copies from old patch src at local offset aux, kind 1 prolongs from
  // the new coarse patch src holding the parent cell of the wrapped position
  // g + aux (for a face on the high side of a bounded domain, the last cell;
  // its coarse face is (g + aux) >> 1)
  std::vector<int32_t> boxes;
  std::vector<int32_t> closure;  // (dst, L of the first child) of prolonged coarse cells next to copied ones
};

// Maps filling level lf of the new hierarchy Hn from level lf of the old
// hierarchy Ho and level lf-1 of Hn. Returns 0, or < 0 if a source is missing.
int transfer_maps(const Hierarchy& Hn, const Hierarchy& Ho, int lf, TransferMaps& out);

// K (12 x 8, row-major, faces x children): the least-norm correction of the
// interior fine faces of a coarse cell that cancels the children's
// divergences r, delta = K r; idx: fine 1/dx per dimension.
void closure_matrix(int dim, const double* idx, double* K);

}  // namespace amrmhd
