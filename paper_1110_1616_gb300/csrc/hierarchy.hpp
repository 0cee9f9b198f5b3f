// Host-side patch hierarchy: validation, neighbour lists by inheritance and
// the integer maps the kernels consume (ghost fill, prolongation, registers,
// restriction). Plain C++, no CUDA.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace amrmhd {

constexpr int GHOST_BOX_W = 13;

struct HPatch {
  int level;
  int lo[3], hi[3];
  int n[3];    // interior extent
  int ext[3];  // ghosted storage extent n+9 (1 on inactive z)
};

struct Nbr {
  int q;
  int s[3];
  bool operator<(const Nbr& o) const {
    if (q != o.q) return q < o.q;
    if (s[0] != o.s[0]) return s[0] < o.s[0];
    if (s[1] != o.s[1]) return s[1] < o.s[1];
    return s[2] < o.s[2];
  }
  bool operator==(const Nbr& o) const { return q == o.q && s[0] == o.s[0] && s[1] == o.s[1] && s[2] == o.s[2]; }
};

struct Hierarchy {
  int dim = 2;
  int base[3] = {1, 1, 1};
  bool per[3] = {true, true, true};        // periodic dimension
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // 0 periodic, 1 outflow, 2 inflow
  int max_level = 0;
  int nlev = 0;
  // partial builds (a regrid's intermediate stages): ghost boxes only for the
  // patches of levels >= ghost_from, register/reflux/restriction maps only
  // with with_registers; validation and neighbour lists are always complete
  int ghost_from = 0;
  bool with_registers = true;
  // ghost boxes made elsewhere (on the device, maps_dev.cu): build() leaves
  // ghost_box_cells and ghost_box_faces empty
  bool ghost_elsewhere = false;
  std::vector<HPatch> p;
  std::vector<std::vector<int>> level_patches;  // ids per level, ascending
  std::vector<std::vector<Nbr>> nbr;            // per patch, sorted by (q, shift)
  std::vector<std::vector<int>> parents, children;

  // ghost fill as boxes of GHOST_BOX_W ints: (dst patch, d (-1 cells, else the
  // d-faces), kind, src, lo[3], n[3], aux[3]) with lo in dst's local (ghosted,
  // 0-based) coordinates. kind 0: copy from patch src at local offset aux;
  // kind 1: prolongation from coarse patch src, parent of the wrapped fine
  // position (global g + aux) >> 1; kind 2: copy of dst's own position with
  // the coordinates aux[e] >= 0 replaced by aux[e] (clamped into the domain);
  // kind 3: the inflow state. Boxes of one patch cover its ghost positions once.
  std::vector<int32_t> ghost_box_cells, ghost_box_faces;
  // the same as one row per position (amrmhd.h row formats), made on demand by
  // expand_ghost_rows() (map export, the adjoint's transposed fills)
  std::vector<int32_t> ghost_cells;     // 5
  std::vector<int32_t> ghost_faces;     // 6
  bool ghost_rows_ready = false;
  // maps, rows of fixed width (see amrmhd.h for the row formats)
  std::vector<int32_t> cf_faces;        // 7
  std::vector<int32_t> cf_edges;        // 6
  std::vector<int32_t> emf_faces;       // 8
  std::vector<int32_t> restrict_cells;  // 5
  std::vector<int32_t> restrict_faces;  // 6
  std::vector<int32_t> reflux_cells;    // 9
  // per level row ranges [begin, end) of each list (rows are grouped by level:
  // ghost lists by the patch's level, register lists by the fine level l)
  std::vector<std::array<int64_t, 2>> rng_cf_faces, rng_cf_edges,
      rng_emf_faces, rng_restrict_cells, rng_restrict_faces, rng_reflux_cells;
  std::string err;

  int N(int l, int d) const { return d < dim ? (base[d] << l) : 1; }
  int wrapd(int l, int d, int i) const {
    if (!per[d]) return i;
    int n = N(l, d), r = i % n;
    return r < 0 ? r + n : r;
  }
  int loc(int q, int a, int b, int c) const;  // local index of level position (a,b,c)
  // Returns 0 or a negative amrmhd_status; fills err.
  int build(const int32_t* rows7, int n);
  void expand_ghost_rows();
};

}  // namespace amrmhd
