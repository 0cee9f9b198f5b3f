// Oracle: brute-force construction of the integer maps of a patch hierarchy.
// TEST INFRASTRUCTURE ONLY (see amr_oracle.cpp): the product library builds the
// same lists with its own code (neighbour candidates by inheritance, Sec. 3.1);
// these are the plain definitions, each entry found by scanning every patch and
// every periodic image, so the two can be compared integer by integer.
//
// Conventions (canonical layout, reading R10):
//  * A patch p on level l has interior [lo, hi) in level-l cell indices. Its
//    ghosted storage box spans lo-4 .. hi+4 inclusive in each active
//    dimension: extent n+9 (cells use 0..n+7, faces along d use 0..n+8).
//    Local index of a level-l position g: L = a + gx*(b + gy*c) with
//    a = g_x - lo_x + 4 etc.; in 2D c = 0 and gz = 1.
//  * A d-face at position g (g_d = face index, the face at g_d - 1/2) is owned
//    by p when g_d is in [lo_d, hi_d] and the other coordinates in [lo, hi).
//  * Periodic images: shifts s in {-1,0,1}^dim times the level size.
//  * Neighbours: same-level q whose shifted interior meets p's ghosted box
//    widened by one cell, [lo-5, hi+5), so that every owner of one of p's ghost
//    faces is a neighbour.
//  * Face-copy lists (EMF_FACES, RESTRICT_FACES) hold every stored copy of a
//    face: each owner patch and, for a patch spanning the periodic domain, each
//    of its two representatives of the seam face.
//  * Kinds: 0 same-level copy, 1 prolongation from the parent level,
//    2 boundary copy (zero-gradient outflow: src is the patch itself, Lsrc the
//    nearest position inside the domain), 3 boundary inflow (src = Lsrc = -1).
//    A ghost cell outside the domain of a non-periodic dimension is a boundary
//    entry; so is a ghost face whose normal index lies beyond the boundary
//    face or whose cell lies outside along another dimension.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct P { int level, lo[3], hi[3]; };

struct H {
  int dim;
  int base[3];
  bool per[3] = {true, true, true};
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  std::vector<P> p;
  int N(int l, int d) const { return d < dim ? (base[d] << l) : 1; }
  int ext(int q, int d) const { return d < dim ? (p[q].hi[d] - p[q].lo[d]) + 9 : 1; }
  int loc(int q, const int* g) const {
    int a = g[0] - p[q].lo[0] + 4;
    int b = g[1] - p[q].lo[1] + 4;
    int c = dim == 3 ? g[2] - p[q].lo[2] + 4 : 0;
    return a + ext(q, 0) * (b + ext(q, 1) * c);
  }
};

static int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static bool cell_in(const P& q, const int* g, int dim) {
  for (int d = 0; d < dim; ++d) if (g[d] < q.lo[d] || g[d] >= q.hi[d]) return false;
  return true;
}
static bool face_owned(const P& q, const int* g, int d, int dim) {
  for (int e = 0; e < dim; ++e) {
    if (e == d) { if (g[e] < q.lo[e] || g[e] > q.hi[e]) return false; }
    else if (g[e] < q.lo[e] || g[e] >= q.hi[e]) return false;
  }
  return true;
}

// all shift vectors in {-1,0,1} per periodic dimension (0 otherwise),
// lexicographic (x most significant)
static const bool* g_per = nullptr;
static std::vector<std::vector<int>> shifts(int dim) {
  std::vector<std::vector<int>> out;
  const int nx = g_per[0] ? 1 : 0, ny = g_per[1] ? 1 : 0, nz = (dim == 3 && g_per[2]) ? 1 : 0;
  for (int sx = -nx; sx <= nx; ++sx)
    for (int sy = -ny; sy <= ny; ++sy)
      for (int sz = -nz; sz <= nz; ++sz) out.push_back({sx, sy, sz});
  return out;
}

// The same-level patch (and local index) whose interior holds the cell at g,
// scanning every patch and image; -1 if none.
static int find_cell(const H& h, int l, const int* g, int* L) {
  for (int q = 0; q < (int)h.p.size(); ++q) {
    if (h.p[q].level != l) continue;
    for (auto& s : shifts(h.dim)) {
      int gg[3] = {g[0] - s[0] * h.N(l, 0), g[1] - s[1] * h.N(l, 1), h.dim == 3 ? g[2] - s[2] * h.N(l, 2) : 0};
      if (cell_in(h.p[q], gg, h.dim)) { *L = h.loc(q, gg); return q; }
    }
  }
  return -1;
}

// Owner of a d-face with the smallest (patch, local index); -1 if none.
static int find_face(const H& h, int l, const int* g, int d, int* L) {
  int best = -1, bl = 0;
  for (int q = 0; q < (int)h.p.size(); ++q) {
    if (h.p[q].level != l) continue;
    for (auto& s : shifts(h.dim)) {
      int gg[3] = {g[0] - s[0] * h.N(l, 0), g[1] - s[1] * h.N(l, 1), h.dim == 3 ? g[2] - s[2] * h.N(l, 2) : 0};
      if (!face_owned(h.p[q], gg, d, h.dim)) continue;
      int li = h.loc(q, gg);
      if (best < 0 || q < best || (q == best && li < bl)) { best = q; bl = li; }
    }
  }
  if (best >= 0) *L = bl;
  return best;
}

// Every stored copy of a d-face: (patch, local index) over all owners and
// all periodic images (a patch spanning the domain stores the seam face twice).
static void face_owners(const H& h, int l, const int* g, int d, std::vector<std::pair<int, int>>& out) {
  out.clear();
  for (int q = 0; q < (int)h.p.size(); ++q) {
    if (h.p[q].level != l) continue;
    for (auto& s : shifts(h.dim)) {
      int gg[3] = {g[0] - s[0] * h.N(l, 0), g[1] - s[1] * h.N(l, 1), h.dim == 3 ? g[2] - s[2] * h.N(l, 2) : 0};
      if (!face_owned(h.p[q], gg, d, h.dim)) continue;
      std::pair<int, int> e = {q, h.loc(q, gg)};
      if (std::find(out.begin(), out.end(), e) == out.end()) out.push_back(e);
    }
  }
}

// Owner of the c-edge at position g (edge storage cell: the a,b face indices
// and the c cell index) with the smallest (patch, local index); -1 if none.
static int find_edge(const H& h, int l, const int* g, int c, int* L) {
  int best = -1, bl = 0;
  for (int q = 0; q < (int)h.p.size(); ++q) {
    if (h.p[q].level != l) continue;
    for (auto& s : shifts(h.dim)) {
      int gg[3] = {g[0] - s[0] * h.N(l, 0), g[1] - s[1] * h.N(l, 1), h.dim == 3 ? g[2] - s[2] * h.N(l, 2) : 0};
      bool ok = true;
      for (int e = 0; e < h.dim; ++e) {
        if (e == c) { if (gg[e] < h.p[q].lo[e] || gg[e] >= h.p[q].hi[e]) ok = false; }
        else if (gg[e] < h.p[q].lo[e] || gg[e] > h.p[q].hi[e]) ok = false;
      }
      if (!ok) continue;
      int li = h.loc(q, gg);
      if (best < 0 || q < best || (q == best && li < bl)) { best = q; bl = li; }
    }
  }
  if (best >= 0) *L = bl;
  return best;
}

static bool in_domain(const H& h, int l, const int* g) {
  for (int d = 0; d < h.dim; ++d)
    if (!h.per[d] && (g[d] < 0 || g[d] >= h.N(l, d))) return false;
  return true;
}
static int wrapd(const H& h, int l, int d, int i) { return h.per[d] ? wrapi(i, h.N(l, d)) : i; }

static bool covered(const H& h, int l, const int* gc) {
  // coarse cell gc on level l is covered by level l+1 (never outside the domain)
  if (!in_domain(h, l, gc)) return false;
  int g[3] = {2 * wrapd(h, l, 0, gc[0]), 2 * wrapd(h, l, 1, gc[1]), h.dim == 3 ? 2 * wrapd(h, l, 2, gc[2]) : 0};
  int L;
  return find_cell(h, l + 1, g, &L) >= 0;
}

static int nlevels(const H& h) {
  int m = 0;
  for (auto& q : h.p) m = std::max(m, q.level + 1);
  return m;
}

}  // namespace

extern "C" {

enum {
  MAP_NEIGHBORS = 0, MAP_GHOST_CELLS = 1, MAP_GHOST_FACES = 2, MAP_CF_FACES = 3,
  MAP_CF_EDGES = 4, MAP_EMF_FACES = 5, MAP_RESTRICT_CELLS = 6, MAP_RESTRICT_FACES = 7,
  MAP_REFLUX_CELLS = 8
};

// Builds map `which` for the hierarchy; rows of int32 appended to out (up to
// cap ints); *len receives the total number of ints. Returns the row width.
int oc_build_map2(int dim, const int* base, const int* bc, const int* patches, int n, int which, int* out,
                  long long cap, long long* len) {
  H h;
  h.dim = dim;
  for (int d = 0; d < 3; ++d) {
    h.base[d] = d < dim ? base[d] : 1;
    h.bc[d][0] = d < dim ? bc[2 * d] : 0;
    h.bc[d][1] = d < dim ? bc[2 * d + 1] : 0;
    h.per[d] = d >= dim || h.bc[d][0] == 0;
  }
  g_per = h.per;
  for (int i = 0; i < n; ++i) {
    P q;
    q.level = patches[7 * i];
    for (int d = 0; d < 3; ++d) { q.lo[d] = patches[7 * i + 1 + d]; q.hi[d] = patches[7 * i + 4 + d]; }
    h.p.push_back(q);
  }
  std::vector<int> v;
  int width = 0;
  const int np = (int)h.p.size();
  const int nl = nlevels(h);
  auto emit = [&](std::initializer_list<int> row) { for (int x : row) v.push_back(x); };

  if (which == MAP_NEIGHBORS) {
    width = 5;
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        if (h.p[b].level != h.p[a].level) continue;
        for (auto& s : shifts(dim)) {
          if (a == b && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
          bool hit = true;
          for (int d = 0; d < dim; ++d) {
            int lo = h.p[b].lo[d] + s[d] * h.N(h.p[a].level, d), hi = h.p[b].hi[d] + s[d] * h.N(h.p[a].level, d);
            if (hi <= h.p[a].lo[d] - 5 || lo >= h.p[a].hi[d] + 5) hit = false;
          }
          if (hit) emit({a, b, s[0], s[1], s[2]});
        }
      }
  } else if (which == MAP_GHOST_CELLS || which == MAP_GHOST_FACES) {
    width = which == MAP_GHOST_CELLS ? 5 : 6;
    for (int a = 0; a < np; ++a) {
      const P& q = h.p[a];
      int l = q.level;
      int nd = which == MAP_GHOST_CELLS ? 1 : dim;
      for (int d = 0; d < nd; ++d) {
        int ext[3];
        for (int e = 0; e < 3; ++e) ext[e] = e < dim ? (q.hi[e] - q.lo[e]) + 8 + (which == MAP_GHOST_FACES && e == d) : 1;
        for (int c = 0; c < ext[2]; ++c)
          for (int b = 0; b < ext[1]; ++b)
            for (int i = 0; i < ext[0]; ++i) {
              int g[3] = {q.lo[0] + i - 4, q.lo[1] + b - 4, dim == 3 ? q.lo[2] + c - 4 : 0};
              bool own = which == MAP_GHOST_CELLS ? cell_in(q, g, dim) : face_owned(q, g, d, dim);
              if (own) continue;
              int Ld = h.loc(a, g);
              int Ls = -1, src = -1, kind;
              // outside the domain of a non-periodic dimension: boundary entry
              bool out = false, inflow = false;
              int gc[3] = {g[0], g[1], g[2]};
              for (int e = 0; e < dim; ++e) {
                if (h.per[e]) continue;
                const int top = (which == MAP_GHOST_FACES && e == d) ? h.N(l, e) : h.N(l, e) - 1;
                if (g[e] < 0) { out = true; gc[e] = 0; inflow |= h.bc[e][0] == 2; }
                else if (g[e] > top) { out = true; gc[e] = top; inflow |= h.bc[e][1] == 2; }
              }
              if (out) {
                if (inflow) { kind = 3; src = -1; Ls = -1; }
                else { kind = 2; src = a; Ls = h.loc(a, gc); }
                if (which == MAP_GHOST_CELLS) emit({a, Ld, kind, src, Ls});
                else emit({a, d, Ld, kind, src, Ls});
                continue;
              }
              if (which == MAP_GHOST_CELLS) src = find_cell(h, l, g, &Ls);
              else src = find_face(h, l, g, d, &Ls);
              if (src >= 0) kind = 0;
              else {
                kind = 1;
                int gc[3];
                for (int e = 0; e < 3; ++e) gc[e] = e < dim ? (wrapd(h, l, e, g[e]) >> 1) : 0;
                // a face on the high side of a non-periodic domain lies on the
                // high face of the last coarse cell: search that cell, index the
                // coarse face position one past it
                const bool top_face = which == MAP_GHOST_FACES && !h.per[d] && g[d] == h.N(l, d);
                if (top_face) gc[d] -= 1;
                src = find_cell(h, l - 1, gc, &Ls);
                if (top_face && src >= 0) {
                  gc[d] += 1;
                  Ls = h.loc(src, gc);
                }
              }
              if (which == MAP_GHOST_CELLS) emit({a, Ld, kind, src, Ls});
              else emit({a, d, Ld, kind, src, Ls});
            }
      }
    }
  } else if (which == MAP_CF_FACES || which == MAP_REFLUX_CELLS || which == MAP_CF_EDGES ||
             which == MAP_EMF_FACES) {
    // C/F faces: rows (l, qc, d, Lface, side, pf, Lfine) sorted by (l, qc, d, Lface)
    std::vector<std::vector<int>> faces, edges;
    for (int l = 1; l < nl; ++l) {
      for (int qc = 0; qc < np; ++qc) {
        const P& c = h.p[qc];
        if (c.level != l - 1) continue;
        std::vector<std::vector<int>> rows;
        for (int d = 0; d < dim; ++d)
          for (int k = c.lo[2]; k < (dim == 3 ? c.hi[2] : 1); ++k)
            for (int j = c.lo[1]; j < c.hi[1]; ++j)
              for (int i = c.lo[0]; i < c.hi[0]; ++i) {
                int g[3] = {i, j, k};
                if (covered(h, l - 1, g)) continue;
                for (int side = 0; side < 2; ++side) {  // low face, high face of the uncovered cell
                  int gn[3] = {i, j, k};
                  gn[d] += side == 0 ? -1 : 1;
                  if (!covered(h, l - 1, gn)) continue;
                  int gf[3] = {i, j, k};
                  if (side == 1) gf[d] += 1;
                  // children of the covered cell, in the fine patch's frame
                  int ch[3];
                  for (int e = 0; e < 3; ++e) ch[e] = e < dim ? 2 * wrapd(h, l - 1, e, gn[e]) : 0;
                  int Lc;
                  int pf = find_cell(h, l, ch, &Lc);
                  int ff[3] = {ch[0], ch[1], ch[2]};
                  if (side == 0) ff[d] += 2;  // covered cell on the low side: its high face
                  // ff is in pf's frame up to a period: bring it into pf's closure
                  for (int e = 0; e < dim; ++e) {
                    if (!h.per[e]) continue;
                    int Ne = h.N(l, e);
                    while (ff[e] > h.p[pf].hi[e]) ff[e] -= Ne;
                    while (ff[e] < h.p[pf].lo[e]) ff[e] += Ne;
                  }
                  rows.push_back({l, qc, d, h.loc(qc, gf), side == 0 ? 1 : -1, pf, h.loc(pf, ff)});
                }
              }
        std::sort(rows.begin(), rows.end());
        for (auto& r : rows) faces.push_back(r);
      }
      // C/F edges: rows (l, qc, c, Ledge, pf, Lfine) over the lowest-ID owner qc
      std::vector<std::vector<int>> erows;
      for (int ce = 0; ce < 3; ++ce) {
        if (dim == 2 && ce != 2) continue;
        int a = (ce + 1) % 3, b = (ce + 2) % 3;
        int Nc[3] = {h.N(l - 1, 0), h.N(l - 1, 1), h.N(l - 1, 2)};
        int Ne[3] = {Nc[0], Nc[1], Nc[2]};
        for (int e = 0; e < dim; ++e)
          if (e != ce && !h.per[e]) Ne[e] += 1;
        for (int k = 0; k < Ne[2]; ++k)
          for (int j = 0; j < Ne[1]; ++j)
            for (int i = 0; i < Ne[0]; ++i) {
              int g[3] = {i, j, k};
              int ncov = 0, cpf = -1;
              int firstcov[3] = {0, 0, 0};
              for (int sb = -1; sb <= 0; ++sb)
                for (int sa = -1; sa <= 0; ++sa) {
                  int gn[3] = {i, j, k};
                  gn[a] += sa; gn[b] += sb;
                  if (covered(h, l - 1, gn)) {
                    ++ncov;
                    (void)firstcov;
                  }
                }
              if (ncov < 1 || ncov > 3) continue;
              int Le;
              int qc = find_edge(h, l - 1, g, ce, &Le);
              int gf[3] = {2 * i, 2 * j, dim == 3 ? 2 * k : 0};
              int Lf;
              cpf = find_edge(h, l, gf, ce, &Lf);
              erows.push_back({l, qc, ce, Le, cpf, Lf});
            }
      }
      std::sort(erows.begin(), erows.end());
      for (auto& r : erows) edges.push_back(r);
    }
    if (which == MAP_CF_FACES) {
      width = 7;
      for (auto& r : faces) for (int x : r) v.push_back(x);
    } else if (which == MAP_CF_EDGES) {
      width = 6;
      for (auto& r : edges) for (int x : r) v.push_back(x);
    } else if (which == MAP_REFLUX_CELLS) {
      // rows (l, qc, Lcell, f0..f5): C/F face row indices for faces x-,x+,y-,y+,z-,z+
      width = 9;
      std::vector<std::vector<int>> rows;
      for (size_t r = 0; r < faces.size(); ++r) {
        auto& f = faces[r];
        int l = f[0], qc = f[1], d = f[2], Lf = f[3], side = f[4];
        int sd = 1;
        for (int e = 0; e < d; ++e) sd *= h.ext(qc, e);
        int Lcell = side == 1 ? Lf : Lf - sd;
        int slot = 2 * d + (side == 1 ? 0 : 1);
        bool found = false;
        for (auto& row : rows)
          if (row[0] == l && row[1] == qc && row[2] == Lcell) { row[3 + slot] = (int)r; found = true; }
        if (!found) {
          std::vector<int> row = {l, qc, Lcell, -1, -1, -1, -1, -1, -1};
          row[3 + slot] = (int)r;
          rows.push_back(row);
        }
      }
      std::sort(rows.begin(), rows.end());
      for (auto& r : rows) for (int x : r) v.push_back(x);
    } else {
      // EMF faces: every owner copy of a coarse face with both cells uncovered
      // that touches a C/F edge; rows (l, qc, d, Lface, e0, e1, e2, e3) with the
      // C/F edge row indices (or -1). For a d-face with t1 = (d+1)%3,
      // t2 = (d+2)%3: slots 0,1 are the t2-component edges at the face's own
      // storage cell and one cell up along t1; slots 2,3 are the t1-component
      // edges at the storage cell and one cell up along t2. The correction is
      // +e0/dx_t1 - e1/dx_t1 - e2/dx_t2 + e3/dx_t2. In 2D only z-edges exist.
      width = 8;
      std::vector<std::vector<int>> rows;
      for (int l = 1; l < nl; ++l) {
        int Nc[3] = {h.N(l - 1, 0), h.N(l - 1, 1), h.N(l - 1, 2)};
        auto edge_row = [&](int c, const int* g) {
          int w[3] = {wrapd(h, l - 1, 0, g[0]), wrapd(h, l - 1, 1, g[1]), dim == 3 ? wrapd(h, l - 1, 2, g[2]) : 0};
          int Le;
          int qc = find_edge(h, l - 1, w, c, &Le);
          for (size_t r = 0; r < edges.size(); ++r)
            if (edges[r][0] == l && edges[r][1] == qc && edges[r][2] == c && edges[r][3] == Le) return (int)r;
          return -1;
        };
        for (int d = 0; d < dim; ++d)
          for (int k = 0; k < Nc[2] + ((d == 2 && !h.per[2]) ? 1 : 0); ++k)
            for (int j = 0; j < Nc[1] + ((d == 1 && !h.per[1]) ? 1 : 0); ++j)
              for (int i = 0; i < Nc[0] + ((d == 0 && !h.per[0]) ? 1 : 0); ++i) {
                int g[3] = {i, j, k};
                int gm[3] = {i, j, k};
                gm[d] -= 1;
                if (covered(h, l - 1, g) || covered(h, l - 1, gm)) continue;
                int e[4] = {-1, -1, -1, -1};
                const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                for (int slot = 0; slot < 4; ++slot) {
                  int comp = slot < 2 ? t2 : t1;
                  if (dim == 2 && comp != 2) continue;
                  int gs[3] = {i, j, k};
                  gs[slot < 2 ? t1 : t2] += slot & 1;
                  e[slot] = edge_row(comp, gs);
                }
                if (e[0] < 0 && e[1] < 0 && e[2] < 0 && e[3] < 0) continue;
                std::vector<std::pair<int, int>> own;
                face_owners(h, l - 1, g, d, own);
                for (auto& o : own) rows.push_back({l, o.first, d, o.second, e[0], e[1], e[2], e[3]});
              }
      }
      std::sort(rows.begin(), rows.end());
      for (auto& r : rows) for (int x : r) v.push_back(x);
    }
  } else if (which == MAP_RESTRICT_CELLS || which == MAP_RESTRICT_FACES) {
    width = which == MAP_RESTRICT_CELLS ? 5 : 6;
    std::vector<std::vector<int>> rows;
    for (int l = 1; l < nl; ++l) {
      int Nc[3] = {h.N(l - 1, 0), h.N(l - 1, 1), h.N(l - 1, 2)};
      if (which == MAP_RESTRICT_CELLS) {
        for (int qc = 0; qc < np; ++qc) {
          const P& c = h.p[qc];
          if (c.level != l - 1) continue;
          for (int k = c.lo[2]; k < (dim == 3 ? c.hi[2] : 1); ++k)
            for (int j = c.lo[1]; j < c.hi[1]; ++j)
              for (int i = c.lo[0]; i < c.hi[0]; ++i) {
                int g[3] = {i, j, k};
                int ch[3] = {2 * i, 2 * j, dim == 3 ? 2 * k : 0};
                int Lf;
                int pf = find_cell(h, l, ch, &Lf);
                if (pf < 0) continue;
                rows.push_back({l, qc, h.loc(qc, g), pf, Lf});
              }
        }
      } else {
        for (int d = 0; d < dim; ++d)
          for (int k = 0; k < Nc[2] + ((d == 2 && !h.per[2]) ? 1 : 0); ++k)
            for (int j = 0; j < Nc[1] + ((d == 1 && !h.per[1]) ? 1 : 0); ++j)
              for (int i = 0; i < Nc[0] + ((d == 0 && !h.per[0]) ? 1 : 0); ++i) {
                int g[3] = {i, j, k};
                int gm[3] = {i, j, k};
                gm[d] -= 1;
                if (!covered(h, l - 1, g) && !covered(h, l - 1, gm)) continue;
                int gf[3] = {2 * i, 2 * j, dim == 3 ? 2 * k : 0};
                int Lf;
                int pf = find_face(h, l, gf, d, &Lf);
                std::vector<std::pair<int, int>> own;
                face_owners(h, l - 1, g, d, own);
                for (auto& o : own) rows.push_back({l, o.first, d, o.second, pf, Lf});
              }
      }
    }
    std::sort(rows.begin(), rows.end());
    for (auto& r : rows) for (int x : r) v.push_back(x);
  } else {
    return -1;
  }
  *len = (long long)v.size();
  long long m = std::min<long long>(cap, (long long)v.size());
  if (out && m > 0) std::memcpy(out, v.data(), sizeof(int) * (size_t)m);
  return width;
}

int oc_build_map(int dim, const int* base, const int* patches, int n, int which, int* out, long long cap,
                 long long* len) {
  const int bc[6] = {0, 0, 0, 0, 0, 0};
  return oc_build_map2(dim, base, bc, patches, n, which, out, cap, len);
}

}  // extern "C"
