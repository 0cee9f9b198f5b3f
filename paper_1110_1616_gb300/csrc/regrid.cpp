// Host side of the regrid: block clustering of flagged cells into new
// fine-level boxes, and the integer maps that transfer data into a new fine
// level (copy from the old fine level where it covered the parent cell, else
// prolongation from the new coarse level; divergence-free closure rows where
// prolonged coarse cells meet copied ones). Plain C++, no CUDA.
#include "regrid.hpp"

#include <algorithm>
#include <cmath>

namespace amrmhd {

namespace {

constexpr int kBlock = 4;     // block edge in coarse (level-l) cells
constexpr int kMaxBlocks = 4; // blocks per box side at most: 8..32 fine cells

struct Dense {  // a byte per cell of one level's domain
  int n[3];
  std::vector<uint8_t> v;
  size_t at(int i, int j, int k) const { return ((size_t)k * n[1] + j) * n[0] + i; }
};

}  // namespace

std::vector<std::array<int, 7>> regrid_boxes(const Hierarchy& H, int l, const std::vector<int32_t>& flags) {
  const int dim = H.dim;
  Dense region, buf;
  for (int d = 0; d < 3; ++d) region.n[d] = buf.n[d] = H.N(l, d);
  region.v.assign((size_t)region.n[0] * region.n[1] * region.n[2], 0);
  buf.v.assign(region.v.size(), 0);
  for (int q : H.level_patches[l]) {
    const HPatch& P = H.p[q];
    for (int k = P.lo[2]; k < P.hi[2]; ++k)
      for (int j = P.lo[1]; j < P.hi[1]; ++j)
        for (int i = P.lo[0]; i < P.hi[0]; ++i) region.v[region.at(i, j, k)] = 1;
  }
  // position inside the domain (periodic wrap), false if outside a bounded side
  auto inside = [&](int* c) {
    for (int d = 0; d < dim; ++d) {
      if (H.per[d]) c[d] = H.wrapd(l, d, c[d]);
      else if (c[d] < 0 || c[d] >= region.n[d]) return false;
    }
    return true;
  };
  const int kz = dim == 3 ? 1 : 0;
  for (size_t f = 0; f + 2 < flags.size(); f += 3) {
    for (int c = -2 * kz; c <= 2 * kz; ++c)
      for (int b = -2; b <= 2; ++b)
        for (int a = -2; a <= 2; ++a) {
          int p[3] = {flags[f] + a, flags[f + 1] + b, dim == 3 ? flags[f + 2] + c : 0};
          if (!inside(p)) continue;
          const size_t q = region.at(p[0], p[1], p[2]);
          if (region.v[q]) buf.v[q] = 1;
        }
  }
  int nb[3];
  for (int d = 0; d < 3; ++d) nb[d] = d < dim ? region.n[d] / kBlock : 1;
  auto bi = [&](int a, int b, int c) { return ((size_t)c * nb[1] + b) * nb[0] + a; };
  // blocks holding a buffered flag (found from the flags' neighbourhoods)
  std::vector<uint8_t> want((size_t)nb[0] * nb[1] * nb[2], 0);
  std::vector<size_t> wanted;
  for (size_t f = 0; f + 2 < flags.size(); f += 3)
    for (int c = -2 * kz; c <= 2 * kz; ++c)
      for (int b = -2; b <= 2; ++b)
        for (int a = -2; a <= 2; ++a) {
          int p[3] = {flags[f] + a, flags[f + 1] + b, dim == 3 ? flags[f + 2] + c : 0};
          if (!inside(p)) continue;
          if (!buf.v[buf.at(p[0], p[1], p[2])]) continue;
          const size_t w = bi(p[0] / kBlock, p[1] / kBlock, dim == 3 ? p[2] / kBlock : 0);
          if (!want[w]) { want[w] = 1; wanted.push_back(w); }
        }
  std::sort(wanted.begin(), wanted.end());
  std::vector<uint8_t> ok((size_t)nb[0] * nb[1] * nb[2], 0);
  for (size_t w : wanted) {
    const int a = (int)(w % nb[0]), b = (int)((w / nb[0]) % nb[1]), c = (int)(w / ((size_t)nb[0] * nb[1]));
    {
        const int lo[3] = {a * kBlock, b * kBlock, dim == 3 ? c * kBlock : 0};
        const int hi[3] = {lo[0] + kBlock, lo[1] + kBlock, dim == 3 ? lo[2] + kBlock : 1};
        // proper nesting: every cell within 3 of the block is in the region
        bool allowed = true;
        for (int k = lo[2] - 3 * kz; k < hi[2] + 3 * kz && allowed; ++k)
          for (int j = lo[1] - 3; j < hi[1] + 3 && allowed; ++j)
            for (int i = lo[0] - 3; i < hi[0] + 3 && allowed; ++i) {
              int p[3] = {i, j, k};
              if (!inside(p)) continue;
              if (!region.v[region.at(p[0], p[1], p[2])]) allowed = false;
            }
        if (allowed) ok[bi(a, b, c)] = 1;
    }
  }
  std::vector<std::array<int, 7>> out;
  for (size_t w : wanted) {
    const int a = (int)(w % nb[0]), b = (int)((w / nb[0]) % nb[1]), c = (int)(w / ((size_t)nb[0] * nb[1]));
    {
        if (!ok[w]) continue;
        int sx = 1, sy = 1, sz = 1;
        while (sx < kMaxBlocks && a + sx < nb[0] && ok[bi(a + sx, b, c)]) ++sx;
        auto row = [&](int bb, int cc) {
          for (int t = 0; t < sx; ++t)
            if (!ok[bi(a + t, bb, cc)]) return false;
          return true;
        };
        while (sy < kMaxBlocks && b + sy < nb[1] && row(b + sy, c)) ++sy;
        if (dim == 3) {
          auto slab = [&](int cc) {
            for (int u = 0; u < sy; ++u)
              if (!row(b + u, cc)) return false;
            return true;
          };
          while (sz < kMaxBlocks && c + sz < nb[2] && slab(c + sz)) ++sz;
        }
        for (int z = 0; z < sz; ++z)
          for (int y = 0; y < sy; ++y)
            for (int x = 0; x < sx; ++x) ok[bi(a + x, b + y, c + z)] = 0;
        std::array<int, 7> p;
        p[0] = l + 1;
        p[1] = 2 * kBlock * a;
        p[2] = 2 * kBlock * b;
        p[3] = dim == 3 ? 2 * kBlock * c : 0;
        p[4] = 2 * kBlock * (a + sx);
        p[5] = 2 * kBlock * (b + sy);
        p[6] = dim == 3 ? 2 * kBlock * (c + sz) : 1;
        out.push_back(p);
    }
  }
  return out;
}

int transfer_maps(const Hierarchy& Hn, const Hierarchy& Ho, int lf, TransferMaps& out) {
  const int dim = Hn.dim;
  const int lc = lf - 1;
  out.cells.clear();
  out.faces.clear();
  out.closure.clear();
  const bool have_old = Ho.nlev > lf;
  // old fine patches as boxes
  std::vector<int> oldp;
  if (have_old) oldp = Ho.level_patches[lf];
  auto old_cell = [&](const int* g, int* Lo) -> int {  // old fine patch holding fine cell g
    for (int q : oldp) {
      const HPatch& P = Ho.p[q];
      bool in = true;
      for (int d = 0; d < dim; ++d)
        if (g[d] < P.lo[d] || g[d] >= P.hi[d]) in = false;
      if (in) {
        if (Lo) *Lo = Ho.loc(q, g[0], g[1], g[2]);
        return q;
      }
    }
    return -1;
  };
  auto oldcov = [&](const int* c) -> bool {  // coarse cell c covered by the old fine level
    if (!have_old) return false;
    for (int d = 0; d < dim; ++d)
      if (!Hn.per[d] && (c[d] < 0 || c[d] >= Hn.N(lc, d))) return false;
    int g[3];
    for (int d = 0; d < 3; ++d) g[d] = d < dim ? 2 * Hn.wrapd(lc, d, c[d]) : 0;
    return old_cell(g, nullptr) >= 0;
  };
  // owner of fine d-face g in the old fine level: smallest (patch, local index)
  auto old_face = [&](int d, const int* g, int* Lo) -> int {
    int best = -1, bl = 0;
    for (int q : oldp) {
      const HPatch& P = Ho.p[q];
      bool in = true;
      for (int e = 0; e < dim; ++e) {
        if (e == d) { if (g[e] < P.lo[e] || g[e] > P.hi[e]) in = false; }
        else if (g[e] < P.lo[e] || g[e] >= P.hi[e]) in = false;
      }
      if (!in) continue;
      const int L = Ho.loc(q, g[0], g[1], g[2]);
      if (best < 0 || q < best || (q == best && L < bl)) { best = q; bl = L; }
    }
    *Lo = bl;
    return best;
  };
  // new coarse patch holding coarse cell c (after periodic wrap)
  auto coarse = [&](int qf, int* c, int* Lc) -> int {
    int w[3];
    for (int d = 0; d < 3; ++d) w[d] = d < dim ? Hn.wrapd(lc, d, c[d]) : 0;
    for (int Q : Hn.parents[qf]) {
      const HPatch& P = Hn.p[Q];
      bool in = true;
      for (int d = 0; d < dim; ++d)
        if (w[d] < P.lo[d] || w[d] >= P.hi[d]) in = false;
      if (in) {
        *Lc = Hn.loc(Q, w[0], w[1], w[2]);
        return Q;
      }
    }
    for (int Q : Hn.level_patches[lc]) {
      const HPatch& P = Hn.p[Q];
      bool in = true;
      for (int d = 0; d < dim; ++d)
        if (w[d] < P.lo[d] || w[d] >= P.hi[d]) in = false;
      if (in) {
        *Lc = Hn.loc(Q, w[0], w[1], w[2]);
        return Q;
      }
    }
    return -1;
  };
  const std::vector<int> all_old = oldp;
  for (int q : Hn.level_patches[lf]) {
    const HPatch& P = Hn.p[q];
    const int kz = dim == 3 ? 1 : 0;
    // old fine patches meeting this patch grown by 2 cells (periodic images included)
    oldp.clear();
    for (int o : all_old) {
      const HPatch& Q = Ho.p[o];
      bool meet = true;
      for (int d = 0; d < dim && meet; ++d) {
        const int n = Hn.N(lf, d);
        bool m = false;
        for (int sft = -1; sft <= 1; ++sft) {
          if (!Hn.per[d] && sft != 0) continue;
          if (Q.lo[d] + sft * n < P.hi[d] + 2 && P.lo[d] - 2 < Q.hi[d] + sft * n) m = true;
        }
        meet = m;
      }
      if (meet) oldp.push_back(o);
    }
    // cells
    for (int k = P.lo[2]; k < P.hi[2]; ++k)
      for (int j = P.lo[1]; j < P.hi[1]; ++j)
        for (int i = P.lo[0]; i < P.hi[0]; ++i) {
          int g[3] = {i, j, k};
          int c[3] = {i >> 1, j >> 1, dim == 3 ? k >> 1 : 0};
          const int L = Hn.loc(q, i, j, k);
          if (oldcov(c)) {
            int Lo = 0;
            const int o = old_cell(g, &Lo);
            out.cells.insert(out.cells.end(), {q, L, 0, o, Lo});
          } else {
            int Lc = 0;
            const int Q = coarse(q, c, &Lc);
            if (Q < 0) return -1;
            out.cells.insert(out.cells.end(), {q, L, 1, Q, Lc});
          }
        }
    // own faces
    for (int d = 0; d < dim; ++d) {
      int hi[3] = {P.hi[0], P.hi[1], P.hi[2]};
      hi[d] += 1;
      for (int k = P.lo[2]; k < hi[2]; ++k)
        for (int j = P.lo[1]; j < hi[1]; ++j)
          for (int i = P.lo[0]; i < hi[0]; ++i) {
            int g[3] = {i, j, k};
            int m[3] = {i, j, k};
            m[d] -= 1;
            int pq[3] = {i >> 1, j >> 1, dim == 3 ? k >> 1 : 0};
            int pm[3] = {m[0] >> 1, m[1] >> 1, dim == 3 ? m[2] >> 1 : 0};
            const bool interior = pq[d] == pm[d];
            const bool copy = interior ? oldcov(pq) : (oldcov(pq) || oldcov(pm));
            const int L = Hn.loc(q, i, j, k);
            if (copy) {
              int gw[3];
              for (int e = 0; e < 3; ++e) gw[e] = e < dim ? g[e] : 0;
              // the face as stored: wrap a periodic position into the domain
              for (int e = 0; e < dim; ++e)
                if (Hn.per[e] && (e != d || gw[e] != Hn.N(lf, e))) gw[e] = Hn.wrapd(lf, e, gw[e]);
              int Lo = 0;
              int o = old_face(d, gw, &Lo);
              if (o < 0 && Hn.per[d] && (gw[d] == 0 || gw[d] == Hn.N(lf, d))) {
                gw[d] = gw[d] == 0 ? Hn.N(lf, d) : 0;  // the other stored position of the seam face
                o = old_face(d, gw, &Lo);
              }
              if (o < 0) return -2;
              out.faces.insert(out.faces.end(), {q, d, L, 0, o, Lo});
            } else {
              // parent cell of the face position (the top face of a bounded domain
              // indexes one past the last coarse cell)
              int c[3] = {pq[0], pq[1], pq[2]};
              const bool top = !Hn.per[d] && g[d] == Hn.N(lf, d);
              if (top) c[d] -= 1;
              int Lc = 0;
              const int Q = coarse(q, c, &Lc);
              if (Q < 0) return -1;
              if (top) Lc += d == 0 ? 1 : (d == 1 ? Hn.p[Q].ext[0] : Hn.p[Q].ext[0] * Hn.p[Q].ext[1]);
              out.faces.insert(out.faces.end(), {q, d, L, 1, Q, Lc});
            }
          }
    }
    // closure rows: prolonged coarse cells with an old-covered face neighbour
    for (int ck = P.lo[2] >> kz; ck < (dim == 3 ? P.hi[2] >> 1 : 1); ++ck)
      for (int cj = P.lo[1] >> 1; cj < P.hi[1] >> 1; ++cj)
        for (int ci = P.lo[0] >> 1; ci < P.hi[0] >> 1; ++ci) {
          int c[3] = {ci, cj, ck};
          if (oldcov(c)) continue;
          bool touches = false;
          for (int d = 0; d < dim; ++d)
            for (int s = -1; s <= 1; s += 2) {
              int n[3] = {ci, cj, ck};
              n[d] += s;
              touches |= oldcov(n);
            }
          if (!touches) continue;
          out.closure.push_back(q);
          out.closure.push_back(Hn.loc(q, 2 * ci, 2 * cj, dim == 3 ? 2 * ck : 0));
        }
  }
  return 0;
}

void closure_matrix(int dim, const double* idx, double* K) {
  // M: child divergence per unit correction of each interior face; faces in
  // order d, then the transverse children in z,y,x bit order; children z,y,x.
  const int nc = dim == 3 ? 8 : 4, nt = dim == 3 ? 4 : 2, nf = dim * nt;
  double M[8][12] = {};
  int f = 0;
  for (int d = 0; d < dim; ++d)
    for (int t = 0; t < nt; ++t, ++f) {
      int o[3] = {0, 0, 0}, b = 0;
      for (int e = 0; e < dim; ++e) {
        if (e == d) continue;
        o[e] = (t >> b) & 1;
        ++b;
      }
      int lo[3] = {o[0], o[1], o[2]}, hi[3] = {o[0], o[1], o[2]};
      lo[d] = 0;
      hi[d] = 1;
      M[lo[0] + 2 * lo[1] + 4 * lo[2]][f] += idx[d];
      M[hi[0] + 2 * hi[1] + 4 * hi[2]][f] -= idx[d];
    }
  // inverse of G = M M^T + 1 1^T by Gauss-Jordan, then K = -M^T G^-1
  double G[8][16];
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < 2 * nc; ++j) {
      if (j < nc) {
        double s = 1.0;
        for (int k = 0; k < nf; ++k) s += M[i][k] * M[j][k];
        G[i][j] = s;
      } else {
        G[i][j] = (j - nc == i) ? 1.0 : 0.0;
      }
    }
  for (int c = 0; c < nc; ++c) {
    int piv = c;
    for (int i = c + 1; i < nc; ++i)
      if (std::fabs(G[i][c]) > std::fabs(G[piv][c])) piv = i;
    for (int j = 0; j < 2 * nc; ++j) std::swap(G[c][j], G[piv][j]);
    const double inv = 1.0 / G[c][c];
    for (int j = 0; j < 2 * nc; ++j) G[c][j] *= inv;
    for (int i = 0; i < nc; ++i) {
      if (i == c) continue;
      const double m = G[i][c];
      for (int j = 0; j < 2 * nc; ++j) G[i][j] -= m * G[c][j];
    }
  }
  for (int k = 0; k < nf; ++k)
    for (int c = 0; c < nc; ++c) {
      double s = 0.0;
      for (int i = 0; i < nc; ++i) s += M[i][k] * G[i][nc + c];
      K[k * 8 + c] = -s;
    }
}

}  // namespace amrmhd
