// Host side of the regrid: block clustering of flagged cells into new
// fine-level boxes, and the integer maps that transfer data into a new fine
// level (copy from the old fine level where it covered the parent cell, else
// prolongation from the new coarse level; divergence-free closure rows where
// prolonged coarse cells meet copied ones). Plain C++, no CUDA.
#include "regrid.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

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

ClusterFrame cluster_frame(const Hierarchy& H, int l) {
  // the dense arrays cover the level region's bounding box, aligned to blocks
  // and widened by the 3-cell nesting margin; a dimension whose widened box
  // reaches around the domain (periodic) or is bounded keeps the whole level
  // extent, so wrapped neighbours are found as before
  ClusterFrame f;
  const std::vector<int>& lp = H.level_patches[l];
  for (int d = 0; d < 3; ++d) {
    f.off[d] = 0;
    f.n[d] = H.N(l, d);
    f.full[d] = 1;
    if (d >= H.dim || lp.empty()) continue;
    int lo = f.n[d], hi = 0;
    for (int q : lp) {
      lo = std::min(lo, H.p[q].lo[d]);
      hi = std::max(hi, H.p[q].hi[d]);
    }
    lo = (lo / kBlock) * kBlock - 2 * kBlock;
    hi = ((hi + kBlock - 1) / kBlock) * kBlock + 2 * kBlock;
    if (lo >= 0 && hi <= f.n[d]) {
      f.full[d] = 0;
      f.off[d] = lo;
      f.n[d] = hi - lo;
    }
  }
  for (int d = 0; d < 3; ++d) f.nb[d] = d < H.dim ? f.n[d] / kBlock : 1;
  return f;
}

std::vector<std::array<int, 7>> merge_blocks(const Hierarchy& H, int l, const ClusterFrame& fr, uint8_t* ok) {
  const int dim = H.dim;
  const int* nb = fr.nb;
  const int* off = fr.off;
  auto bi = [&](int a, int b, int c) { return ((size_t)c * nb[1] + b) * nb[0] + a; };
  const size_t nblk = (size_t)nb[0] * nb[1] * nb[2];
  std::vector<std::array<int, 7>> out;
  for (size_t w = 0; w < nblk; ++w) {
    if (!ok[w]) {
      // skip runs of unmarked blocks 8 at a time
      while (w + 8 < nblk) {
        uint64_t v;
        std::memcpy(&v, ok + w + 1, 8);
        if (v) break;
        w += 8;
      }
      continue;
    }
    const int a = (int)(w % nb[0]), b = (int)((w / nb[0]) % nb[1]), c = (int)(w / ((size_t)nb[0] * nb[1]));
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
    p[1] = 2 * (kBlock * a + off[0]);
    p[2] = 2 * (kBlock * b + off[1]);
    p[3] = dim == 3 ? 2 * (kBlock * c + off[2]) : 0;
    p[4] = 2 * (kBlock * (a + sx) + off[0]);
    p[5] = 2 * (kBlock * (b + sy) + off[1]);
    p[6] = dim == 3 ? 2 * (kBlock * (c + sz) + off[2]) : 1;
    out.push_back(p);
  }
  return out;
}

std::vector<std::array<int, 7>> regrid_boxes(const Hierarchy& H, int l, const std::vector<int32_t>& flags) {
  const int dim = H.dim;
  const std::vector<int>& lp = H.level_patches[l];
  const ClusterFrame fr = cluster_frame(H, l);
  const int* off = fr.off;
  const int* full = fr.full;
  Dense region, buf;
  for (int d = 0; d < 3; ++d) region.n[d] = buf.n[d] = fr.n[d];
  const size_t ncell = (size_t)region.n[0] * region.n[1] * region.n[2];
  region.v.assign(ncell, 0);
  buf.v.assign(ncell, 0);
#pragma omp parallel for schedule(dynamic, 1)
  for (size_t ip = 0; ip < lp.size(); ++ip) {  // patches are disjoint: no shared writes
    const HPatch& P = H.p[lp[ip]];
    for (int k = P.lo[2]; k < P.hi[2]; ++k)
      for (int j = P.lo[1]; j < P.hi[1]; ++j)
        for (int i = P.lo[0]; i < P.hi[0]; ++i) region.v[region.at(i - off[0], j - off[1], k - off[2])] = 1;
  }
  // a local position inside the level domain (periodic wrap in a whole-extent
  // dimension), false if outside a bounded side; a position of a bounding-box
  // dimension outside the box is outside the region
  auto inside = [&](int* c, bool* in_box) {
    *in_box = true;
    for (int d = 0; d < dim; ++d) {
      if (full[d]) {
        if (H.per[d]) c[d] = H.wrapd(l, d, c[d]);
        else if (c[d] < 0 || c[d] >= region.n[d]) return false;
      } else {
        const int g = c[d] + off[d];
        if (!H.per[d] && (g < 0 || g >= H.N(l, d))) return false;
        if (c[d] < 0 || c[d] >= region.n[d]) *in_box = false;
      }
    }
    return true;
  };
  const int kz = dim == 3 ? 1 : 0;
  // buffer of 2 cells: the flags dilated (Chebyshev) along x, then y, then z,
  // then restricted to the region
  for (size_t f = 0; f + 2 < flags.size(); f += 3) {
    int c[3] = {flags[f] - off[0], flags[f + 1] - off[1], dim == 3 ? flags[f + 2] - off[2] : 0};
    bool ok = true;
    for (int d = 0; d < 3; ++d) ok = ok && c[d] >= 0 && c[d] < region.n[d];
    if (ok) buf.v[buf.at(c[0], c[1], c[2])] = 1;
  }
  for (int d = 0; d < dim; ++d) {
    const int n = region.n[d];
    const bool wrap = full[d] && H.per[d];
    const size_t st = d == 0 ? 1 : (d == 1 ? (size_t)region.n[0] : (size_t)region.n[0] * region.n[1]);
    const size_t lines = ncell / n;
    std::vector<uint8_t> src = buf.v;
#pragma omp parallel for schedule(static)
    for (long long li = 0; li < (long long)lines; ++li) {
      // the line's first element: li enumerates the other two coordinates
      size_t base;
      if (d == 0) base = (size_t)li * n;
      else if (d == 1) base = ((size_t)li / region.n[0]) * region.n[0] * n + (size_t)li % region.n[0];
      else base = (size_t)li;
      for (int x = 0; x < n; ++x) {
        if (!src[base + x * st]) continue;
        for (int o = -2; o <= 2; ++o) {
          int y = x + o;
          if (wrap) y = (y % n + n) % n;
          else if (y < 0 || y >= n) continue;
          buf.v[base + y * st] = 1;
        }
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (long long c = 0; c < (long long)ncell; ++c) buf.v[c] &= region.v[c];
  int nb[3];
  for (int d = 0; d < 3; ++d) nb[d] = d < dim ? region.n[d] / kBlock : 1;
  const size_t nblk = (size_t)nb[0] * nb[1] * nb[2];
  std::vector<uint8_t> ok(nblk, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (long long w = 0; w < (long long)nblk; ++w) {
    const int a = (int)(w % nb[0]), b = (int)((w / nb[0]) % nb[1]), c = (int)(w / ((size_t)nb[0] * nb[1]));
    const int lo[3] = {a * kBlock, b * kBlock, dim == 3 ? c * kBlock : 0};
    const int hi[3] = {lo[0] + kBlock, lo[1] + kBlock, dim == 3 ? lo[2] + kBlock : 1};
    bool want = false;
    for (int k = lo[2]; k < hi[2] && !want; ++k)
      for (int j = lo[1]; j < hi[1] && !want; ++j)
        for (int i = lo[0]; i < hi[0] && !want; ++i) want = buf.v[buf.at(i, j, k)] != 0;
    if (!want) continue;
    // proper nesting: every cell within 3 of the block is in the region
    bool allowed = true;
    for (int k = lo[2] - 3 * kz; k < hi[2] + 3 * kz && allowed; ++k)
      for (int j = lo[1] - 3; j < hi[1] + 3 && allowed; ++j)
        for (int i = lo[0] - 3; i < hi[0] + 3 && allowed; ++i) {
          int p[3] = {i, j, k};
          bool in_box;
          if (!inside(p, &in_box)) continue;
          if (!in_box || !region.v[region.at(p[0], p[1], p[2])]) allowed = false;
        }
    if (allowed) ok[w] = 1;
  }
  return merge_blocks(H, l, fr, ok.data());
}

int transfer_maps(const Hierarchy& Hn, const Hierarchy& Ho, int lf, TransferMaps& out) {
  const int dim = Hn.dim;
  const int lc = lf - 1;
  out.boxes.clear();
  out.closure.clear();
  const bool have_old = Ho.nlev > lf;
  const std::vector<int> empty;
  const std::vector<int>& oldp = have_old ? Ho.level_patches[lf] : empty;
  const std::vector<int>& newp = Hn.level_patches[lf];
  const int np = (int)newp.size();
  std::vector<TransferMaps> per(np);
  std::vector<int> status(np, 0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int ip = 0; ip < np; ++ip) {
    const int q = newp[ip];
    const HPatch& P = Hn.p[q];
    TransferMaps& o = per[ip];
    // owner map over the patch grown by 2 fine cells (unwrapped positions):
    // the old fine patch (and its periodic shift) holding each fine cell
    int glo[3], gex[3];
    for (int d = 0; d < 3; ++d) {
      glo[d] = d < dim ? P.lo[d] - 2 : 0;
      gex[d] = d < dim ? P.n[d] + 4 : 1;
    }
    const size_t gsz = (size_t)gex[0] * gex[1] * gex[2];
    std::vector<int> own(gsz, -1), shf(gsz, 0);
    auto gi = [&](const int* g) -> long long {
      for (int d = 0; d < 3; ++d)
        if (g[d] < glo[d] || g[d] >= glo[d] + gex[d]) return -1;
      return ((long long)(g[2] - glo[2]) * gex[1] + (g[1] - glo[1])) * gex[0] + (g[0] - glo[0]);
    };
    for (int oq : oldp) {
      const HPatch& Q = Ho.p[oq];
      int sr[3][2];
      for (int d = 0; d < 3; ++d) {
        const bool per = d < dim && Hn.per[d];
        sr[d][0] = per ? -1 : 0;
        sr[d][1] = per ? 1 : 0;
      }
      for (int sz = sr[2][0]; sz <= sr[2][1]; ++sz)
        for (int sy = sr[1][0]; sy <= sr[1][1]; ++sy)
          for (int sx = sr[0][0]; sx <= sr[0][1]; ++sx) {
            const int s3[3] = {sx, sy, sz};
            int a0[3], a1[3];
            bool any = true;
            for (int d = 0; d < 3; ++d) {
              const int off = d < dim ? s3[d] * Hn.N(lf, d) : 0;
              a0[d] = std::max(glo[d], (d < dim ? Q.lo[d] : 0) + off);
              a1[d] = std::min(glo[d] + gex[d], (d < dim ? Q.hi[d] : 1) + off);
              if (a1[d] <= a0[d]) any = false;
            }
            if (!any) continue;
            const int code = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
            for (int z = a0[2]; z < a1[2]; ++z)
              for (int y = a0[1]; y < a1[1]; ++y)
                for (int x = a0[0]; x < a1[0]; ++x) {
                  const int g[3] = {x, y, z};
                  const long long k = gi(g);
                  if (own[k] < 0) { own[k] = oq; shf[k] = code; }
                }
          }
    }
    // local index in the old patch of the position g seen through the owner's shift
    auto old_loc = [&](long long k, const int* g) {
      const int code = shf[k];
      const int s3[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
      int w[3];
      for (int d = 0; d < 3; ++d) w[d] = d < dim ? g[d] - s3[d] * Hn.N(lf, d) : 0;
      return Ho.loc(own[k], w[0], w[1], w[2]);
    };
    auto oldcov = [&](const int* c) -> bool {  // coarse cell c covered by the old fine level
      if (!have_old) return false;
      int g[3];
      for (int d = 0; d < 3; ++d) g[d] = d < dim ? 2 * c[d] : 0;
      const long long k = gi(g);
      return k >= 0 && own[k] >= 0;
    };
    // new coarse patch holding coarse cell c (after periodic wrap)
    auto coarse = [&](int* c, int* Lc) -> int {
      int w[3];
      for (int d = 0; d < 3; ++d) w[d] = d < dim ? Hn.wrapd(lc, d, c[d]) : 0;
      auto inside = [&](int Q) {
        const HPatch& C = Hn.p[Q];
        for (int d = 0; d < dim; ++d)
          if (w[d] < C.lo[d] || w[d] >= C.hi[d]) return false;
        return true;
      };
      for (int Q : Hn.parents[q])
        if (inside(Q)) { *Lc = Hn.loc(Q, w[0], w[1], w[2]); return Q; }
      for (int Q : Hn.level_patches[lc])
        if (inside(Q)) { *Lc = Hn.loc(Q, w[0], w[1], w[2]); return Q; }
      return -1;
    };
    // labels of the new patch's own cells and faces: a copy from old patch src at
    // local offset delta, or a prolongation from coarse patch src; positions
    // with equal labels are merged into boxes as for the ghost fill
    struct TLab {
      int kind, src, dl[3];
      bool operator==(const TLab& o) const {
        return kind == o.kind && src == o.src && dl[0] == o.dl[0] && dl[1] == o.dl[1] && dl[2] == o.dl[2];
      }
    };
    std::vector<TLab> labs;
    int last_id = -1;
    auto label_id = [&](const TLab& t) {
      if (last_id >= 0 && labs[last_id] == t) return last_id;
      for (size_t i = 0; i < labs.size(); ++i)
        if (labs[i] == t) return last_id = (int)i;
      labs.push_back(t);
      return last_id = (int)labs.size() - 1;
    };
    auto copy_label = [&](long long k) {
      const int code = shf[k];
      const int s3[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
      const HPatch& O = Ho.p[own[k]];
      TLab t{0, own[k], {0, 0, 0}};
      for (int d = 0; d < dim; ++d) t.dl[d] = P.lo[d] - O.lo[d] - s3[d] * Hn.N(lf, d);
      return t;
    };
    std::vector<int> lid;
    // greedy boxes (x runs, then y, then z) over a grid of label ids; ids are
    // cleared as positions are taken
    auto merge = [&](const int* ex, int d) {
      auto at = [&](int x, int y, int z) { return ((size_t)z * ex[1] + y) * ex[0] + x; };
      for (int c = 0; c < ex[2]; ++c)
        for (int b = 0; b < ex[1]; ++b)
          for (int a = 0; a < ex[0]; ++a) {
            const int k = lid[at(a, b, c)];
            if (k < 0) continue;
            int nx = 1, ny = 1, nz = 1;
            while (a + nx < ex[0] && lid[at(a + nx, b, c)] == k) ++nx;
            auto row_ok = [&](int y, int z) {
              for (int i = 0; i < nx; ++i)
                if (lid[at(a + i, y, z)] != k) return false;
              return true;
            };
            while (b + ny < ex[1] && row_ok(b + ny, c)) ++ny;
            auto slab_ok = [&](int z) {
              for (int j = 0; j < ny; ++j)
                if (!row_ok(b + j, z)) return false;
              return true;
            };
            while (c + nz < ex[2] && slab_ok(c + nz)) ++nz;
            for (int z = 0; z < nz; ++z)
              for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) lid[at(a + x, b + y, c + z)] = -1;
            const TLab& t = labs[k];
            const int32_t row[GHOST_BOX_W] = {q, d, t.kind, t.src, 4 + a, 4 + b, dim == 3 ? 4 + c : 0, nx, ny, nz,
                                              t.dl[0], t.dl[1], t.dl[2]};
            o.boxes.insert(o.boxes.end(), row, row + GHOST_BOX_W);
          }
    };
    // cells
    {
      const int ex[3] = {P.n[0], P.n[1], dim == 3 ? P.n[2] : 1};
      lid.assign((size_t)ex[0] * ex[1] * ex[2], -1);
      size_t t = 0;
      for (int k = P.lo[2]; k < P.hi[2] && !status[ip]; ++k)
        for (int j = P.lo[1]; j < P.hi[1] && !status[ip]; ++j)
          for (int i = P.lo[0]; i < P.hi[0]; ++i, ++t) {
            const int g[3] = {i, j, k};
            int c[3] = {i >> 1, j >> 1, dim == 3 ? k >> 1 : 0};
            if (oldcov(c)) {
              lid[t] = label_id(copy_label(gi(g)));
            } else {
              int Lc = 0;
              const int Q = coarse(c, &Lc);
              if (Q < 0) { status[ip] = -1; break; }
              lid[t] = label_id(TLab{1, Q, {0, 0, 0}});
            }
          }
      if (!status[ip]) merge(ex, -1);
    }
    // own faces
    for (int d = 0; d < dim && !status[ip]; ++d) {
      int hi[3] = {P.hi[0], P.hi[1], P.hi[2]};
      hi[d] += 1;
      const int ex[3] = {hi[0] - P.lo[0], hi[1] - P.lo[1], dim == 3 ? hi[2] - P.lo[2] : 1};
      lid.assign((size_t)ex[0] * ex[1] * ex[2], -1);
      size_t t = 0;
      for (int k = P.lo[2]; k < hi[2] && !status[ip]; ++k)
        for (int j = P.lo[1]; j < hi[1] && !status[ip]; ++j)
          for (int i = P.lo[0]; i < hi[0]; ++i, ++t) {
            const int g[3] = {i, j, k};
            int m[3] = {i, j, k};
            m[d] -= 1;
            int pq[3] = {i >> 1, j >> 1, dim == 3 ? k >> 1 : 0};
            int pm[3] = {m[0] >> 1, m[1] >> 1, dim == 3 ? m[2] >> 1 : 0};
            const bool interior = pq[d] == pm[d];
            const bool copy = interior ? oldcov(pq) : (oldcov(pq) || oldcov(pm));
            if (copy) {
              // owners of the face: the old patches holding the cells on its two sides;
              // the smallest (patch, local index) as for ghost faces
              int best = -1, bl = 0;
              long long bk = -1;
              const long long k1 = gi(g), k0 = gi(m);
              if (k1 >= 0 && own[k1] >= 0) { best = own[k1]; bl = old_loc(k1, g); bk = k1; }
              if (k0 >= 0 && own[k0] >= 0) {
                const int Lo = old_loc(k0, g);  // the same face position, in the low cell's patch
                if (best < 0 || own[k0] < best || (own[k0] == best && Lo < bl)) { best = own[k0]; bl = Lo; bk = k0; }
              }
              if (best < 0) { status[ip] = -2; break; }
              lid[t] = label_id(copy_label(bk));
            } else {
              int c[3] = {pq[0], pq[1], pq[2]};
              const bool top = !Hn.per[d] && g[d] == Hn.N(lf, d);
              if (top) c[d] -= 1;
              int Lc = 0;
              const int Q = coarse(c, &Lc);
              if (Q < 0) { status[ip] = -1; break; }
              // the periodic wrap of the face position (the face at N of a
              // periodic dimension is the coarse face 0 of the wrapped patch)
              TLab t1{1, Q, {0, 0, 0}};
              for (int e = 0; e < dim; ++e) t1.dl[e] = Hn.wrapd(lf, e, g[e]) - g[e];
              lid[t] = label_id(t1);
            }
          }
      if (!status[ip]) merge(ex, d);
    }
    // closure rows: prolonged coarse cells with an old-covered face neighbour
    const int kz = dim == 3 ? 1 : 0;
    for (int ck = P.lo[2] >> kz; ck < (dim == 3 ? P.hi[2] >> 1 : 1); ++ck)
      for (int cj = P.lo[1] >> 1; cj < P.hi[1] >> 1; ++cj)
        for (int ci = P.lo[0] >> 1; ci < P.hi[0] >> 1; ++ci) {
          int c[3] = {ci, cj, ck};
          if (oldcov(c)) continue;
          bool touches = false;
          for (int d = 0; d < dim; ++d)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              int nb[3] = {ci, cj, ck};
              nb[d] += sgn;
              // a neighbour outside a bounded domain is never covered
              bool in = true;
              for (int e = 0; e < dim; ++e)
                if (!Hn.per[e] && (nb[e] < 0 || nb[e] >= Hn.N(lc, e))) in = false;
              touches |= in && oldcov(nb);
            }
          if (!touches) continue;
          o.closure.push_back(q);
          o.closure.push_back(Hn.loc(q, 2 * ci, 2 * cj, dim == 3 ? 2 * ck : 0));
        }
  }
  for (int ip = 0; ip < np; ++ip) {
    if (status[ip]) return status[ip];
    out.boxes.insert(out.boxes.end(), per[ip].boxes.begin(), per[ip].boxes.end());
    out.closure.insert(out.closure.end(), per[ip].closure.begin(), per[ip].closure.end());
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
