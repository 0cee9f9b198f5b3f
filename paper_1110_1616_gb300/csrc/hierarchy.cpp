// Patch hierarchy builder (host). See hierarchy.hpp.
//
// Sec. 2: patches on levels with ratio 2, every level above 0 nested in the
// coarser one. Sec. 3.1: neighbour relations are inherited from the parents'
// relations -- the neighbours of a node's children are children of that node's
// neighbours (or siblings) -- so only level 0 needs a spatial search; every
// finer level's candidates come from its parents' neighbour lists.
#include "hierarchy.hpp"

#include <unordered_map>

#include <algorithm>
#include <map>
#include <tuple>

#include "../../include/amrmhd.h"

namespace amrmhd {

static inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

int Hierarchy::loc(int q, int a, int b, int c) const {
  const HPatch& P = p[q];
  int x = a - P.lo[0] + 4, y = b - P.lo[1] + 4, z = dim == 3 ? c - P.lo[2] + 4 : 0;
  return x + P.ext[0] * (y + P.ext[1] * z);
}

namespace {

// Uniform bins over one level, for the level-0 neighbour search and the parent search.
struct Bins {
  int N[3] = {1, 1, 1}, nb[3] = {1, 1, 1}, B = 16, dim = 2;
  bool per[3] = {true, true, true};
  std::vector<std::vector<int>> bin;
  std::vector<int> stamp;
  int tick = 0;
  void init(const Hierarchy& h, int l, int B_) {
    dim = h.dim;
    for (int d = 0; d < 3; ++d) per[d] = h.per[d];
    B = B_;
    for (int d = 0; d < 3; ++d) {
      N[d] = h.N(l, d);
      nb[d] = d < dim ? (N[d] + B - 1) / B : 1;
    }
    bin.assign((size_t)nb[0] * nb[1] * nb[2], {});
    stamp.assign(h.p.size(), -1);
    for (int q : h.level_patches[l]) {
      const HPatch& P = h.p[q];
      int b0[3], b1[3];
      for (int d = 0; d < 3; ++d) {
        b0[d] = d < dim ? P.lo[d] / B : 0;
        b1[d] = d < dim ? (P.hi[d] - 1) / B : 0;
      }
      for (int k = b0[2]; k <= b1[2]; ++k)
        for (int j = b0[1]; j <= b1[1]; ++j)
          for (int i = b0[0]; i <= b1[0]; ++i) bin[((size_t)k * nb[1] + j) * nb[0] + i].push_back(q);
    }
  }
  // All (q, s) whose interior shifted by s*N meets [lo, hi) (unwrapped).
  void query(const Hierarchy& h, const int* lo, const int* hi, bool only_zero_shift, std::vector<Nbr>& out) {
    const int xs = per[0] ? 1 : 0, ys = per[1] ? 1 : 0, zs = (dim == 3 && per[2]) ? 1 : 0;
    for (int sx = -xs; sx <= xs; ++sx)
      for (int sy = -ys; sy <= ys; ++sy)
        for (int sz = -zs; sz <= zs; ++sz) {
          int s[3] = {sx, sy, sz};
          if (only_zero_shift && (sx || sy || sz)) continue;
          int a[3], b[3];
          bool empty = false;
          for (int d = 0; d < 3; ++d) {
            if (d >= dim) { a[d] = 0; b[d] = 1; continue; }
            a[d] = std::max(lo[d] - s[d] * N[d], 0);
            b[d] = std::min(hi[d] - s[d] * N[d], N[d]);
            if (a[d] >= b[d]) empty = true;
          }
          if (empty) continue;
          ++tick;
          int b0[3], b1[3];
          for (int d = 0; d < 3; ++d) {
            b0[d] = d < dim ? a[d] / B : 0;
            b1[d] = d < dim ? (b[d] - 1) / B : 0;
          }
          for (int k = b0[2]; k <= b1[2]; ++k)
            for (int j = b0[1]; j <= b1[1]; ++j)
              for (int i = b0[0]; i <= b1[0]; ++i)
                for (int q : bin[((size_t)k * nb[1] + j) * nb[0] + i]) {
                  if (stamp[q] == tick) continue;
                  stamp[q] = tick;
                  const HPatch& P = h.p[q];
                  bool hit = true;
                  for (int d = 0; d < dim; ++d)
                    if (P.hi[d] <= a[d] || P.lo[d] >= b[d]) hit = false;
                  if (hit) out.push_back({q, {s[0], s[1], s[2]}});
                }
        }
  }
};

struct Key {
  int c, a, b, z;
  bool operator<(const Key& o) const { return std::tie(c, a, b, z) < std::tie(o.c, o.a, o.b, o.z); }
  bool operator==(const Key& o) const { return c == o.c && a == o.a && b == o.b && z == o.z; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)(uint32_t)k.c * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k.a + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k.b + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k.z + 0xBF58476D1CE4E5B9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};
struct PairHash {
  size_t operator()(const std::pair<int, int>& k) const {
    return (size_t)(((uint64_t)(uint32_t)k.first << 32) ^ (uint64_t)(uint32_t)k.second) * 0x9E3779B97F4A7C15ull;
  }
};

}  // namespace

int Hierarchy::build(const int32_t* rows7, int n) {
  err.clear();
  p.clear();
  ghost_cells.clear(); ghost_faces.clear(); cf_faces.clear(); cf_edges.clear();
  emf_faces.clear(); restrict_cells.clear(); restrict_faces.clear(); reflux_cells.clear();
  if (n <= 0) { err = "empty patch list"; return AMRMHD_EINVAL; }
  for (int d = 0; d < dim; ++d)
    if (base[d] < 8) { err = "base grid must have at least 8 cells per dimension"; return AMRMHD_EINVAL; }
  nlev = 0;
  for (int i = 0; i < n; ++i) {
    HPatch P;
    P.level = rows7[7 * i];
    for (int d = 0; d < 3; ++d) { P.lo[d] = rows7[7 * i + 1 + d]; P.hi[d] = rows7[7 * i + 4 + d]; }
    if (P.level < 0 || P.level > max_level) { err = "patch " + std::to_string(i) + ": level out of range"; return AMRMHD_EINVAL; }
    for (int d = 0; d < 3; ++d) {
      if (d >= dim) {
        if (P.lo[d] != 0 || P.hi[d] != 1) { err = "patch " + std::to_string(i) + ": 2D patches need z range [0,1)"; return AMRMHD_EINVAL; }
        P.n[d] = 1; P.ext[d] = 1;
        continue;
      }
      if (P.lo[d] < 0 || P.hi[d] > N(P.level, d) || P.hi[d] <= P.lo[d]) {
        err = "patch " + std::to_string(i) + ": box outside its level domain"; return AMRMHD_EINVAL;
      }
      if (P.level > 0 && ((P.lo[d] & 1) || (P.hi[d] & 1))) {
        err = "patch " + std::to_string(i) + ": box not aligned to parent cells"; return AMRMHD_EINVAL;
      }
      P.n[d] = P.hi[d] - P.lo[d];
      P.ext[d] = P.n[d] + 9;
    }
    nlev = std::max(nlev, P.level + 1);
    p.push_back(P);
  }
  const int np = (int)p.size();
  level_patches.assign(nlev, {});
  for (int i = 0; i < np; ++i) level_patches[p[i].level].push_back(i);
  for (int l = 0; l < nlev; ++l)
    if (level_patches[l].empty()) { err = "level " + std::to_string(l) + " has no patches"; return AMRMHD_EINVAL; }
  nbr.assign(np, {});
  parents.assign(np, {});
  children.assign(np, {});

  auto meets = [&](const HPatch& Q, const int* s, int l, const int* lo, const int* hi) {
    for (int d = 0; d < dim; ++d) {
      int a = Q.lo[d] + s[d] * N(l, d), b = Q.hi[d] + s[d] * N(l, d);
      if (b <= lo[d] || a >= hi[d]) return false;
    }
    return true;
  };
  auto finish_nbr = [&](int q, std::vector<Nbr>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    v.erase(std::remove_if(v.begin(), v.end(), [&](const Nbr& x) { return x.q == q && !x.s[0] && !x.s[1] && !x.s[2]; }),
            v.end());
  };
  auto check_overlap = [&](int q) {
    for (const Nbr& x : nbr[q]) {
      if (x.s[0] || x.s[1] || x.s[2]) continue;
      bool hit = true;
      for (int d = 0; d < dim; ++d)
        if (p[x.q].hi[d] <= p[q].lo[d] || p[x.q].lo[d] >= p[q].hi[d]) hit = false;
      if (hit) return true;
    }
    return false;
  };

  // level 0: spatial search
  {
    Bins b0;
    b0.init(*this, 0, 16);
    long long vol = 0;
    for (int q : level_patches[0]) {
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) { lo[d] = d < dim ? p[q].lo[d] - 5 : 0; hi[d] = d < dim ? p[q].hi[d] + 5 : 1; }
      b0.query(*this, lo, hi, false, nbr[q]);
      finish_nbr(q, nbr[q]);
      if (check_overlap(q)) { err = "level 0 patches overlap (patch " + std::to_string(q) + ")"; return AMRMHD_EOVERLAP; }
      vol += (long long)p[q].n[0] * p[q].n[1] * p[q].n[2];
    }
    if (vol != (long long)N(0, 0) * N(0, 1) * N(0, 2)) { err = "level 0 patches must tile the domain"; return AMRMHD_EINVAL; }
  }
  // finer levels: parents by search on the parent level, neighbours by inheritance
  for (int l = 1; l < nlev; ++l) {
    Bins bc;
    bc.init(*this, l - 1, 16);
    for (int q : level_patches[l]) {
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) { lo[d] = d < dim ? p[q].lo[d] / 2 : 0; hi[d] = d < dim ? p[q].hi[d] / 2 : 1; }
      std::vector<Nbr> par;
      bc.query(*this, lo, hi, true, par);
      std::sort(par.begin(), par.end());
      if (par.empty()) { err = "patch " + std::to_string(q) + " has no parent"; return AMRMHD_ENEST; }
      for (auto& x : par) { parents[q].push_back(x.q); children[x.q].push_back(q); }
    }
    for (int q : level_patches[l]) {
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) { lo[d] = d < dim ? p[q].lo[d] - 5 : 0; hi[d] = d < dim ? p[q].hi[d] + 5 : 1; }
      std::vector<Nbr> cand;
      for (int par : parents[q]) {
        std::vector<Nbr> pn = nbr[par];
        pn.push_back({par, {0, 0, 0}});
        for (const Nbr& x : pn)
          for (int c : children[x.q])
            if (meets(p[c], x.s, l, lo, hi)) cand.push_back({c, {x.s[0], x.s[1], x.s[2]}});
      }
      finish_nbr(q, cand);
      nbr[q] = cand;
      if (check_overlap(q)) { err = "level " + std::to_string(l) + " patches overlap (patch " + std::to_string(q) + ")"; return AMRMHD_EOVERLAP; }
    }
    // proper nesting: parent cells within 3 of every covered cell lie in the parent region
    for (int q : level_patches[l]) {
      int lo[3], hi[3];
      long long need = 1;
      for (int d = 0; d < 3; ++d) {
        if (d >= dim) { lo[d] = 0; hi[d] = 1; continue; }
        lo[d] = p[q].lo[d] / 2 - 3;
        hi[d] = p[q].hi[d] / 2 + 3;
        if (!per[d]) { lo[d] = std::max(lo[d], 0); hi[d] = std::min(hi[d], N(l - 1, d)); }
        else if (hi[d] - lo[d] >= N(l - 1, d)) { lo[d] = 0; hi[d] = N(l - 1, d); }
        need *= hi[d] - lo[d];
      }
      std::vector<Nbr> cov;
      bc.query(*this, lo, hi, false, cov);
      long long got = 0;
      for (const Nbr& x : cov) {
        long long v = 1;
        for (int d = 0; d < dim; ++d) {
          int a = std::max(lo[d], p[x.q].lo[d] + x.s[d] * N(l - 1, d));
          int b = std::min(hi[d], p[x.q].hi[d] + x.s[d] * N(l - 1, d));
          v *= std::max(0, b - a);
        }
        got += v;
      }
      if (got != need) { err = "patch " + std::to_string(q) + " violates proper nesting (3 parent cells)"; return AMRMHD_ENEST; }
    }
  }

  // ---------------- ghost maps (patches in parallel, rows concatenated in patch order)
  rng_ghost_cells.assign(nlev, {0, 0});
  rng_ghost_faces.assign(nlev, {0, 0});
  std::vector<std::vector<int32_t>> gc_rows(np), gf_rows(np);
  std::vector<std::string> gerr(np);
  std::vector<int> gst(np, 0);
  auto ghost_patch = [&](int q, std::vector<int32_t>& gcq, std::vector<int32_t>& gfq, std::string& errq) -> int {
    const HPatch& P = p[q];
    const int l = P.level;
    // coarse candidates for prolongation sources
    std::vector<int> cc;
    for (int par : parents[q]) {
      cc.push_back(par);
      for (const Nbr& x : nbr[par]) cc.push_back(x.q);
    }
    std::sort(cc.begin(), cc.end());
    cc.erase(std::unique(cc.begin(), cc.end()), cc.end());
    // parent cell of fine position g; for a d-face (dn >= 0) on the high side
    // of a non-periodic domain the parent is the last coarse cell and L indexes
    // the coarse face one past it
    int last_src = -1;
    auto coarse_src = [&](const int* g, int* L, int dn) {
      int c[3];
      for (int d = 0; d < 3; ++d) c[d] = d < dim ? (wrapd(l, d, g[d]) >> 1) : 0;
      const bool top = dn >= 0 && !per[dn] && g[dn] == N(l, dn);
      if (top) c[dn] -= 1;
      auto inside = [&](int Q) {
        for (int d = 0; d < dim; ++d)
          if (c[d] < p[Q].lo[d] || c[d] >= p[Q].hi[d]) return false;
        return true;
      };
      // consecutive positions usually share the parent patch: try the last one first
      int hit = (last_src >= 0 && inside(last_src)) ? last_src : -1;
      for (size_t i = 0; hit < 0 && i < cc.size(); ++i)
        if (inside(cc[i])) hit = cc[i];
      if (hit < 0) return -1;
      last_src = hit;
      if (top) c[dn] += 1;
      *L = loc(hit, c[0], c[1], c[2]);
      return hit;
    };
    // cells
    {
      int e[3];
      for (int d = 0; d < 3; ++d) e[d] = d < dim ? P.n[d] + 8 : 1;
      size_t tot = (size_t)e[0] * e[1] * e[2];
      std::vector<int> sq(tot, -1), sl(tot, 0);
      auto idx = [&](int a, int b, int c) { return ((size_t)(c - (dim == 3 ? P.lo[2] - 4 : 0)) * e[1] + (b - P.lo[1] + 4)) * e[0] + (a - P.lo[0] + 4); };
      for (const Nbr& x : nbr[q]) {
        const HPatch& Q = p[x.q];
        int a0[3], a1[3];
        for (int d = 0; d < 3; ++d) {
          if (d >= dim) { a0[d] = 0; a1[d] = 1; continue; }
          a0[d] = std::max(P.lo[d] - 4, Q.lo[d] + x.s[d] * N(l, d));
          a1[d] = std::min(P.hi[d] + 4, Q.hi[d] + x.s[d] * N(l, d));
        }
        for (int c = a0[2]; c < a1[2]; ++c)
          for (int b = a0[1]; b < a1[1]; ++b)
            for (int a = a0[0]; a < a1[0]; ++a) {
              size_t t = idx(a, b, c);
              sq[t] = x.q;
              sl[t] = loc(x.q, a - x.s[0] * N(l, 0), b - x.s[1] * N(l, 1), c - x.s[2] * N(l, 2));
            }
      }
      for (int c = (dim == 3 ? P.lo[2] - 4 : 0); c < (dim == 3 ? P.hi[2] + 4 : 1); ++c)
        for (int b = P.lo[1] - 4; b < P.hi[1] + 4; ++b)
          for (int a = P.lo[0] - 4; a < P.hi[0] + 4; ++a) {
            bool inner = a >= P.lo[0] && a < P.hi[0] && b >= P.lo[1] && b < P.hi[1] &&
                         (dim == 2 || (c >= P.lo[2] && c < P.hi[2]));
            if (inner) continue;
            {
              // outside the domain of a non-periodic dimension: boundary entry
              int g[3] = {a, b, c}, gc[3] = {a, b, c};
              bool out = false, inflow = false;
              for (int e = 0; e < dim; ++e) {
                if (per[e]) continue;
                if (g[e] < 0) { out = true; gc[e] = 0; inflow |= bc[e][0] == 2; }
                else if (g[e] > N(l, e) - 1) { out = true; gc[e] = N(l, e) - 1; inflow |= bc[e][1] == 2; }
              }
              if (out) {
                int row[5] = {q, loc(q, a, b, c), inflow ? 3 : 2, inflow ? -1 : q, inflow ? -1 : loc(q, gc[0], gc[1], gc[2])};
                gcq.insert(gcq.end(), row, row + 5);
                continue;
              }
            }
            size_t t = idx(a, b, c);
            int kind = 0, src = sq[t], L = sl[t];
            if (src < 0) {
              if (l == 0) { errq = "level-0 ghost cell without a source"; return AMRMHD_EINVAL; }
              int g[3] = {a, b, c};
              kind = 1;
              src = coarse_src(g, &L, -1);
              if (src < 0) { errq = "no parent-level source for the ghost cell (" + std::to_string(a) + ", " + std::to_string(b) + ", " +
                      std::to_string(c) + ") of patch " + std::to_string(q);
                return AMRMHD_ENEST;
              }
            }
            int row[5] = {q, loc(q, a, b, c), kind, src, L};
            gcq.insert(gcq.end(), row, row + 5);
          }
    }
    // faces
    for (int d = 0; d < dim; ++d) {
      int lo[3], hi[3];  // face box (inclusive-exclusive per dim)
      for (int e = 0; e < 3; ++e) {
        if (e >= dim) { lo[e] = 0; hi[e] = 1; continue; }
        lo[e] = P.lo[e] - 4;
        hi[e] = P.hi[e] + 4 + (e == d ? 1 : 0);
      }
      int ex[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
      size_t tot = (size_t)ex[0] * ex[1] * ex[2];
      std::vector<int> sq(tot, -1), sl(tot, 0);
      auto idx = [&](int a, int b, int c) { return ((size_t)(c - lo[2]) * ex[1] + (b - lo[1])) * ex[0] + (a - lo[0]); };
      for (const Nbr& x : nbr[q]) {
        const HPatch& Q = p[x.q];
        int a0[3], a1[3];
        for (int e = 0; e < 3; ++e) {
          if (e >= dim) { a0[e] = 0; a1[e] = 1; continue; }
          int qlo = Q.lo[e] + x.s[e] * N(l, e), qhi = Q.hi[e] + x.s[e] * N(l, e) + (e == d ? 1 : 0);
          a0[e] = std::max(lo[e], qlo);
          a1[e] = std::min(hi[e], qhi);
        }
        for (int c = a0[2]; c < a1[2]; ++c)
          for (int b = a0[1]; b < a1[1]; ++b)
            for (int a = a0[0]; a < a1[0]; ++a) {
              size_t t = idx(a, b, c);
              int L = loc(x.q, a - x.s[0] * N(l, 0), b - x.s[1] * N(l, 1), c - x.s[2] * N(l, 2));
              if (sq[t] < 0 || x.q < sq[t] || (x.q == sq[t] && L < sl[t])) { sq[t] = x.q; sl[t] = L; }
            }
      }
      for (int c = lo[2]; c < hi[2]; ++c)
        for (int b = lo[1]; b < hi[1]; ++b)
          for (int a = lo[0]; a < hi[0]; ++a) {
            int g[3] = {a, b, c};
            bool own = true;
            for (int e = 0; e < dim; ++e) {
              if (e == d) { if (g[e] < P.lo[e] || g[e] > P.hi[e]) own = false; }
              else if (g[e] < P.lo[e] || g[e] >= P.hi[e]) own = false;
            }
            if (own) continue;
            {
              int gc[3] = {a, b, c};
              bool out = false, inflow = false;
              for (int e = 0; e < dim; ++e) {
                if (per[e]) continue;
                const int top = e == d ? N(l, e) : N(l, e) - 1;
                if (g[e] < 0) { out = true; gc[e] = 0; inflow |= bc[e][0] == 2; }
                else if (g[e] > top) { out = true; gc[e] = top; inflow |= bc[e][1] == 2; }
              }
              if (out) {
                int row[6] = {q, d, loc(q, a, b, c), inflow ? 3 : 2, inflow ? -1 : q,
                              inflow ? -1 : loc(q, gc[0], gc[1], gc[2])};
                gfq.insert(gfq.end(), row, row + 6);
                continue;
              }
            }
            size_t t = idx(a, b, c);
            int kind = 0, src = sq[t], L = sl[t];
            if (src < 0) {
              if (l == 0) { errq = "level-0 ghost face without a source"; return AMRMHD_EINVAL; }
              kind = 1;
              src = coarse_src(g, &L, d);
              if (src < 0) { errq = "no parent-level source for the ghost face (" + std::to_string(d) + "; " + std::to_string(a) + ", " +
                      std::to_string(b) + ", " + std::to_string(c) + ") of patch " + std::to_string(q);
                return AMRMHD_ENEST;
              }
            }
            int row[6] = {q, d, loc(q, a, b, c), kind, src, L};
            gfq.insert(gfq.end(), row, row + 6);
          }
    }
      return 0;
  };
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < np; ++q) gst[q] = ghost_patch(q, gc_rows[q], gf_rows[q], gerr[q]);
  for (int q = 0; q < np; ++q)
    if (gst[q]) { err = gerr[q]; return gst[q]; }
  {
    size_t nc = 0, nf = 0;
    for (int q = 0; q < np; ++q) { nc += gc_rows[q].size(); nf += gf_rows[q].size(); }
    ghost_cells.reserve(nc);
    ghost_faces.reserve(nf);
    for (int q = 0; q < np; ++q) {
      ghost_cells.insert(ghost_cells.end(), gc_rows[q].begin(), gc_rows[q].end());
      ghost_faces.insert(ghost_faces.end(), gf_rows[q].begin(), gf_rows[q].end());
      std::vector<int32_t>().swap(gc_rows[q]);
      std::vector<int32_t>().swap(gf_rows[q]);
    }
  }

  // ---------------- register, reflux and restriction maps, per fine level
  rng_cf_faces.assign(nlev, {0, 0});
  rng_cf_edges.assign(nlev, {0, 0});
  rng_emf_faces.assign(nlev, {0, 0});
  rng_restrict_cells.assign(nlev, {0, 0});
  rng_restrict_faces.assign(nlev, {0, 0});
  rng_reflux_cells.assign(nlev, {0, 0});
  for (int l = 1; l < nlev; ++l) {
    const int lc = l - 1;
    rng_cf_faces[l][0] = (int64_t)cf_faces.size() / 7;
    rng_cf_edges[l][0] = (int64_t)cf_edges.size() / 6;
    rng_emf_faces[l][0] = (int64_t)emf_faces.size() / 8;
    rng_restrict_cells[l][0] = (int64_t)restrict_cells.size() / 5;
    rng_restrict_faces[l][0] = (int64_t)restrict_faces.size() / 6;
    rng_reflux_cells[l][0] = (int64_t)reflux_cells.size() / 9;
    // per coarse patch: cover map over its cells widened by one, entry (fine patch, shift)
    struct Cov { int c = -1; int s[3] = {0, 0, 0}; };
    std::unordered_map<Key, std::array<int, 4>, KeyHash> edge_best;  // key -> (qc, Le, pf, Lf)
    std::vector<std::vector<std::array<int, 7>>> face_rows(np);
    std::vector<std::vector<std::array<int, 5>>> rcell_rows(np);
    std::vector<std::vector<std::array<int, 6>>> rface_rows(np);
    std::vector<std::vector<Cov>> covmaps(np);
    auto covidx = [&](int qc, int a, int b, int c) {
      const HPatch& C = p[qc];
      int e0 = C.n[0] + 2, e1 = C.n[1] + 2;
      int z = dim == 3 ? c - C.lo[2] + 1 : 0;
      return ((size_t)z * e1 + (b - C.lo[1] + 1)) * e0 + (a - C.lo[0] + 1);
    };
    for (int qc : level_patches[lc]) {
      const HPatch& C = p[qc];
      std::vector<Cov>& cm = covmaps[qc];
      cm.assign((size_t)(C.n[0] + 2) * (C.n[1] + 2) * (dim == 3 ? C.n[2] + 2 : 1), Cov());
      std::vector<Nbr> src = nbr[qc];
      src.push_back({qc, {0, 0, 0}});
      for (const Nbr& x : src)
        for (int f : children[x.q]) {
          int a0[3], a1[3];
          for (int e = 0; e < 3; ++e) {
            if (e >= dim) { a0[e] = 0; a1[e] = 1; continue; }
            a0[e] = std::max(C.lo[e] - 1, p[f].lo[e] / 2 + x.s[e] * N(lc, e));
            a1[e] = std::min(C.hi[e] + 1, p[f].hi[e] / 2 + x.s[e] * N(lc, e));
          }
          for (int c = a0[2]; c < a1[2]; ++c)
            for (int b = a0[1]; b < a1[1]; ++b)
              for (int a = a0[0]; a < a1[0]; ++a) {
                Cov& v = cm[covidx(qc, a, b, c)];
                v.c = f;
                v.s[0] = x.s[0]; v.s[1] = x.s[1]; v.s[2] = x.s[2];
              }
        }
    }
    auto cov_at = [&](int qc, const int* g) -> const Cov& { return covmaps[qc][covidx(qc, g[0], g[1], g[2])]; };
    auto fine_loc = [&](const Cov& v, const int* gc, int add_d, int add) {
      // fine position 2*(gc - s*N) (+add along add_d) in patch v.c's frame
      int f[3];
      for (int e = 0; e < 3; ++e) f[e] = e < dim ? 2 * (gc[e] - v.s[e] * N(lc, e)) : 0;
      if (add_d >= 0) f[add_d] += add;
      return loc(v.c, f[0], f[1], f[2]);
    };
    // per coarse patch: candidate owners of its C/F edges (merged below)
    std::vector<std::vector<std::pair<Key, std::array<int, 4>>>> edge_cand(np);
    const std::vector<int>& lpc = level_patches[lc];
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t ip = 0; ip < lpc.size(); ++ip) {
      const int qc = lpc[ip];
      const HPatch& C = p[qc];
      const int k0 = dim == 3 ? C.lo[2] : 0, k1 = dim == 3 ? C.hi[2] : 1;
      // C/F faces and restricted cells
      for (int d = 0; d < dim; ++d)
        for (int k = k0; k < k1; ++k)
          for (int j = C.lo[1]; j < C.hi[1]; ++j)
            for (int i = C.lo[0]; i < C.hi[0]; ++i) {
              int g[3] = {i, j, k};
              if (cov_at(qc, g).c >= 0) continue;
              int gm[3] = {i, j, k}, gp[3] = {i, j, k};
              gm[d] -= 1;
              gp[d] += 1;
              const Cov& vm = cov_at(qc, gm);
              if (vm.c >= 0) face_rows[qc].push_back({l, qc, d, loc(qc, i, j, k), 1, vm.c, fine_loc(vm, gm, d, 2)});
              const Cov& vp = cov_at(qc, gp);
              if (vp.c >= 0) {
                int gf[3] = {i, j, k};
                gf[d] += 1;
                face_rows[qc].push_back({l, qc, d, loc(qc, gf[0], gf[1], gf[2]), -1, vp.c, fine_loc(vp, gp, -1, 0)});
              }
            }
      for (int k = k0; k < k1; ++k)
        for (int j = C.lo[1]; j < C.hi[1]; ++j)
          for (int i = C.lo[0]; i < C.hi[0]; ++i) {
            int g[3] = {i, j, k};
            const Cov& v = cov_at(qc, g);
            if (v.c >= 0) rcell_rows[qc].push_back({l, qc, loc(qc, i, j, k), v.c, fine_loc(v, g, -1, 0)});
          }
      // faces in the closure: restriction (>= 1 covered side)
      for (int d = 0; d < dim; ++d)
        for (int k = k0; k < k1 + (d == 2 ? 1 : 0); ++k)
          for (int j = C.lo[1]; j < C.hi[1] + (d == 1 ? 1 : 0); ++j)
            for (int i = C.lo[0]; i < C.hi[0] + (d == 0 ? 1 : 0); ++i) {
              int g[3] = {i, j, k}, gm[3] = {i, j, k};
              gm[d] -= 1;
              const Cov& v1 = cov_at(qc, gm);
              const Cov& v2 = cov_at(qc, g);
              if (v1.c < 0 && v2.c < 0) continue;
              int bf = -1, bl = 0;
              if (v1.c >= 0) { bf = v1.c; bl = fine_loc(v1, gm, d, 2); }
              if (v2.c >= 0) {
                int L2 = fine_loc(v2, g, -1, 0);
                if (bf < 0 || v2.c < bf || (v2.c == bf && L2 < bl)) { bf = v2.c; bl = L2; }
              }
              rface_rows[qc].push_back({l, qc, d, loc(qc, i, j, k), bf, bl});
            }
      // C/F edges in the closure
      for (int c = 0; c < 3; ++c) {
        if (dim == 2 && c != 2) continue;
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        int lo[3], hi[3];
        for (int e = 0; e < 3; ++e) {
          if (e >= dim) { lo[e] = 0; hi[e] = 1; continue; }
          lo[e] = C.lo[e];
          hi[e] = C.hi[e] + (e == c ? 0 : 1);
        }
        for (int k = lo[2]; k < hi[2]; ++k)
          for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
              int E[3] = {i, j, k};
              int ncov = 0, bf = -1, bl = 0;
              for (int sb = -1; sb <= 0; ++sb)
                for (int sa = -1; sa <= 0; ++sa) {
                  int g[3] = {i, j, k};
                  g[a] += sa;
                  g[b] += sb;
                  const Cov& v = cov_at(qc, g);
                  if (v.c < 0) continue;
                  ++ncov;
                  int f[3];
                  for (int e = 0; e < 3; ++e) f[e] = e < dim ? 2 * (E[e] - v.s[e] * N(lc, e)) : 0;
                  int Lf = loc(v.c, f[0], f[1], f[2]);
                  if (bf < 0 || v.c < bf || (v.c == bf && Lf < bl)) { bf = v.c; bl = Lf; }
                }
              if (ncov < 1 || ncov > 3) continue;
              Key key{c, wrapd(lc, 0, i), wrapd(lc, 1, j), dim == 3 ? wrapd(lc, 2, k) : 0};
              edge_cand[qc].push_back({key, {qc, loc(qc, i, j, k), bf, bl}});
            }
      }
    }
    // the smallest (coarse patch, local index) and (fine patch, local index) per edge
    for (int qc : lpc)
      for (const auto& kc : edge_cand[qc]) {
        const Key& key = kc.first;
        const int Le = kc.second[1], bf = kc.second[2], bl = kc.second[3];
        auto it = edge_best.find(key);
        if (it == edge_best.end()) edge_best[key] = kc.second;
        else {
          auto& v = it->second;
          if (qc < v[0] || (qc == v[0] && Le < v[1])) { v[0] = qc; v[1] = Le; }
          if (bf < v[2] || (bf == v[2] && bl < v[3])) { v[2] = bf; v[3] = bl; }
        }
      }
    // emit C/F faces (qc ascending, then (d, Lface)), reflux cells, restriction lists
    std::vector<std::array<int, 9>> rrows;
    std::unordered_map<std::pair<int, int>, size_t, PairHash> rrow_of;  // (qc, Lcell) -> index in rrows
    for (int qc : level_patches[lc]) {
      auto& v = face_rows[qc];
      std::sort(v.begin(), v.end());
      for (auto& r : v) {
        int64_t row = (int64_t)cf_faces.size() / 7;
        cf_faces.insert(cf_faces.end(), r.begin(), r.end());
        // the uncovered cell this face belongs to, and the face's slot in it
        int d = r[2], Lf = r[3], side = r[4];
        int sd = 1;
        for (int e = 0; e < d; ++e) sd *= p[qc].ext[e];
        int Lcell = side == 1 ? Lf : Lf - sd;
        int slot = 2 * d + (side == 1 ? 0 : 1);
        auto it = rrow_of.find({qc, Lcell});
        if (it == rrow_of.end()) {
          std::array<int, 9> rr = {l, qc, Lcell, -1, -1, -1, -1, -1, -1};
          rr[3 + slot] = (int)row;
          rrow_of[{qc, Lcell}] = rrows.size();
          rrows.push_back(rr);
        } else {
          rrows[it->second][3 + slot] = (int)row;
        }
      }
    }
    std::sort(rrows.begin(), rrows.end());
    for (auto& r : rrows) reflux_cells.insert(reflux_cells.end(), r.begin(), r.end());
    for (int qc : level_patches[lc]) {
      for (auto& r : rcell_rows[qc]) restrict_cells.insert(restrict_cells.end(), r.begin(), r.end());
    }
    {
      std::vector<std::array<int, 6>> all;
      for (int qc : level_patches[lc]) all.insert(all.end(), rface_rows[qc].begin(), rface_rows[qc].end());
      std::sort(all.begin(), all.end());
      for (auto& r : all) restrict_faces.insert(restrict_faces.end(), r.begin(), r.end());
    }
    // C/F edges sorted by (qc, c, Le); remember their row numbers by key
    std::vector<std::pair<std::array<int, 6>, Key>> erows;
    for (auto& kv : edge_best) erows.push_back({{l, kv.second[0], kv.first.c, kv.second[1], kv.second[2], kv.second[3]}, kv.first});
    std::sort(erows.begin(), erows.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    std::unordered_map<Key, int, KeyHash> edge_row;
    for (auto& e : erows) {
      edge_row[e.second] = (int)(cf_edges.size() / 6);
      cf_edges.insert(cf_edges.end(), e.first.begin(), e.first.end());
    }
    // EMF-corrected faces: every stored copy of an uncovered face touching a C/F edge
    {
      std::vector<std::vector<std::array<int, 8>>> per(np);
#pragma omp parallel for schedule(dynamic, 1)
      for (size_t ip = 0; ip < lpc.size(); ++ip) {
        const int qc = lpc[ip];
        const HPatch& C = p[qc];
        const int k0 = dim == 3 ? C.lo[2] : 0, k1 = dim == 3 ? C.hi[2] : 1;
        // cells within one cell of a covered cell: only faces touching one can
        // touch a C/F edge
        const int e0 = C.n[0] + 2, e1 = C.n[1] + 2, e2 = dim == 3 ? C.n[2] + 2 : 1;
        std::vector<char> near((size_t)e0 * e1 * e2, 0);
        for (int z = 0; z < e2; ++z)
          for (int y = 0; y < e1; ++y)
            for (int x = 0; x < e0; ++x) {
              if (covmaps[qc][((size_t)z * e1 + y) * e0 + x].c < 0) continue;
              for (int cz = (dim == 3 ? z - 1 : 0); cz <= (dim == 3 ? z + 1 : 0); ++cz)
                for (int cy = y - 1; cy <= y + 1; ++cy)
                  for (int cx = x - 1; cx <= x + 1; ++cx)
                    if (cz >= 0 && cz < e2 && cy >= 0 && cy < e1 && cx >= 0 && cx < e0)
                      near[((size_t)cz * e1 + cy) * e0 + cx] = 1;
            }
        auto near_at = [&](const int* g) {
          const int z = dim == 3 ? g[2] - C.lo[2] + 1 : 0;
          return near[((size_t)z * e1 + (g[1] - C.lo[1] + 1)) * e0 + (g[0] - C.lo[0] + 1)] != 0;
        };
        std::vector<std::array<int, 8>>& all = per[qc];
        for (int d = 0; d < dim; ++d) {
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          for (int k = k0; k < k1 + (d == 2 ? 1 : 0); ++k)
            for (int j = C.lo[1]; j < C.hi[1] + (d == 1 ? 1 : 0); ++j)
              for (int i = C.lo[0]; i < C.hi[0] + (d == 0 ? 1 : 0); ++i) {
                int g[3] = {i, j, k}, gm[3] = {i, j, k};
                gm[d] -= 1;
                if (!near_at(g) && !near_at(gm)) continue;
                if (cov_at(qc, g).c >= 0 || cov_at(qc, gm).c >= 0) continue;
                int e[4] = {-1, -1, -1, -1};
                bool any = false;
                for (int slot = 0; slot < 4; ++slot) {
                  int comp = slot < 2 ? t2 : t1;
                  if (dim == 2 && comp != 2) continue;
                  int gs[3] = {i, j, k};
                  gs[slot < 2 ? t1 : t2] += slot & 1;
                  Key key{comp, wrapd(lc, 0, gs[0]), wrapd(lc, 1, gs[1]), dim == 3 ? wrapd(lc, 2, gs[2]) : 0};
                  auto it = edge_row.find(key);
                  if (it != edge_row.end()) { e[slot] = it->second; any = true; }
                }
                if (!any) continue;
                all.push_back({l, qc, d, loc(qc, i, j, k), e[0], e[1], e[2], e[3]});
              }
        }
      }
      std::vector<std::array<int, 8>> all;
      for (int qc : lpc) all.insert(all.end(), per[qc].begin(), per[qc].end());
      std::sort(all.begin(), all.end());
      for (auto& r : all) emf_faces.insert(emf_faces.end(), r.begin(), r.end());
    }
    rng_cf_faces[l][1] = (int64_t)cf_faces.size() / 7;
    rng_cf_edges[l][1] = (int64_t)cf_edges.size() / 6;
    rng_emf_faces[l][1] = (int64_t)emf_faces.size() / 8;
    rng_restrict_cells[l][1] = (int64_t)restrict_cells.size() / 5;
    rng_restrict_faces[l][1] = (int64_t)restrict_faces.size() / 6;
    rng_reflux_cells[l][1] = (int64_t)reflux_cells.size() / 9;
  }
  return AMRMHD_OK;
}

}  // namespace amrmhd
