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

#include <parallel/algorithm>

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

// sort in parallel (OpenMP) above a size where it pays
template <class It, class Cmp> void psort(It a, It b, Cmp cmp) {
  if (b - a > (1 << 16)) __gnu_parallel::sort(a, b, cmp);
  else std::sort(a, b, cmp);
}

}  // namespace

int Hierarchy::build(const int32_t* rows7, int n) {
  err.clear();
  p.clear();
  ghost_cells.clear(); ghost_faces.clear(); ghost_box_cells.clear(); ghost_box_faces.clear();
  ghost_rows_ready = false;
  cf_faces.clear(); cf_edges.clear();
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

  // ---------------- ghost fill boxes (patches in parallel, concatenated in patch order)
  // Every ghost position of a patch (cells: the ghosted box minus the interior;
  // d-faces: the face box minus the patch's own faces) gets a label: kind 0 a
  // copy from a same-level patch at a constant local offset, kind 1 a
  // prolongation from the coarse patch holding the parent cell (with the
  // periodic wrap of the fine position), kind 2 a copy of the patch's own
  // position clamped into the domain, kind 3 the inflow state. Positions with
  // equal labels are merged greedily into boxes (x runs, then y, then z), so
  // the work per position is a label and a comparison, and the device lists
  // hold boxes, not positions.
  ghost_rows_ready = false;
  std::vector<std::vector<int32_t>> gbc(np), gbf(np);
  std::vector<std::string> gerr(np);
  std::vector<int> gst(np, 0);
  struct Lab {
    int kind, src, aux[3];
    bool operator==(const Lab& o) const {
      return kind == o.kind && src == o.src && aux[0] == o.aux[0] && aux[1] == o.aux[1] && aux[2] == o.aux[2];
    }
  };
  auto ghost_patch = [&](int q, std::vector<int32_t>& outc, std::vector<int32_t>& outf, std::string& errq) -> int {
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
    // labels are few per patch: positions hold an index into a small table
    std::vector<Lab> labs;
    int last_id = -1;
    auto label_id = [&](const Lab& k) {
      if (last_id >= 0 && labs[last_id] == k) return last_id;
      for (size_t i = 0; i < labs.size(); ++i)
        if (labs[i] == k) return last_id = (int)i;
      labs.push_back(k);
      return last_id = (int)labs.size() - 1;
    };
    static thread_local std::vector<int> lid, sl;
    static thread_local std::vector<uint8_t> state;  // 0 not a ghost, 1 to assign, 2 assigned
    for (int d = -1; d < dim; ++d) {  // -1: cells, else the d-faces
      int ex[3], g0[3], own0[3], own1[3];
      for (int e = 0; e < 3; ++e) {
        ex[e] = e < dim ? P.n[e] + 8 + (e == d ? 1 : 0) : 1;
        g0[e] = e < dim ? P.lo[e] - 4 : 0;  // global position of local coordinate 0
        // the patch's own cells (faces) in local coordinates
        own0[e] = e < dim ? 4 : 0;
        own1[e] = e < dim ? P.n[e] + 4 + (e == d ? 1 : 0) : 1;
      }
      const size_t tot = (size_t)ex[0] * ex[1] * ex[2];
      lid.assign(tot, -1);
      sl.resize(tot);
      state.assign(tot, 0);
      labs.clear();
      last_id = -1;
      auto at = [&](int a, int b, int c) { return ((size_t)c * ex[1] + b) * ex[0] + a; };
      // the ghost positions of row (b, c): all of it, or the two ends when the
      // row passes through the patch's own positions
      auto for_ghosts = [&](auto&& f) {
        for (int c = 0; c < ex[2]; ++c)
          for (int b = 0; b < ex[1]; ++b) {
            const bool through = b >= own0[1] && b < own1[1] && c >= own0[2] && c < own1[2];
            if (!through) {
              for (int a = 0; a < ex[0]; ++a) f(a, b, c);
            } else {
              for (int a = 0; a < own0[0]; ++a) f(a, b, c);
              for (int a = own1[0]; a < ex[0]; ++a) f(a, b, c);
            }
          }
      };
      // same-level sources: the neighbour (with its periodic shift) whose
      // interior (or own faces) holds the position; on a face stored by two
      // neighbours the smaller (patch, local index) wins
      for (const Nbr& x : nbr[q]) {
        const HPatch& Q = p[x.q];
        int a0[3], a1[3], delta[3] = {0, 0, 0};
        bool empty = false;
        for (int e = 0; e < 3; ++e) {
          if (e >= dim) { a0[e] = 0; a1[e] = 1; continue; }
          const int qlo = Q.lo[e] + x.s[e] * N(l, e), qhi = Q.hi[e] + x.s[e] * N(l, e) + (e == d ? 1 : 0);
          a0[e] = std::max(0, qlo - g0[e]);
          a1[e] = std::min(ex[e], qhi - g0[e]);
          if (a1[e] <= a0[e]) empty = true;
          delta[e] = P.lo[e] - Q.lo[e] - x.s[e] * N(l, e);
        }
        if (empty) continue;
        const int id = label_id(Lab{0, x.q, {delta[0], delta[1], delta[2]}});
        for (int c = a0[2]; c < a1[2]; ++c)
          for (int b = a0[1]; b < a1[1]; ++b)
            for (int a = a0[0]; a < a1[0]; ++a) {
              const size_t t = at(a, b, c);
              const int L = (a + delta[0]) + Q.ext[0] * ((b + delta[1]) + Q.ext[1] * (c + delta[2]));
              const int cur = lid[t];
              if (d < 0 || cur < 0 || x.q < labs[cur].src || (x.q == labs[cur].src && L < sl[t])) {
                lid[t] = id;
                sl[t] = L;
              }
            }
      }
      // prolongation: each coarse candidate, at each periodic image w, is the
      // source of the positions whose wrapped parent cell (g + w N) >> 1 it
      // holds; along a non-periodic d the face at the domain's top belongs to
      // the coarse patch holding the last cell
      if (l > 0) {
        for (int Cq : cc) {
          const HPatch& Cp = p[Cq];
          int wlo[3], whi[3];
          for (int e = 0; e < 3; ++e) {
            wlo[e] = (e < dim && per[e]) ? -1 : 0;
            whi[e] = (e < dim && per[e]) ? 1 : 0;
          }
          for (int wz = wlo[2]; wz <= whi[2]; ++wz)
            for (int wy = wlo[1]; wy <= whi[1]; ++wy)
              for (int wx = wlo[0]; wx <= whi[0]; ++wx) {
                const int w[3] = {wx, wy, wz};
                int a0[3], a1[3], aux[3] = {0, 0, 0};
                bool empty = false;
                for (int e = 0; e < 3; ++e) {
                  if (e >= dim) { a0[e] = 0; a1[e] = 1; continue; }
                  aux[e] = w[e] * N(l, e);
                  const int top = (e == d && !per[e] && Cp.hi[e] == N(l - 1, e)) ? 1 : 0;
                  a0[e] = std::max(0, 2 * Cp.lo[e] - aux[e] - g0[e]);
                  a1[e] = std::min(ex[e], 2 * Cp.hi[e] + top - aux[e] - g0[e]);
                  if (a1[e] <= a0[e]) empty = true;
                }
                if (empty) continue;
                const int id = label_id(Lab{1, Cq, {aux[0], aux[1], aux[2]}});
                for (int c = a0[2]; c < a1[2]; ++c)
                  for (int b = a0[1]; b < a1[1]; ++b)
                    for (int a = a0[0]; a < a1[0]; ++a) {
                      const size_t t = at(a, b, c);
                      if (lid[t] < 0) lid[t] = id;
                    }
              }
        }
      }
      // physical boundaries (outside the domain of a non-periodic dimension),
      // then a check that every ghost position has a source
      bool touches = false;
      for (int e = 0; e < dim; ++e)
        if (!per[e] && (g0[e] < 0 || g0[e] + ex[e] - 1 > (e == d ? N(l, e) : N(l, e) - 1))) touches = true;
      int fail = 0;
      for_ghosts([&](int a, int b, int c) {
        if (fail) return;
        const size_t t = at(a, b, c);
        state[t] = 1;
        const int g[3] = {g0[0] + a, g0[1] + b, g0[2] + c};
        if (touches) {
          Lab bl{2, q, {-1, -1, -1}};
          bool out = false, inflow = false;
          for (int e = 0; e < dim; ++e) {
            if (per[e]) continue;
            const int top = e == d ? N(l, e) : N(l, e) - 1;
            if (g[e] < 0) { out = true; bl.aux[e] = 0; inflow |= bc[e][0] == 2; }
            else if (g[e] > top) { out = true; bl.aux[e] = top; inflow |= bc[e][1] == 2; }
          }
          if (out) {
            lid[t] = label_id(inflow ? Lab{3, -1, {0, 0, 0}} : bl);
            return;
          }
        }
        if (lid[t] >= 0) return;
        if (l == 0) {
          errq = d < 0 ? "level-0 ghost cell without a source" : "level-0 ghost face without a source";
          fail = AMRMHD_EINVAL;
          return;
        }
        errq = d < 0 ? "no parent-level source for the ghost cell (" + std::to_string(g[0]) + ", " +
                           std::to_string(g[1]) + ", " + std::to_string(g[2]) + ") of patch " + std::to_string(q)
                     : "no parent-level source for the ghost face (" + std::to_string(d) + "; " +
                           std::to_string(g[0]) + ", " + std::to_string(g[1]) + ", " + std::to_string(g[2]) +
                           ") of patch " + std::to_string(q);
        fail = AMRMHD_ENEST;
      });
      if (fail) return fail;
      // greedy boxes of equal labels
      std::vector<int32_t>& out = d < 0 ? outc : outf;
      for_ghosts([&](int a, int b, int c) {
        const size_t t0 = at(a, b, c);
        if (state[t0] != 1) return;
        const int k = lid[t0];
        auto same = [&](int x, int y, int z) {
          const size_t t = at(x, y, z);
          return state[t] == 1 && lid[t] == k;
        };
        int nx = 1, ny = 1, nz = 1;
        while (a + nx < ex[0] && same(a + nx, b, c)) ++nx;
        auto row_ok = [&](int y, int z) {
          for (int i = 0; i < nx; ++i)
            if (!same(a + i, y, z)) return false;
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
            for (int x = 0; x < nx; ++x) state[at(a + x, b + y, c + z)] = 2;
        const Lab& kk = labs[k];
        const int32_t row[GHOST_BOX_W] = {q, d, kk.kind, kk.src, a, b, c, nx, ny, nz, kk.aux[0], kk.aux[1], kk.aux[2]};
        out.insert(out.end(), row, row + GHOST_BOX_W);
      });
    }
    return 0;
  };
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < np; ++q)
    if (p[q].level >= ghost_from && !ghost_elsewhere) gst[q] = ghost_patch(q, gbc[q], gbf[q], gerr[q]);
  for (int q = 0; q < np; ++q)
    if (gst[q]) { err = gerr[q]; return gst[q]; }
  {
    size_t nc = 0, nf = 0;
    for (int q = 0; q < np; ++q) { nc += gbc[q].size(); nf += gbf[q].size(); }
    ghost_box_cells.clear();
    ghost_box_faces.clear();
    ghost_box_cells.reserve(nc);
    ghost_box_faces.reserve(nf);
    for (int q = 0; q < np; ++q) {
      ghost_box_cells.insert(ghost_box_cells.end(), gbc[q].begin(), gbc[q].end());
      ghost_box_faces.insert(ghost_box_faces.end(), gbf[q].begin(), gbf[q].end());
    }
  }

  // ---------------- register, reflux and restriction maps, per fine level
  rng_cf_faces.assign(nlev, {0, 0});
  rng_cf_edges.assign(nlev, {0, 0});
  rng_emf_faces.assign(nlev, {0, 0});
  rng_restrict_cells.assign(nlev, {0, 0});
  rng_restrict_faces.assign(nlev, {0, 0});
  rng_reflux_cells.assign(nlev, {0, 0});
  for (int l = 1; l < nlev && with_registers; ++l) {
    const int lc = l - 1;
    rng_cf_faces[l][0] = (int64_t)cf_faces.size() / 7;
    rng_cf_edges[l][0] = (int64_t)cf_edges.size() / 6;
    rng_emf_faces[l][0] = (int64_t)emf_faces.size() / 8;
    rng_restrict_cells[l][0] = (int64_t)restrict_cells.size() / 5;
    rng_restrict_faces[l][0] = (int64_t)restrict_faces.size() / 6;
    rng_reflux_cells[l][0] = (int64_t)reflux_cells.size() / 9;
    // per coarse patch: cover map over its cells widened by one, entry (fine patch, shift)
    struct Cov { int c = -1; int s[3] = {0, 0, 0}; };
    std::vector<std::vector<std::array<int, 7>>> face_rows(np);
    std::vector<std::vector<std::array<int, 5>>> rcell_rows(np);
    std::vector<std::vector<std::array<int, 6>>> rface_rows(np);
    std::vector<std::vector<Cov>> covmaps(np);
    const std::vector<int>& lpc = level_patches[lc];
    const int npc = (int)lpc.size();
    auto covidx = [&](int qc, int a, int b, int c) {
      const HPatch& C = p[qc];
      int e0 = C.n[0] + 2, e1 = C.n[1] + 2;
      int z = dim == 3 ? c - C.lo[2] + 1 : 0;
      return ((size_t)z * e1 + (b - C.lo[1] + 1)) * e0 + (a - C.lo[0] + 1);
    };
#pragma omp parallel for schedule(dynamic, 1)
    for (int ip = 0; ip < npc; ++ip) {
      const int qc = lpc[ip];
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
    // per coarse patch: C/F faces (sorted by (d, Lface)), restricted cells and
    // faces (generated in (d,) local index order), candidate owners of its C/F
    // edges (merged below)
    struct ECand { Key key; int qc, Le, bf, bl; };
    std::vector<std::vector<ECand>> edge_cand(np);
#pragma omp parallel for schedule(dynamic, 1)
    for (int ip = 0; ip < npc; ++ip) {
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
              edge_cand[qc].push_back({key, qc, loc(qc, i, j, k), bf, bl});
            }
      }
      std::sort(face_rows[qc].begin(), face_rows[qc].end());
    }
    // row offsets of each coarse patch's rows in the level's lists
    std::vector<size_t> o_face(npc + 1, 0), o_rcell(npc + 1, 0), o_rface(npc + 1, 0), o_ecand(npc + 1, 0);
    for (int ip = 0; ip < npc; ++ip) {
      const int qc = lpc[ip];
      o_face[ip + 1] = o_face[ip] + face_rows[qc].size();
      o_rcell[ip + 1] = o_rcell[ip] + rcell_rows[qc].size();
      o_rface[ip + 1] = o_rface[ip] + rface_rows[qc].size();
      o_ecand[ip + 1] = o_ecand[ip] + edge_cand[qc].size();
    }
    // C/F edges: the candidates sorted by edge; per edge the smallest (coarse
    // patch, local index) and (fine patch, local index)
    std::vector<ECand> ec(o_ecand[npc]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int ip = 0; ip < npc; ++ip)
      std::copy(edge_cand[lpc[ip]].begin(), edge_cand[lpc[ip]].end(), ec.begin() + o_ecand[ip]);
    std::vector<std::vector<ECand>>().swap(edge_cand);
    psort(ec.begin(), ec.end(), [](const ECand& x, const ECand& y) { return x.key < y.key; });
    std::vector<std::pair<std::array<int, 6>, Key>> erows;
    for (size_t i = 0; i < ec.size();) {
      size_t j = i;
      std::array<int, 4> v = {ec[i].qc, ec[i].Le, ec[i].bf, ec[i].bl};
      for (; j < ec.size() && ec[j].key == ec[i].key; ++j) {
        const ECand& x = ec[j];
        if (x.qc < v[0] || (x.qc == v[0] && x.Le < v[1])) { v[0] = x.qc; v[1] = x.Le; }
        if (x.bf < v[2] || (x.bf == v[2] && x.bl < v[3])) { v[2] = x.bf; v[3] = x.bl; }
      }
      erows.push_back({{l, v[0], ec[i].key.c, v[1], v[2], v[3]}, ec[i].key});
      i = j;
    }
    std::vector<ECand>().swap(ec);
    // C/F edges sorted by (qc, c, Le); their row numbers by key (sorted for lookup)
    psort(erows.begin(), erows.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    const int64_t erow0 = (int64_t)cf_edges.size() / 6;
    std::vector<std::pair<Key, int>> edge_row((size_t)erows.size());
    cf_edges.resize(cf_edges.size() + 6 * erows.size());
#pragma omp parallel for
    for (int64_t i = 0; i < (int64_t)erows.size(); ++i) {
      std::copy(erows[i].first.begin(), erows[i].first.end(), cf_edges.begin() + 6 * (erow0 + i));
      edge_row[i] = {erows[i].second, (int)(erow0 + i)};
    }
    std::vector<std::pair<std::array<int, 6>, Key>>().swap(erows);
    psort(edge_row.begin(), edge_row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    auto edge_row_of = [&](const Key& k) {
      auto it = std::lower_bound(edge_row.begin(), edge_row.end(), k,
                                 [](const std::pair<Key, int>& x, const Key& y) { return x.first < y; });
      return (it != edge_row.end() && it->first == k) ? it->second : -1;
    };
    // emit C/F faces (qc ascending, then (d, Lface)), reflux cells (per
    // uncovered cell with a C/F face: the rows of its faces by slot), restriction lists
    const int64_t frow0 = (int64_t)cf_faces.size() / 7;
    cf_faces.resize(cf_faces.size() + 7 * o_face[npc]);
    const size_t rc0 = restrict_cells.size(), rf0 = restrict_faces.size();
    restrict_cells.resize(rc0 + 5 * o_rcell[npc]);
    restrict_faces.resize(rf0 + 6 * o_rface[npc]);
    std::vector<std::vector<std::array<int, 9>>> rrows(npc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int ip = 0; ip < npc; ++ip) {
      const int qc = lpc[ip];
      const auto& v = face_rows[qc];
      std::vector<std::array<int, 3>> cells;  // (Lcell, slot, row)
      cells.reserve(v.size());
      for (size_t k = 0; k < v.size(); ++k) {
        const auto& r = v[k];
        const int64_t row = frow0 + (int64_t)(o_face[ip] + k);
        std::copy(r.begin(), r.end(), cf_faces.begin() + 7 * row);
        // the uncovered cell this face belongs to, and the face's slot in it
        const int d = r[2], Lf = r[3], side = r[4];
        int sd = 1;
        for (int e = 0; e < d; ++e) sd *= p[qc].ext[e];
        cells.push_back({side == 1 ? Lf : Lf - sd, 2 * d + (side == 1 ? 0 : 1), (int)row});
      }
      std::sort(cells.begin(), cells.end());
      for (size_t k = 0; k < cells.size();) {
        std::array<int, 9> rr = {l, qc, cells[k][0], -1, -1, -1, -1, -1, -1};
        size_t m = k;
        for (; m < cells.size() && cells[m][0] == cells[k][0]; ++m) rr[3 + cells[m][1]] = cells[m][2];
        rrows[ip].push_back(rr);
        k = m;
      }
      size_t o = rc0 + 5 * o_rcell[ip];
      for (const auto& r : rcell_rows[qc]) {
        std::copy(r.begin(), r.end(), restrict_cells.begin() + o);
        o += 5;
      }
      o = rf0 + 6 * o_rface[ip];
      for (const auto& r : rface_rows[qc]) {
        std::copy(r.begin(), r.end(), restrict_faces.begin() + o);
        o += 6;
      }
    }
    for (int ip = 0; ip < npc; ++ip)
      for (const auto& r : rrows[ip]) reflux_cells.insert(reflux_cells.end(), r.begin(), r.end());
    // EMF-corrected faces: every stored copy of an uncovered face touching a C/F
    // edge, generated per coarse patch in (d, local index) order
    {
      std::vector<std::vector<std::array<int, 8>>> per(np);
#pragma omp parallel for schedule(dynamic, 1)
      for (int ip = 0; ip < npc; ++ip) {
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
                  const int row = edge_row_of(key);
                  if (row >= 0) { e[slot] = row; any = true; }
                }
                if (!any) continue;
                all.push_back({l, qc, d, loc(qc, i, j, k), e[0], e[1], e[2], e[3]});
              }
        }
      }
      for (int qc : lpc)
        for (const auto& r : per[qc]) emf_faces.insert(emf_faces.end(), r.begin(), r.end());
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

void Hierarchy::expand_ghost_rows() {
  if (ghost_rows_ready) return;
  const int np = (int)p.size();
  // positions of every box, per patch, sorted into the row order (patch; cells
  // by local index; faces by direction, then local index)
  std::vector<std::vector<std::array<int64_t, 2>>> keyc(np), keyf(np);  // (sort key, row start)
  std::vector<int32_t> rc, rf;
  auto emit = [&](const std::vector<int32_t>& boxes, bool faces) {
    for (size_t r = 0; r < boxes.size(); r += GHOST_BOX_W) {
      const int32_t* b = &boxes[r];
      const int q = b[0], d = b[1], kind = b[2], src = b[3];
      const HPatch& P = p[q];
      for (int z = b[6]; z < b[6] + b[9]; ++z)
        for (int y = b[5]; y < b[5] + b[8]; ++y)
          for (int x = b[4]; x < b[4] + b[7]; ++x) {
            const int Ld = x + P.ext[0] * (y + P.ext[1] * z);
            const int g[3] = {P.lo[0] + x - 4, P.lo[1] + y - 4, dim == 3 ? P.lo[2] + z - 4 : 0};
            int Ls = -1;
            if (kind == 0) {
              const HPatch& S = p[src];
              Ls = (x + b[10]) + S.ext[0] * ((y + b[11]) + S.ext[1] * (z + b[12]));
            } else if (kind == 1) {
              int c[3];
              for (int e = 0; e < 3; ++e) c[e] = e < dim ? (g[e] + b[10 + e]) >> 1 : 0;
              Ls = loc(src, c[0], c[1], c[2]);
            } else if (kind == 2) {
              int gc[3];
              for (int e = 0; e < 3; ++e) gc[e] = b[10 + e] >= 0 ? b[10 + e] : g[e];
              Ls = loc(q, gc[0], gc[1], gc[2]);
            }
            std::vector<int32_t>& v = faces ? rf : rc;
            if (faces) {
              keyf[q].push_back({(int64_t)d << 40 | Ld, (int64_t)v.size()});
              const int32_t row[6] = {q, d, Ld, kind, src, Ls};
              v.insert(v.end(), row, row + 6);
            } else {
              keyc[q].push_back({(int64_t)Ld, (int64_t)v.size()});
              const int32_t row[5] = {q, Ld, kind, src, Ls};
              v.insert(v.end(), row, row + 5);
            }
          }
    }
  };
  emit(ghost_box_cells, false);
  emit(ghost_box_faces, true);
  ghost_cells.clear();
  ghost_faces.clear();
  ghost_cells.reserve(rc.size());
  ghost_faces.reserve(rf.size());
  for (int q = 0; q < np; ++q) {
    std::sort(keyc[q].begin(), keyc[q].end());
    for (const auto& k : keyc[q]) ghost_cells.insert(ghost_cells.end(), rc.begin() + k[1], rc.begin() + k[1] + 5);
    std::sort(keyf[q].begin(), keyf[q].end());
    for (const auto& k : keyf[q]) ghost_faces.insert(ghost_faces.end(), rf.begin() + k[1], rf.begin() + k[1] + 6);
  }
  ghost_rows_ready = true;
}

}  // namespace amrmhd
