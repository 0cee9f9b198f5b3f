// Register, reflux and restriction maps of a hierarchy built on the device
// (Sec. 4's synchronize step: the fine fluxes and EMFs on coarse-fine faces
// and edges that correct the coarse level, and the restriction of covered
// coarse data). The rows are those of the host builder (hierarchy.cpp), bit
// for bit and in the same order:
//
// * every coarse patch (levels 0 .. nlev-2, level by level, ascending ids)
//   owns three position ranges: its faces (per direction d, the face box
//   n + e_d in raster order), its cells, and its edges (per component c, the
//   closure box n + 1 - e_c);
// * a cover map per coarse patch (its cells widened by one) holds the fine
//   patch (and its periodic shift) over each coarse cell;
// * each position decides from the cover map alone whether it carries a row of
//   each list; a count pass per 1024-position chunk, a host prefix sum over the
//   chunks and an emit pass with a block-wide scan write the rows in position
//   order, which is the host builder's order (coarse patch, then direction or
//   component, then local index);
// * a coarse-fine edge shared by several coarse patches is listed once, by the
//   smallest (coarse patch, local index) holding it: each candidate finds that
//   owner among its patch and its same-level neighbours (with their shifts),
//   which are all the patches whose closure can hold the edge.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.hpp"

namespace amrdm {

constexpr int CHUNK = 1024;  // positions per block (256 threads x 4)
constexpr int NT = 256;

struct MPatch {
  int lo[3], n[3], ext[3], level;
};

struct MQc {        // a coarse patch
  int q;            // patch id
  int nb0, nb1;     // its neighbour entries [nb0, nb1) (itself at shift 0 first)
  long long cov;    // first entry of its cover map ((n + 2)^dim)
  long long fo, eo; // first entry of its face and edge positions in the row maps
};

struct MArgs {
  int dim;
  int base[3];
  const MPatch* P;
  const MQc* Q;
  const int* nbrs;        // (coarse patch index, shift code) pairs
  int* cov_c;             // fine patch over the cell, or -1
  signed char* cov_s;     // its shift code (sx + 1) + 3 (sy + 1) + 9 (sz + 1)
  const int* chunks;      // (coarse patch index, first position, count)
  int nchunks;
  long long* counts;      // per chunk and list
  const long long* first; // per chunk and list: the first row number
  int* face_row;          // per face position: its coarse-fine face row, or -1
  int* edge_row;          // per edge position: its coarse-fine edge row (owner only), or -1
  int* out[6];            // cf_faces, cf_edges, emf_faces, restrict_cells, restrict_faces, reflux_cells
};

enum { L_CF = 0, L_EDGE = 1, L_EMF = 2, L_RCELL = 3, L_RFACE = 4, L_REFLUX = 5 };

__host__ __device__ __forceinline__ int Nl(const MArgs& a, int l, int e) { return e < a.dim ? (a.base[e] << l) : 1; }

__host__ __device__ __forceinline__ int loc(const MArgs& a, int q, const int* g) {
  const MPatch& P = a.P[q];
  const int x = g[0] - P.lo[0] + 4, y = g[1] - P.lo[1] + 4, z = a.dim == 3 ? g[2] - P.lo[2] + 4 : 0;
  return x + P.ext[0] * (y + P.ext[1] * z);
}

struct Cov {
  int c, code;
};

// the cover entry of level-lc cell g (within one cell of the coarse patch)
__host__ __device__ __forceinline__ Cov cov(const MArgs& a, const MQc& Q, const MPatch& C, const int* g) {
  const int e0 = C.n[0] + 2, e1 = C.n[1] + 2;
  const int z = a.dim == 3 ? g[2] - C.lo[2] + 1 : 0;
  const long long i = Q.cov + ((long long)z * e1 + (g[1] - C.lo[1] + 1)) * e0 + (g[0] - C.lo[0] + 1);
  return Cov{a.cov_c[i], a.cov_s[i]};
}

__host__ __device__ __forceinline__ void shift_of(int code, int* s) {
  s[0] = code % 3 - 1;
  s[1] = (code / 3) % 3 - 1;
  s[2] = code / 9 - 1;
}

// local index, in fine patch v.c, of the fine position 2 (gc - s N) (+ add along add_d)
__host__ __device__ __forceinline__ int fine_loc(const MArgs& a, int lc, const Cov& v, const int* gc, int add_d, int add) {
  int s[3], f[3];
  shift_of(v.code, s);
  for (int e = 0; e < 3; ++e) f[e] = e < a.dim ? 2 * (gc[e] - s[e] * Nl(a, lc, e)) : 0;
  if (add_d >= 0) f[add_d] += add;
  return loc(a, v.c, f);
}

// the box of sub-range k of a coarse patch's face (space 0), cell (1) or edge (2) positions
__host__ __device__ __forceinline__ int nsub(int space, int dim) { return space == 1 ? 1 : (space == 0 ? dim : (dim == 3 ? 3 : 1)); }
__host__ __device__ __forceinline__ void sub_box(int space, int dim, int k, const int* n, int* b, int* dir) {
  int d = space == 2 ? (dim == 3 ? k : 2) : k;
  *dir = d;
  for (int e = 0; e < 3; ++e) {
    if (e >= dim) { b[e] = 1; continue; }
    if (space == 0) b[e] = n[e] + (e == d ? 1 : 0);
    else if (space == 1) b[e] = n[e];
    else b[e] = n[e] + (e == d ? 0 : 1);
  }
}

// position p of a coarse patch's space: the sub-range's direction and the global level position
__host__ __device__ __forceinline__ void decode(int space, int dim, const MPatch& C, long long p, int* dir, int* g, long long* sub0) {
  long long o = 0;
  int b[3];
  for (int k = 0;; ++k) {
    sub_box(space, dim, k, C.n, b, dir);
    const long long v = (long long)b[0] * b[1] * b[2];
    if (p < o + v || k + 1 == nsub(space, dim)) break;
    o += v;
  }
  *sub0 = o;
  const long long r = p - o;
  g[0] = C.lo[0] + (int)(r % b[0]);
  g[1] = C.lo[1] + (int)((r / b[0]) % b[1]);
  g[2] = (dim == 3 ? C.lo[2] : 0) + (int)(r / ((long long)b[0] * b[1]));
}

// edge of component c at level position E, seen from coarse patch index qi:
// the number of covered cells around it and the smallest (fine patch, local
// index) of the fine edge
__host__ __device__ void edge_cover(const MArgs& a, int qi, int c, const int* E, int* ncov, int* bf, int* bl) {
  const MQc& Q = a.Q[qi];
  const MPatch& C = a.P[Q.q];
  const int lc = C.level;
  const int ea = (c + 1) % 3, eb = (c + 2) % 3;
  *ncov = 0;
  *bf = -1;
  *bl = 0;
  for (int sb = -1; sb <= 0; ++sb)
    for (int sa = -1; sa <= 0; ++sa) {
      int g[3] = {E[0], E[1], E[2]};
      g[ea] += sa;
      g[eb] += sb;
      const Cov v = cov(a, Q, C, g);
      if (v.c < 0) continue;
      ++*ncov;
      const int Lf = fine_loc(a, lc, v, E, -1, 0);
      if (*bf < 0 || v.c < *bf || (v.c == *bf && Lf < *bl)) { *bf = v.c; *bl = Lf; }
    }
}

// the owner of the edge (c, E) of coarse patch index qi: the smallest (patch,
// local index) among the same-level patches whose closure holds it; returns
// the owner's coarse patch index, its local index and its edge position index
__host__ __device__ int edge_owner(const MArgs& a, int qi, int c, const int* E, int* Lmin, long long* pos) {
  const MQc& Q = a.Q[qi];
  const int lc = a.P[Q.q].level;
  int best = -1, bq = 0;
  *Lmin = 0;
  *pos = -1;
  for (int k = Q.nb0; k < Q.nb1; ++k) {
    const int oi = a.nbrs[2 * k];
    const MQc& O = a.Q[oi];
    const MPatch& P = a.P[O.q];
    int s[3], w[3];
    shift_of(a.nbrs[2 * k + 1], s);
    bool in = true;
    for (int e = 0; e < 3; ++e) {
      w[e] = e < a.dim ? E[e] - s[e] * Nl(a, lc, e) : 0;
      if (e < a.dim && (w[e] < P.lo[e] || w[e] > P.lo[e] + P.n[e] - (e == c ? 1 : 0))) in = false;
    }
    if (!in) continue;
    const int L = loc(a, O.q, w);
    if (best < 0 || O.q < bq || (O.q == bq && L < *Lmin)) {
      best = oi;
      bq = O.q;
      *Lmin = L;
      // position index of w in the owner's edge range
      int b[3], dir;
      long long o = 0;
      const int nk = a.dim == 3 ? 3 : 1;
      for (int k2 = 0; k2 < nk; ++k2) {
        sub_box(2, a.dim, k2, P.n, b, &dir);
        if (dir == c) break;
        o += (long long)b[0] * b[1] * b[2];
      }
      sub_box(2, a.dim, a.dim == 3 ? c : 0, P.n, b, &dir);
      const int z = a.dim == 3 ? w[2] - P.lo[2] : 0;
      *pos = O.eo + o + (w[0] - P.lo[0]) + (long long)b[0] * ((w[1] - P.lo[1]) + (long long)b[1] * z);
    }
  }
  return best;
}

// up to 3 lists per space: 0 faces (cf, restrict faces, emf), 1 cells
// (restrict cells, reflux), 2 edges (cf edges)
__host__ __device__ __forceinline__ int lists_of(int space, int k) {
  if (space == 0) return k == 0 ? L_CF : (k == 1 ? L_RFACE : L_EMF);
  if (space == 1) return k == 0 ? L_RCELL : L_REFLUX;
  return L_EDGE;
}
__host__ __device__ __forceinline__ int width(int list) {
  return list == L_CF ? 7 : list == L_EDGE ? 6 : list == L_EMF ? 8 : list == L_RCELL ? 5 : list == L_RFACE ? 6 : 9;
}
__host__ __device__ __forceinline__ int nlists(int space) { return space == 0 ? 3 : (space == 1 ? 2 : 1); }

// Evaluates position p of coarse patch qi for list k; with row != nullptr
// writes the row (and the row maps). Returns whether the position has a row.
template <int SPACE>
__host__ __device__ bool eval(const MArgs& a, int qi, long long p, int k, int* row, long long rown) {
  const MQc& Q = a.Q[qi];
  const MPatch& C = a.P[Q.q];
  const int lc = C.level, l = lc + 1, dim = a.dim;
  int d, g[3];
  long long sub0;
  decode(SPACE, dim, C, p, &d, g, &sub0);
  if (SPACE == 0) {  // the d-face at g: lower cell m = g - e_d, upper cell g
    int m[3] = {g[0], g[1], g[2]};
    m[d] -= 1;
    const Cov cu = cov(a, Q, C, g), cm = cov(a, Q, C, m);
    if (k == 0) {
      int side = 0, f = -1, fl = 0;
      if (g[d] < C.lo[d] + C.n[d] && cu.c < 0 && cm.c >= 0) {
        side = 1; f = cm.c; fl = fine_loc(a, lc, cm, m, d, 2);
      } else if (g[d] > C.lo[d] && cm.c < 0 && cu.c >= 0) {
        side = -1; f = cu.c; fl = fine_loc(a, lc, cu, g, -1, 0);
      }
      if (!side) return false;
      if (row) {
        const int r[7] = {l, Q.q, d, loc(a, Q.q, g), side, f, fl};
        for (int i = 0; i < 7; ++i) row[i] = r[i];
        a.face_row[Q.fo + p] = (int)rown;
      }
      return true;
    }
    if (k == 1) {
      if (cm.c < 0 && cu.c < 0) return false;
      if (row) {
        int bf = -1, bl = 0;
        if (cm.c >= 0) { bf = cm.c; bl = fine_loc(a, lc, cm, m, d, 2); }
        if (cu.c >= 0) {
          const int L2 = fine_loc(a, lc, cu, g, -1, 0);
          if (bf < 0 || cu.c < bf || (cu.c == bf && L2 < bl)) { bf = cu.c; bl = L2; }
        }
        const int r[6] = {l, Q.q, d, loc(a, Q.q, g), bf, bl};
        for (int i = 0; i < 6; ++i) row[i] = r[i];
      }
      return true;
    }
    // k == 2: a face with both cells uncovered touching a coarse-fine edge
    if (cm.c >= 0 || cu.c >= 0) return false;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int e[4] = {-1, -1, -1, -1};
    bool any = false;
    for (int slot = 0; slot < 4; ++slot) {
      const int comp = slot < 2 ? t2 : t1;
      if (dim == 2 && comp != 2) continue;
      int gs[3] = {g[0], g[1], g[2]};
      gs[slot < 2 ? t1 : t2] += slot & 1;
      int ncov, bf, bl;
      edge_cover(a, qi, comp, gs, &ncov, &bf, &bl);
      if (ncov < 1 || ncov > 3) continue;
      any = true;
      if (row) {
        int Lm;
        long long pos;
        edge_owner(a, qi, comp, gs, &Lm, &pos);
        e[slot] = pos >= 0 ? a.edge_row[pos] : -1;
      }
    }
    if (!any) return false;
    if (row) {
      const int r[8] = {l, Q.q, d, loc(a, Q.q, g), e[0], e[1], e[2], e[3]};
      for (int i = 0; i < 8; ++i) row[i] = r[i];
    }
    return true;
  }
  if (SPACE == 1) {  // the cell g
    const Cov v = cov(a, Q, C, g);
    if (k == 0) {
      if (v.c < 0) return false;
      if (row) {
        const int r[5] = {l, Q.q, loc(a, Q.q, g), v.c, fine_loc(a, lc, v, g, -1, 0)};
        for (int i = 0; i < 5; ++i) row[i] = r[i];
      }
      return true;
    }
    if (v.c >= 0) return false;
    int slots[6] = {-1, -1, -1, -1, -1, -1};
    bool any = false;
    long long fo = 0;  // first position of the d-faces in the patch's face range
    for (int dd = 0; dd < dim; ++dd) {
      int b[3], dir;
      sub_box(0, dim, dd, C.n, b, &dir);
      for (int side = 0; side < 2; ++side) {
        int h[3] = {g[0], g[1], g[2]};
        h[dd] += side ? 1 : -1;
        if (cov(a, Q, C, h).c < 0) continue;
        any = true;
        if (row) {
          int f[3] = {g[0] - C.lo[0], g[1] - C.lo[1], dim == 3 ? g[2] - C.lo[2] : 0};
          f[dd] += side;
          slots[2 * dd + side] = a.face_row[Q.fo + fo + f[0] + (long long)b[0] * (f[1] + (long long)b[1] * f[2])];
        }
      }
      fo += (long long)b[0] * b[1] * b[2];
    }
    if (!any) return false;
    if (row) {
      const int r[9] = {l, Q.q, loc(a, Q.q, g), slots[0], slots[1], slots[2], slots[3], slots[4], slots[5]};
      for (int i = 0; i < 9; ++i) row[i] = r[i];
    }
    return true;
  }
  // SPACE 2: the edge of component d at g
  int ncov, bf, bl;
  edge_cover(a, qi, d, g, &ncov, &bf, &bl);
  if (ncov < 1 || ncov > 3) return false;
  int Lm;
  long long pos;
  const int Le = loc(a, Q.q, g);
  const int own = edge_owner(a, qi, d, g, &Lm, &pos);
  if (own != qi || Lm != Le) return false;
  if (row) {
    const int r[6] = {l, Q.q, d, Le, bf, bl};
    for (int i = 0; i < 6; ++i) row[i] = r[i];
    a.edge_row[Q.eo + p] = (int)rown;
  }
  return true;
}

__global__ void k_cover(MArgs a, const int* pairs, int npairs) {
  const int pi = blockIdx.x;
  if (pi >= npairs) return;
  const int qi = pairs[3 * pi], f = pairs[3 * pi + 1], code = pairs[3 * pi + 2];
  const MQc& Q = a.Q[qi];
  const MPatch& C = a.P[Q.q];
  const MPatch& F = a.P[f];
  const int lc = C.level;
  int s[3], a0[3], a1[3];
  shift_of(code, s);
  for (int e = 0; e < 3; ++e) {
    if (e >= a.dim) { a0[e] = 0; a1[e] = 1; continue; }
    a0[e] = max(C.lo[e] - 1, F.lo[e] / 2 + s[e] * Nl(a, lc, e));
    a1[e] = min(C.lo[e] + C.n[e] + 1, (F.lo[e] + F.n[e]) / 2 + s[e] * Nl(a, lc, e));
    if (a1[e] <= a0[e]) return;
  }
  const int nx = a1[0] - a0[0], ny = a1[1] - a0[1], nz = a1[2] - a0[2];
  const long long tot = (long long)nx * ny * nz;
  const int e0 = C.n[0] + 2, e1 = C.n[1] + 2;
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int x = a0[0] + (int)(t % nx), y = a0[1] + (int)((t / nx) % ny), z = a0[2] + (int)(t / ((long long)nx * ny));
    const int zz = a.dim == 3 ? z - C.lo[2] + 1 : 0;
    const long long i = Q.cov + ((long long)zz * e1 + (y - C.lo[1] + 1)) * e0 + (x - C.lo[0] + 1);
    a.cov_c[i] = f;
    a.cov_s[i] = (signed char)code;
  }
}

// exclusive scan of one value per thread over the block; *total gets the sum
__device__ __forceinline__ int block_scan(int v, int* total) {
  __shared__ int warp_sum[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < NT / 32 ? warp_sum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_sum[lane] = s;  // inclusive prefix of the warp sums
  }
  __syncthreads();
  const int before = (w ? warp_sum[w - 1] : 0) + x - v;
  *total = warp_sum[NT / 32 - 1];
  __syncthreads();
  return before;
}

// count (EMIT false) or emit (EMIT true) the rows of one space's lists, one
// chunk of 1024 positions per block, 4 consecutive positions per thread
template <int SPACE, bool EMIT>
__global__ void __launch_bounds__(NT) k_rows(MArgs a) {
  const int ch = blockIdx.x;
  if (ch >= a.nchunks) return;
  const int qi = a.chunks[3 * ch], cnt = a.chunks[3 * ch + 2];
  const long long p0 = a.chunks[3 * ch + 1];
  const int nl = nlists(SPACE);
  for (int k = 0; k < nl; ++k) {
    const int list = lists_of(SPACE, k);
    unsigned has = 0;
    int mine = 0;
    for (int i = 0; i < 4; ++i) {
      const int t = 4 * threadIdx.x + i;
      if (t < cnt && eval<SPACE>(a, qi, p0 + t, k, nullptr, 0)) { has |= 1u << i; ++mine; }
    }
    int total;
    const int before = block_scan(mine, &total);
    if (!EMIT) {
      if (threadIdx.x == 0) a.counts[(long long)ch * 3 + k] = total;
      continue;
    }
    long long r = a.first[(long long)ch * 3 + k] + before;
    for (int i = 0; i < 4; ++i) {
      if (!(has & (1u << i))) continue;
      eval<SPACE>(a, qi, p0 + 4 * threadIdx.x + i, k, a.out[list] + width(list) * r, r);
      ++r;
    }
  }
}


// Host tables of a hierarchy for the builder: patches, coarse patches (levels
// 0 .. nlev-2 in level order, ascending ids), neighbour entries, cover pairs
// and the chunks of the three position spaces.
struct Tables {
  std::vector<MPatch> P;
  std::vector<MQc> Q;
  std::vector<int> nbrs, pairs, chunks[3];
  long long cov_tot = 0, face_tot = 0, edge_tot = 0;
  int nch(int s) const { return (int)chunks[s].size() / 3; }
};

inline void build_tables(const amrmhd::Hierarchy& H, Tables& t) {
  const int dim = H.dim, nlev = H.nlev, np = (int)H.p.size();
  t.P.assign(np, MPatch());
  for (int q = 0; q < np; ++q) {
    for (int d = 0; d < 3; ++d) { t.P[q].lo[d] = H.p[q].lo[d]; t.P[q].n[d] = H.p[q].n[d]; t.P[q].ext[d] = H.p[q].ext[d]; }
    t.P[q].level = H.p[q].level;
  }
  std::vector<int> qi_of(np, -1);
  for (int l = 0; l + 1 < nlev; ++l)
    for (int q : H.level_patches[l]) { qi_of[q] = (int)t.Q.size(); t.Q.push_back(MQc{q, 0, 0, 0, 0, 0}); }
  auto vol = [](int a, int b, int c) { return (long long)a * b * c; };
  auto code = [](const int* s) { return (s[0] + 1) + 3 * (s[1] + 1) + 9 * (s[2] + 1); };
  for (int i = 0; i < (int)t.Q.size(); ++i) {
    MQc& C = t.Q[i];
    const int* n = H.p[C.q].n;
    C.nb0 = (int)t.nbrs.size() / 2;
    t.nbrs.push_back(i);
    t.nbrs.push_back(13);
    for (const amrmhd::Nbr& x : H.nbr[C.q]) {
      t.nbrs.push_back(qi_of[x.q]);
      t.nbrs.push_back(code(x.s));
    }
    C.nb1 = (int)t.nbrs.size() / 2;
    // cover pairs: the children of the patch and of its neighbours, with the neighbour's shift
    auto add_children = [&](int src, const int* s) {
      for (int f : H.children[src]) {
        t.pairs.push_back(i);
        t.pairs.push_back(f);
        t.pairs.push_back(code(s));
      }
    };
    for (const amrmhd::Nbr& x : H.nbr[C.q]) add_children(x.q, x.s);
    const int z0[3] = {0, 0, 0};
    add_children(C.q, z0);
    C.cov = t.cov_tot;
    t.cov_tot += vol(n[0] + 2, n[1] + 2, dim == 3 ? n[2] + 2 : 1);
    long long sizes[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d)
      sizes[0] += vol(n[0] + (d == 0), n[1] + (d == 1), dim == 3 ? n[2] + (d == 2) : 1);
    sizes[1] = vol(n[0], n[1], dim == 3 ? n[2] : 1);
    if (dim == 3)
      for (int c = 0; c < 3; ++c) sizes[2] += vol(n[0] + (c != 0), n[1] + (c != 1), n[2] + (c != 2));
    else
      sizes[2] = vol(n[0] + 1, n[1] + 1, 1);
    C.fo = t.face_tot;
    C.eo = t.edge_tot;
    t.face_tot += sizes[0];
    t.edge_tot += sizes[2];
    for (int s = 0; s < 3; ++s)
      for (long long p = 0; p < sizes[s]; p += CHUNK) {
        t.chunks[s].push_back(i);
        t.chunks[s].push_back((int)p);
        t.chunks[s].push_back((int)std::min<long long>(CHUNK, sizes[s] - p));
      }
  }
}

// From the per-chunk row counts (3 per chunk): the first row of every chunk
// per list (the rows of all levels in one list), the row ranges per fine level
// l (the rows of the coarse patches of level l - 1) and the totals.
inline void first_rows(const amrmhd::Hierarchy& H, const Tables& t, const std::vector<long long>* cnt,
                       std::vector<long long>* first, std::vector<std::array<int64_t, 2>>** rng, int64_t* total) {
  const int space_of[6] = {0, 2, 0, 1, 0, 1}, k_of[6] = {0, 0, 2, 0, 1, 1};
  for (int s = 0; s < 3; ++s) first[s].assign(3 * (size_t)t.nch(s), 0);
  for (int list = 0; list < 6; ++list) {
    const int s = space_of[list], k = k_of[list];
    std::vector<std::array<int64_t, 2>>& r = *rng[list];
    r.assign(H.nlev, {0, 0});
    long long acc = 0;
    int lev_prev = -1;
    for (int c = 0; c < t.nch(s); ++c) {
      const int lc = H.p[t.Q[t.chunks[s][3 * c]].q].level;
      if (lc != lev_prev) {
        for (int l = lev_prev + 2; l <= lc + 1; ++l) r[l] = {acc, acc};
        lev_prev = lc;
      }
      first[s][3 * (size_t)c + k] = acc;
      acc += cnt[s][3 * (size_t)c + k];
      r[lc + 1][1] = acc;
    }
    total[list] = acc;
  }
}


}  // namespace amrdm

namespace amrapi {

// Builds the register, reflux and restriction maps of ctx->H on the device
// into ctx->d_maps and sets H's row ranges (the host lists stay empty).
amrmhd_status device_register_maps(amrmhd_ctx* ctx) {
  using namespace amrdm;
  amrmhd::Hierarchy& H = ctx->H;
  const int dim = H.dim, nlev = H.nlev, np = (int)H.p.size();
  static const int W[6] = {7, 6, 8, 5, 6, 9};
  std::array<std::vector<std::array<int64_t, 2>>*, 6> rng = {&H.rng_cf_faces, &H.rng_cf_edges, &H.rng_emf_faces,
                                                             &H.rng_restrict_cells, &H.rng_restrict_faces,
                                                             &H.rng_reflux_cells};
  for (auto* r : rng) r->assign(nlev, {0, 0});
  for (int i = 0; i < 6; ++i) { ctx->dmap_off[i] = 0; ctx->dmap_n[i] = 0; }
  if (ctx->d_maps) { cudaFree(ctx->d_maps); ctx->d_maps = nullptr; }
  ctx->dmaps = true;
  ctx->dmaps_host = false;
  if (nlev < 2) return AMRMHD_OK;
  Tables t;
  build_tables(H, t);
  const std::vector<MPatch>& P = t.P;
  const std::vector<MQc>& Q = t.Q;
  const std::vector<int>& nbrs = t.nbrs;
  const std::vector<int>& pairs = t.pairs;
  const std::vector<int>* chunks = t.chunks;
  const int nq = (int)Q.size();
  const long long cov_tot = t.cov_tot, face_tot = t.face_tot, edge_tot = t.edge_tot;
  const int nch[3] = {(int)chunks[0].size() / 3, (int)chunks[1].size() / 3, (int)chunks[2].size() / 3};
  // one device block for the inputs and the scratch
  std::vector<char> img;
  auto put = [&](const void* src, size_t bytes) {
    const size_t o = (img.size() + 255) / 256 * 256;
    img.resize(o + bytes);
    if (bytes) std::memcpy(img.data() + o, src, bytes);
    return o;
  };
  const size_t oP = put(P.data(), sizeof(MPatch) * np), oQ = put(Q.data(), sizeof(MQc) * nq),
               oN = put(nbrs.data(), sizeof(int) * nbrs.size()), oPr = put(pairs.data(), sizeof(int) * pairs.size());
  size_t oC[3];
  for (int s = 0; s < 3; ++s) oC[s] = put(chunks[s].data(), sizeof(int) * chunks[s].size());
  const size_t in_bytes = img.size();
  size_t o = (in_bytes + 255) / 256 * 256;
  auto reserve = [&](size_t bytes) { const size_t r = o; o = (o + bytes + 255) / 256 * 256; return r; };
  const size_t oCovC = reserve(sizeof(int) * cov_tot), oCovS = reserve(cov_tot), oFR = reserve(sizeof(int) * face_tot),
               oER = reserve(sizeof(int) * edge_tot);
  size_t oCnt[3], oFirst[3];
  for (int s = 0; s < 3; ++s) {
    oCnt[s] = reserve(sizeof(long long) * 3 * nch[s]);
    oFirst[s] = reserve(sizeof(long long) * 3 * nch[s]);
  }
  // scratch from the stream-ordered allocator: freed on the stream, reused by
  // the next builder call without a device-wide synchronisation
  char* dev = nullptr;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMallocAsync((void**)&dev, o, st);
  if (e != cudaSuccess) return fail(ctx, AMRMHD_ENOMEM, std::string("device maps: ") + cudaGetErrorString(e));
  auto done = [&](amrmhd_status s, const std::string& m) {
    cudaFreeAsync(dev, st);
    return s == AMRMHD_OK ? s : fail(ctx, s, m);
  };
  e = cudaMemcpyAsync(dev, img.data(), in_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev + oCovC, 0xff, sizeof(int) * cov_tot, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev + oFR, 0xff, sizeof(int) * face_tot, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev + oER, 0xff, sizeof(int) * edge_tot, st);
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string("device maps: ") + cudaGetErrorString(e));
  MArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dim = dim;
  for (int d = 0; d < 3; ++d) a.base[d] = H.base[d];
  a.P = (const MPatch*)(dev + oP);
  a.Q = (const MQc*)(dev + oQ);
  a.nbrs = (const int*)(dev + oN);
  a.cov_c = (int*)(dev + oCovC);
  a.cov_s = (signed char*)(dev + oCovS);
  a.face_row = (int*)(dev + oFR);
  a.edge_row = (int*)(dev + oER);
  const int npairs = (int)pairs.size() / 3;
  if (npairs) k_cover<<<npairs, 128, 0, st>>>(a, (const int*)(dev + oPr), npairs);
  auto args_for = [&](int s) {
    MArgs b = a;
    b.chunks = (const int*)(dev + oC[s]);
    b.nchunks = nch[s];
    b.counts = (long long*)(dev + oCnt[s]);
    b.first = (const long long*)(dev + oFirst[s]);
    return b;
  };
  if (nch[0]) k_rows<0, false><<<nch[0], NT, 0, st>>>(args_for(0));
  if (nch[1]) k_rows<1, false><<<nch[1], NT, 0, st>>>(args_for(1));
  if (nch[2]) k_rows<2, false><<<nch[2], NT, 0, st>>>(args_for(2));
  ctx->launches += (npairs ? 1 : 0) + (nch[0] ? 1 : 0) + (nch[1] ? 1 : 0) + (nch[2] ? 1 : 0);
  std::vector<long long> cnt[3];
  for (int s = 0; s < 3; ++s) {
    cnt[s].assign(3 * (size_t)nch[s], 0);
    if (nch[s] && e == cudaSuccess)
      e = cudaMemcpyAsync(cnt[s].data(), dev + oCnt[s], sizeof(long long) * 3 * nch[s], cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string("device maps (count): ") + cudaGetErrorString(e));
  std::vector<long long> first[3];
  first_rows(H, t, cnt, first, rng.data(), ctx->dmap_n);
  size_t out_bytes = 0;
  for (int list = 0; list < 6; ++list) {
    ctx->dmap_off[list] = out_bytes / sizeof(int);
    out_bytes = (out_bytes + sizeof(int) * W[list] * ctx->dmap_n[list] + 255) / 256 * 256;
  }
  e = cudaMalloc((void**)&ctx->d_maps, std::max<size_t>(out_bytes, 256));
  if (e != cudaSuccess) { ctx->d_maps = nullptr; return done(AMRMHD_ENOMEM, std::string("device maps: ") + cudaGetErrorString(e)); }
  for (int s = 0; s < 3 && e == cudaSuccess; ++s)
    if (nch[s])
      e = cudaMemcpyAsync(dev + oFirst[s], first[s].data(), sizeof(long long) * 3 * nch[s], cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string("device maps: ") + cudaGetErrorString(e));
  for (int list = 0; list < 6; ++list) a.out[list] = ctx->d_maps + ctx->dmap_off[list];
  // edges first (the emf faces read their row numbers), then faces (the
  // reflux cells read the coarse-fine face rows), then cells
  if (nch[2]) k_rows<2, true><<<nch[2], NT, 0, st>>>(args_for(2));
  if (nch[0]) k_rows<0, true><<<nch[0], NT, 0, st>>>(args_for(0));
  if (nch[1]) k_rows<1, true><<<nch[1], NT, 0, st>>>(args_for(1));
  ctx->launches += (nch[0] ? 1 : 0) + (nch[1] ? 1 : 0) + (nch[2] ? 1 : 0);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string("device maps (emit): ") + cudaGetErrorString(e));
  return done(AMRMHD_OK, "");
}

// The host copies of the device-built lists (for the map export).
amrmhd_status download_register_maps(amrmhd_ctx* ctx) {
  if (!ctx->dmaps || ctx->dmaps_host) return AMRMHD_OK;
  static const int W[6] = {7, 6, 8, 5, 6, 9};
  amrmhd::Hierarchy& H = ctx->H;
  std::vector<int32_t>* v[6] = {&H.cf_faces, &H.cf_edges, &H.emf_faces, &H.restrict_cells, &H.restrict_faces,
                                &H.reflux_cells};
  for (int list = 0; list < 6; ++list) {
    v[list]->assign((size_t)W[list] * ctx->dmap_n[list], 0);
    if (ctx->dmap_n[list]) {
      cudaError_t e = cudaMemcpy(v[list]->data(), ctx->d_maps + ctx->dmap_off[list],
                                 sizeof(int32_t) * v[list]->size(), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return fail(ctx, AMRMHD_ECUDA, std::string("map download: ") + cudaGetErrorString(e));
    }
  }
  ctx->dmaps_host = true;
  return AMRMHD_OK;
}

}  // namespace amrapi
