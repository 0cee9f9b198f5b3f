// Ghost-fill boxes and regrid transfer boxes built on the device: the rows of
// the host builders (hierarchy.cpp's ghost boxes, regrid.cpp's transfer_maps)
// bit for bit and in the same order.
//
// A task is one patch and one kind of position: d = -1 its cells, d >= 0 its
// d-faces. Every position of the task's box gets a label id:
//
// * ghost boxes (Sec. 2 and 4: the ghost zones of a patch, filled from its
//   same-level neighbours, by prolongation from the coarser level, or from the
//   physical boundary): the same-level neighbour (with its periodic shift)
//   holding the position, on a face held by two the smaller (patch, local
//   index); else the first coarse candidate and periodic image holding the
//   parent cell; outside a bounded side the boundary state; the patch's own
//   positions are not labelled;
// * transfer boxes (Sec. 2, the overlap step of a regrid): a copy from the old
//   fine patch (and shift) holding the position where the old fine level
//   covered the parent cell (on a face between two old patches the smaller
//   (patch, local index)), else a prolongation from the new coarse patch.
//
// Equal ids are then merged greedily into boxes (x runs, then y rows, then z
// slabs, in raster order of the first position), the host builders' merge, by
// one warp with warp-wide comparisons. A task whose label grid fits in shared
// memory is labelled and merged by one CTA there; larger tasks use a grid in
// global memory. Candidate lists are pruned on the host to the entries that
// can meet the task's box, in the host builders' order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.hpp"

namespace amrbx {

struct BPatch {
  int lo[3], n[3], ext[3], level;
};

struct BTask {
  int q, d;          // patch; -1 its cells, else its d-faces
  int ex[3], g0[3];  // the label box and the global position of its local origin
  int s0, s1;        // ghost: same-level (patch, shift) entries; transfer: old (patch, shift) entries, in pairs
  int p0, p1;        // ghost: prolongation (coarse patch, image) entries in pairs; transfer: coarse ids in ids
  int touches;       // ghost: the box reaches outside a bounded side
  int transfer;      // 1: a transfer task
  long long go;      // its grid in global memory (large tasks), else -1
};

struct BArgs {
  int dim;
  int base[3], per[3], bc[3][2];
  const BPatch* P;   // the (new) hierarchy's patches
  const BPatch* PO;  // transfer: the old hierarchy's patches
  int have_old;      // transfer: the old hierarchy has the level
  const BTask* T;
  const int* pairs;  // (patch, code) entries
  const int* ids;    // transfer: coarse candidate ids
  int* G;            // label grids of the large tasks
  long long* cnt;    // boxes per task
  const long long* first;
  int* out_cells;
  int* out_faces;
  unsigned long long* err;  // smallest (task << 32 | position) without a source
  int* scratch;             // one pass: up to cap rows per task at task * cap
  int cap;
};

__host__ __device__ __forceinline__ int Nl(const BArgs& a, int l, int e) { return e < a.dim ? (a.base[e] << l) : 1; }

__host__ __device__ __forceinline__ void shift_of(int code, int* s) {
  s[0] = code % 3 - 1;
  s[1] = (code / 3) % 3 - 1;
  s[2] = code / 9 - 1;
}

// (positions within a task are below 2^31: a patch has at most 2^28 elements per field)
__host__ __device__ __forceinline__ void decode(const BTask& T, int t, int* x) {
  const int r = t / T.ex[0];
  x[0] = t - r * T.ex[0];
  x[1] = r % T.ex[1];
  x[2] = r / T.ex[1];
}

// ---- ghost boxes

// label of position t of ghost task T: -1 the patch's own position, -3 no source
__host__ __device__ inline int ghost_label(const BArgs& a, const BTask& T, int t) {
  const BPatch& P = a.P[T.q];
  const int l = P.level, d = T.d, dim = a.dim;
  const int ns = T.s1 - T.s0, np = T.p1 - T.p0;
  int x[3];
  decode(T, t, x);
  bool own = true;
  for (int e = 0; e < dim; ++e) own = own && x[e] >= 4 && x[e] < P.n[e] + 4 + (e == d ? 1 : 0);
  if (own) return -1;
  const int g[3] = {T.g0[0] + x[0], T.g0[1] + x[1], T.g0[2] + x[2]};
  if (T.touches) {  // outside a bounded side: the boundary state
    bool out = false, inflow = false;
    int code = 0, w3 = 1;
    for (int e = 0; e < dim; ++e, w3 *= 3) {
      if (a.per[e]) continue;
      const int top = e == d ? Nl(a, l, e) : Nl(a, l, e) - 1;
      if (g[e] < 0) { out = true; code += 1 * w3; inflow |= a.bc[e][0] == 2; }
      else if (g[e] > top) { out = true; code += 2 * w3; inflow |= a.bc[e][1] == 2; }
    }
    if (out) return ns + np + (inflow ? 27 : code);
  }
  // same-level neighbours: a cell lies in one; a face held by two goes to the
  // smaller (patch, local index)
  int id = -1, bq = 0, bL = 0;
  for (int i = T.s0; i < T.s1; ++i) {
    const int qq = a.pairs[2 * i];
    const BPatch& Q = a.P[qq];
    int s[3];
    shift_of(a.pairs[2 * i + 1], s);
    bool in = true;
    int dl[3] = {0, 0, 0};
    for (int e = 0; e < dim; ++e) {
      const int o = s[e] * Nl(a, l, e);
      in = in && x[e] >= Q.lo[e] + o - T.g0[e] && x[e] < Q.lo[e] + Q.n[e] + o + (e == d ? 1 : 0) - T.g0[e];
      dl[e] = P.lo[e] - Q.lo[e] - o;
    }
    if (!in) continue;
    const int L = (x[0] + dl[0]) + Q.ext[0] * ((x[1] + dl[1]) + Q.ext[1] * (x[2] + dl[2]));
    if (d < 0 || id < 0 || qq < bq || (qq == bq && L < bL)) { id = i - T.s0; bq = qq; bL = L; }
  }
  if (id >= 0) return id;
  // prolongation: the first coarse candidate and image holding the parent cell
  for (int j = T.p0; j < T.p1; ++j) {
    const BPatch& C = a.P[a.pairs[2 * j]];
    int w[3];
    shift_of(a.pairs[2 * j + 1], w);
    bool in = true;
    for (int e = 0; e < dim; ++e) {
      const int aux = w[e] * Nl(a, l, e);
      const int top = (e == d && !a.per[e] && C.lo[e] + C.n[e] == Nl(a, l - 1, e)) ? 1 : 0;
      in = in && x[e] >= 2 * C.lo[e] - aux - T.g0[e] && x[e] < 2 * (C.lo[e] + C.n[e]) + top - aux - T.g0[e];
    }
    if (in) return ns + (j - T.p0);
  }
  return -3;
}

__host__ __device__ inline void ghost_row(const BArgs& a, const BTask& T, int id, int* row) {
  const BPatch& P = a.P[T.q];
  const int l = P.level, dim = a.dim, ns = T.s1 - T.s0, np = T.p1 - T.p0;
  int kind, src, aux[3] = {0, 0, 0};
  if (id < ns) {
    const int i = T.s0 + id;
    src = a.pairs[2 * i];
    kind = 0;
    int s[3];
    shift_of(a.pairs[2 * i + 1], s);
    for (int e = 0; e < dim; ++e) aux[e] = P.lo[e] - a.P[src].lo[e] - s[e] * Nl(a, l, e);
  } else if (id < ns + np) {
    const int j = T.p0 + id - ns;
    kind = 1;
    src = a.pairs[2 * j];
    int w[3];
    shift_of(a.pairs[2 * j + 1], w);
    for (int e = 0; e < dim; ++e) aux[e] = w[e] * Nl(a, l, e);
  } else if (id < ns + np + 27) {
    kind = 2;
    src = T.q;
    int code = id - ns - np;
    for (int e = 0; e < 3; ++e) {
      const int digit = code % 3;
      code /= 3;
      const int top = e == T.d ? Nl(a, l, e) : Nl(a, l, e) - 1;
      aux[e] = (e >= dim || digit == 0) ? -1 : (digit == 1 ? 0 : top);
    }
  } else {
    kind = 3;
    src = -1;
  }
  row[0] = T.q;
  row[1] = T.d;
  row[2] = kind;
  row[3] = src;
  row[10] = aux[0];
  row[11] = aux[1];
  row[12] = aux[2];
}

// ---- transfer boxes

// the old (patch, shift) entry holding fine cell h, or -1
__host__ __device__ inline int old_owner(const BArgs& a, const BTask& T, const int* h) {
  const int lf = a.P[T.q].level;
  for (int i = T.s0; i < T.s1; ++i) {
    const BPatch& O = a.PO[a.pairs[2 * i]];
    int s[3];
    shift_of(a.pairs[2 * i + 1], s);
    bool in = true;
    for (int e = 0; e < a.dim; ++e) {
      const int o = s[e] * Nl(a, lf, e);
      in = in && h[e] >= O.lo[e] + o && h[e] < O.lo[e] + O.n[e] + o;
    }
    if (in) return i;
  }
  return -1;
}

// the owner lookup of the host emulation and the global-memory path: a scan of the entries
struct LoopOwner {
  const BArgs& a;
  const BTask& T;
  __host__ __device__ int operator()(const int* h) const { return old_owner(a, T, h); }
};

// the shared-memory path: the entries scattered over the patch's box grown by
// 2 fine cells (entry index relative to T.s0, or -1)
template <class ET>
struct GridOwner {
  const BArgs& a;
  const BTask& T;
  const ET* grid;
  __host__ __device__ int operator()(const int* h) const {
    const BPatch& P = a.P[T.q];
    long long i = 0, st = 1;
    for (int e = 0; e < a.dim; ++e) {
      const int x = h[e] - (P.lo[e] - 2), n = P.n[e] + 4;
      if (x < 0 || x >= n) return old_owner(a, T, h);
      i += x * st;
      st *= n;
    }
    return grid[i] < 0 ? -1 : T.s0 + grid[i];
  }
};

// coarse cell c covered by the old fine level
template <class OW>
__host__ __device__ inline bool old_covers(const BArgs& a, const OW& own, const int* c) {
  if (!a.have_old) return false;
  int h[3];
  for (int e = 0; e < 3; ++e) h[e] = e < a.dim ? 2 * c[e] : 0;
  return own(h) >= 0;
}

// the new coarse patch candidate holding coarse cell c (periodic wrap), or -1
__host__ __device__ inline int new_coarse(const BArgs& a, const BTask& T, const int* c) {
  const int lc = a.P[T.q].level - 1;
  int w[3];
  for (int e = 0; e < 3; ++e) {
    w[e] = c[e];
    if (e < a.dim && a.per[e]) { const int n = Nl(a, lc, e); w[e] = (w[e] % n + n) % n; }
  }
  for (int j = T.p0; j < T.p1; ++j) {
    const BPatch& C = a.P[a.ids[j]];
    bool in = true;
    for (int e = 0; e < a.dim; ++e) in = in && w[e] >= C.lo[e] && w[e] < C.lo[e] + C.n[e];
    if (in) return j;
  }
  return -1;
}

// local index, in the old patch of entry i seen through its shift, of fine position h
__host__ __device__ inline int old_loc(const BArgs& a, const BTask& T, int i, const int* h) {
  const int lf = a.P[T.q].level;
  const BPatch& O = a.PO[a.pairs[2 * i]];
  int s[3], w[3];
  shift_of(a.pairs[2 * i + 1], s);
  for (int e = 0; e < 3; ++e) w[e] = e < a.dim ? h[e] - s[e] * Nl(a, lf, e) : 0;
  const int x = w[0] - O.lo[0] + 4, y = w[1] - O.lo[1] + 4, z = a.dim == 3 ? w[2] - O.lo[2] + 4 : 0;
  return x + O.ext[0] * (y + O.ext[1] * z);
}

// label of position t of transfer task T: a copy (id = old entry index) or a
// prolongation (id = ns + 8 coarse candidate + the dimensions where the face
// position wraps); -3 no source
template <class OW>
__host__ __device__ inline int transfer_label(const BArgs& a, const BTask& T, int t, const OW& own) {
  const BPatch& P = a.P[T.q];
  const int lf = P.level, d = T.d, dim = a.dim;
  const int ns = T.s1 - T.s0;
  int x[3], g[3], pq[3];
  decode(T, t, x);
  for (int e = 0; e < 3; ++e) {
    g[e] = e < dim ? P.lo[e] + x[e] : 0;
    pq[e] = e < dim ? g[e] >> 1 : 0;
  }
  if (d < 0) {
    if (old_covers(a, own, pq)) {
      const int i = own(g);
      return i < 0 ? -3 : i - T.s0;
    }
    const int jc = new_coarse(a, T, pq);
    return jc < 0 ? -3 : ns + 8 * (jc - T.p0);
  }
  int m[3] = {g[0], g[1], g[2]}, pm[3];
  m[d] -= 1;
  for (int e = 0; e < 3; ++e) pm[e] = e < dim ? m[e] >> 1 : 0;
  const bool interior = pq[d] == pm[d];
  const bool copy = interior ? old_covers(a, own, pq) : (old_covers(a, own, pq) || old_covers(a, own, pm));
  if (copy) {  // the owners of the cells on the face's two sides
    int best = -1, bi = 0, bl = 0;
    const int i1 = own(g);
    if (i1 >= 0) { best = a.pairs[2 * i1]; bi = i1; bl = old_loc(a, T, i1, g); }
    const int i0 = own(m);
    if (i0 >= 0) {
      const int L = old_loc(a, T, i0, g);
      if (best < 0 || a.pairs[2 * i0] < best || (a.pairs[2 * i0] == best && L < bl)) { best = a.pairs[2 * i0]; bi = i0; bl = L; }
    }
    return best < 0 ? -3 : bi - T.s0;
  }
  int c[3] = {pq[0], pq[1], pq[2]};
  if (!a.per[d] && g[d] == Nl(a, lf, d)) c[d] -= 1;
  const int jc = new_coarse(a, T, c);
  if (jc < 0) return -3;
  int bits = 0;
  for (int e = 0; e < dim; ++e)
    if (a.per[e] && g[e] == Nl(a, lf, e)) bits |= 1 << e;
  return ns + 8 * (jc - T.p0) + bits;
}

__host__ __device__ inline void transfer_row(const BArgs& a, const BTask& T, int id, int* row) {
  const BPatch& P = a.P[T.q];
  const int lf = P.level, dim = a.dim, ns = T.s1 - T.s0;
  int kind, src, aux[3] = {0, 0, 0};
  if (id < ns) {
    kind = 0;
    const int i = T.s0 + id;
    src = a.pairs[2 * i];
    int s[3];
    shift_of(a.pairs[2 * i + 1], s);
    for (int e = 0; e < dim; ++e) aux[e] = P.lo[e] - a.PO[src].lo[e] - s[e] * Nl(a, lf, e);
  } else {
    kind = 1;
    src = a.ids[T.p0 + (id - ns) / 8];
    const int bits = (id - ns) % 8;
    for (int e = 0; e < dim; ++e) aux[e] = (bits >> e) & 1 ? -Nl(a, lf, e) : 0;
  }
  row[0] = T.q;
  row[1] = T.d;
  row[2] = kind;
  row[3] = src;
  row[10] = aux[0];
  row[11] = aux[1];
  row[12] = aux[2];
}

// closure cell c of new patch task T: a coarse cell of the footprint not
// covered by the old fine level with a face neighbour (inside the domain) that is
template <class OW>
__host__ __device__ inline bool closure_cell(const BArgs& a, const BTask& T, const int* c, const OW& own) {
  const int lc = a.P[T.q].level - 1, dim = a.dim;
  if (old_covers(a, own, c)) return false;
  for (int e = 0; e < dim; ++e)
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int nb[3] = {c[0], c[1], c[2]};
      nb[e] += sgn;
      bool in = true;
      for (int e2 = 0; e2 < dim; ++e2)
        if (!a.per[e2] && (nb[e2] < 0 || nb[e2] >= Nl(a, lc, e2))) in = false;
      if (in && old_covers(a, own, nb)) return true;
    }
  return false;
}

__host__ __device__ __forceinline__ int label_of(const BArgs& a, const BTask& T, int t) {
  return T.transfer ? transfer_label(a, T, t, LoopOwner{a, T}) : ghost_label(a, T, t);
}

// ---- the greedy merge (one warp)

// MODE 0 counts the boxes, 1 writes them at the task's first row, 2 counts
// them and writes the first a.cap of them into the task's scratch rows
template <int MODE, class GT>
__device__ void warp_merge(const BArgs& a, int ti, GT* G) {
  const BTask& T = a.T[ti];
  const int lane = threadIdx.x & 31;
  const int e0 = T.ex[0], e1 = T.ex[1], e2 = T.ex[2];
  const int tot = e0 * e1 * e2;
  auto at = [&](int x, int y, int z) { return (z * e1 + y) * e0 + x; };
  const unsigned FULL = 0xffffffffu;
  int pos = 0;
  long long count = 0;
  const long long base = MODE == 1 ? a.first[ti] : 0;
  int* out = MODE == 2 ? a.scratch + 13LL * ti * a.cap : (T.d < 0 ? a.out_cells : a.out_faces);
  for (;;) {
    int t0 = -1;
    for (; pos < tot; pos += 32) {
      const int idx = pos + lane;
      const unsigned m = __ballot_sync(FULL, idx < tot && G[idx] >= 0);
      if (m) { t0 = pos + __ffs(m) - 1; break; }
    }
    if (t0 < 0) break;
    const int k = G[t0];
    const int r0 = t0 / e0, a0 = t0 - r0 * e0, b0 = r0 % e1, c0 = r0 / e1;
    int nx = 1;
    for (;;) {
      const int x = a0 + nx + lane;
      const unsigned m = __ballot_sync(FULL, x < e0 && G[t0 + nx + lane] == k);
      if (m == FULL) { nx += 32; continue; }
      nx += __ffs(~m) - 1;
      break;
    }
    auto row_ok = [&](int y, int z) {
      for (int i0 = 0; i0 < nx; i0 += 32) {
        const int i = i0 + lane;
        if (!__all_sync(FULL, i >= nx || G[at(a0 + i, y, z)] == k)) return false;
      }
      return true;
    };
    int ny = 1, nz = 1;
    while (b0 + ny < e1 && row_ok(b0 + ny, c0)) ++ny;
    auto slab_ok = [&](int z) {
      for (int j = 0; j < ny; ++j)
        if (!row_ok(b0 + j, z)) return false;
      return true;
    };
    while (c0 + nz < e2 && slab_ok(c0 + nz)) ++nz;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int i = lane; i < nx; i += 32) G[at(a0 + i, b0 + y, c0 + z)] = -2;
    __syncwarp();
    if (MODE != 0 && lane == 0 && (MODE == 1 || count < a.cap)) {
      int* r = out + 13 * (base + count);
      const int o = T.transfer ? 4 : 0;  // transfer boxes: lo in the patch's ghosted frame
      if (T.transfer) transfer_row(a, T, k, r);
      else ghost_row(a, T, k, r);
      r[4] = a0 + o;
      r[5] = b0 + o;
      r[6] = a.dim == 3 ? c0 + o : c0;
      r[7] = nx;
      r[8] = ny;
      r[9] = nz;
    }
    ++count;
    pos = t0 + 1;
  }
  if (MODE != 1 && lane == 0) a.cnt[ti] = count;
}

// the positions of the task box meeting [lo, hi) (local coordinates): false if none
__device__ __forceinline__ bool clip_box(const BTask& T, int* lo, int* hi) {
  for (int e = 0; e < 3; ++e) {
    lo[e] = max(lo[e], 0);
    hi[e] = min(hi[e], T.ex[e]);
    if (hi[e] <= lo[e]) return false;
  }
  return true;
}

__device__ __forceinline__ bool own_pos(const BPatch& P, int d, int dim, const int* x) {
  bool own = true;
  for (int e = 0; e < dim; ++e) own = own && x[e] >= 4 && x[e] < P.n[e] + 4 + (e == d ? 1 : 0);
  return own;
}

// f(x) for every position x of the box [lo, hi): one warp per row, lanes along x
template <class F>
__device__ __forceinline__ void for_box(const int* lo, const int* hi, F&& f) {
  const int by = hi[1] - lo[1], rows = by * (hi[2] - lo[2]);
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = threadIdx.x >> 5; r < rows; r += nw) {
    int x[3];
    x[1] = lo[1] + r % by;
    x[2] = lo[2] + r / by;
    for (x[0] = lo[0] + lane; x[0] < hi[0]; x[0] += 32) f(x);
  }
}

// f(x) for every position of the box [lo, hi) outside the patch's own
// positions: the box minus the own box, as at most 6 disjoint slabs (z, then
// y, then x)
template <class F>
__device__ __forceinline__ void for_shell(const BPatch& P, int d, int dim, const int* lo, const int* hi, F&& f) {
  int l[3] = {lo[0], lo[1], lo[2]}, h[3] = {hi[0], hi[1], hi[2]};
  for (int e = dim - 1; e >= 0; --e) {
    const int o0 = 4, o1 = P.n[e] + 4 + (e == d ? 1 : 0);
    if (l[e] < o0) {
      int sl[3] = {l[0], l[1], l[2]}, sh[3] = {h[0], h[1], h[2]};
      sh[e] = min(h[e], o0);
      if (sh[e] > sl[e]) for_box(sl, sh, f);
    }
    if (h[e] > o1) {
      int sl[3] = {l[0], l[1], l[2]}, sh[3] = {h[0], h[1], h[2]};
      sl[e] = max(l[e], o1);
      if (sh[e] > sl[e]) for_box(sl, sh, f);
    }
    l[e] = max(l[e], o0);
    h[e] = min(h[e], o1);
    if (h[e] <= l[e]) return;
  }
}

// Ghost labels of task T into the shared-memory grid G by scattering the
// entries' boxes in the host builder's order (the labels of ghost_label)
template <class ET>
__device__ void ghost_scatter(const BArgs& a, int ti, ET* G) {
  const BTask& T = a.T[ti];
  const BPatch& P = a.P[T.q];
  const int l = P.level, d = T.d, dim = a.dim, ns = T.s1 - T.s0, np = T.p1 - T.p0;
  const int tot = T.ex[0] * T.ex[1] * T.ex[2];
  for (int t = threadIdx.x; t < tot; t += blockDim.x) G[t] = -1;
  __syncthreads();
  auto at = [&](const int* x) { return (x[2] * T.ex[1] + x[1]) * T.ex[0] + x[0]; };
  // same-level neighbours in list order: a cell is held by one; a face held by
  // two goes to the smaller (patch, local index)
  for (int i = T.s0; i < T.s1; ++i) {
    const int qq = a.pairs[2 * i];
    const BPatch& Q = a.P[qq];
    int s[3], lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, dl[3] = {0, 0, 0};
    shift_of(a.pairs[2 * i + 1], s);
    for (int e = 0; e < dim; ++e) {
      const int o = s[e] * Nl(a, l, e);
      lo[e] = Q.lo[e] + o - T.g0[e];
      hi[e] = Q.lo[e] + Q.n[e] + o + (e == d ? 1 : 0) - T.g0[e];
      dl[e] = P.lo[e] - Q.lo[e] - o;
    }
    if (clip_box(T, lo, hi))
      for_shell(P, d, dim, lo, hi, [&](const int* x) {
        const int t = at(x);
        const int cur = G[t];
        bool take = d < 0 || cur < 0;
        if (!take) {
          const int L = (x[0] + dl[0]) + Q.ext[0] * ((x[1] + dl[1]) + Q.ext[1] * (x[2] + dl[2]));
          const int ci = T.s0 + cur, cq = a.pairs[2 * ci];
          const BPatch& C = a.P[cq];
          int cs[3], cd[3] = {0, 0, 0};
          shift_of(a.pairs[2 * ci + 1], cs);
          for (int e = 0; e < dim; ++e) cd[e] = P.lo[e] - C.lo[e] - cs[e] * Nl(a, l, e);
          const int Lc = (x[0] + cd[0]) + C.ext[0] * ((x[1] + cd[1]) + C.ext[1] * (x[2] + cd[2]));
          take = qq < cq || (qq == cq && L < Lc);
        }
        if (take) G[t] = (ET)(i - T.s0);
      });
    __syncthreads();
  }
  // prolongation: the first coarse candidate and image holding the parent cell
  for (int j = T.p0; j < T.p1; ++j) {
    const BPatch& C = a.P[a.pairs[2 * j]];
    int w[3], lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    shift_of(a.pairs[2 * j + 1], w);
    for (int e = 0; e < dim; ++e) {
      const int aux = w[e] * Nl(a, l, e);
      const int top = (e == d && !a.per[e] && C.lo[e] + C.n[e] == Nl(a, l - 1, e)) ? 1 : 0;
      lo[e] = 2 * C.lo[e] - aux - T.g0[e];
      hi[e] = 2 * (C.lo[e] + C.n[e]) + top - aux - T.g0[e];
    }
    if (clip_box(T, lo, hi))
      for_shell(P, d, dim, lo, hi, [&](const int* x) {
        const int t = at(x);
        if (G[t] < 0) G[t] = (ET)(ns + (j - T.p0));
      });
    __syncthreads();
  }
  // outside a bounded side: the boundary state; every other ghost position must have a source
  const int lo[3] = {0, 0, 0}, hi[3] = {T.ex[0], T.ex[1], T.ex[2]};
  for_shell(P, d, dim, lo, hi, [&](const int* x) {
    const int t = at(x);
    if (T.touches) {
      const int g[3] = {T.g0[0] + x[0], T.g0[1] + x[1], T.g0[2] + x[2]};
      bool out = false, inflow = false;
      int code = 0, w3 = 1;
      for (int e = 0; e < dim; ++e, w3 *= 3) {
        if (a.per[e]) continue;
        const int top = e == d ? Nl(a, l, e) : Nl(a, l, e) - 1;
        if (g[e] < 0) { out = true; code += 1 * w3; inflow |= a.bc[e][0] == 2; }
        else if (g[e] > top) { out = true; code += 2 * w3; inflow |= a.bc[e][1] == 2; }
      }
      if (out) { G[t] = (ET)(ns + np + (inflow ? 27 : code)); return; }
    }
    if (G[t] < 0) atomicMin(a.err, ((unsigned long long)ti << 32) | (unsigned long long)t);
  });
  __syncthreads();
}

// Transfer labels of task T into G: the old entries scattered over the patch's
// box grown by 2 fine cells (W), then every position's label with owner lookups in W
template <class ET>
__device__ void transfer_fill(const BArgs& a, int ti, ET* G, ET* W) {
  const BTask& T = a.T[ti];
  const BPatch& P = a.P[T.q];
  const int lf = P.level, dim = a.dim;
  int gn[3];
  for (int e = 0; e < 3; ++e) gn[e] = e < dim ? P.n[e] + 4 : 1;
  const int gw = gn[0] * gn[1] * gn[2];
  for (int t = threadIdx.x; t < gw; t += blockDim.x) W[t] = -1;
  __syncthreads();
  if (a.have_old)
    for (int i = T.s0; i < T.s1; ++i) {
      const BPatch& O = a.PO[a.pairs[2 * i]];
      int s[3], lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
      shift_of(a.pairs[2 * i + 1], s);
      bool empty = false;
      for (int e = 0; e < dim; ++e) {
        const int o = s[e] * Nl(a, lf, e);
        lo[e] = max(O.lo[e] + o - (P.lo[e] - 2), 0);
        hi[e] = min(O.lo[e] + O.n[e] + o - (P.lo[e] - 2), gn[e]);
        if (hi[e] <= lo[e]) empty = true;
      }
      if (!empty)
        for_box(lo, hi, [&](const int* x) {
          const int t = (x[2] * gn[1] + x[1]) * gn[0] + x[0];
          if (W[t] < 0) W[t] = (ET)(i - T.s0);
        });
      __syncthreads();
    }
  const GridOwner<ET> own{a, T, W};
  const int tot = T.ex[0] * T.ex[1] * T.ex[2];
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int id = transfer_label(a, T, t, own);
    if (id == -3) atomicMin(a.err, ((unsigned long long)ti << 32) | (unsigned long long)t);
    G[t] = (ET)(id < 0 ? -1 : id);
  }
  __syncthreads();
}

constexpr int kBoxThreads = 256;

// The same greedy merge by the whole CTA (the grid in shared memory): the next
// unmerged position, the x run, the rows and the slabs are each found by all
// threads at once (the smallest failing index by a shared atomic minimum), so
// the critical path is a few barriers per box rather than one warp step per
// row or 32 positions.
template <int MODE, class GT>
__device__ void block_merge(const BArgs& a, int ti, GT* G) {
  __shared__ int sh[4];
  const BTask& T = a.T[ti];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int e0 = T.ex[0], e1 = T.ex[1], e2 = T.ex[2];
  const int tot = e0 * e1 * e2;
  auto at = [&](int x, int y, int z) { return (z * e1 + y) * e0 + x; };
  const long long base = MODE == 1 ? a.first[ti] : 0;
  int* out = MODE == 2 ? a.scratch + 13LL * ti * a.cap : (T.d < 0 ? a.out_cells : a.out_faces);
  const int big = 0x7fffffff;
  int pos = 0;
  long long count = 0;
  for (;;) {
    int t0 = -1;
    while (pos < tot) {
      if (tid == 0) sh[0] = big;
      __syncthreads();
      const int idx = pos + tid;
      if (idx < tot && G[idx] >= 0) atomicMin(&sh[0], idx);
      __syncthreads();
      const int m = sh[0];
      __syncthreads();
      if (m != big) { t0 = m; break; }
      pos += nth;
    }
    if (t0 < 0) break;
    const int k = G[t0];
    const int r0 = t0 / e0, a0 = t0 - r0 * e0, b0 = r0 % e1, c0 = r0 / e1;
    if (tid == 0) { sh[1] = e0; sh[2] = e1; sh[3] = e2; }
    __syncthreads();
    for (int x = a0 + 1 + tid; x < e0; x += nth)
      if (G[at(x, b0, c0)] != k) atomicMin(&sh[1], x);
    __syncthreads();
    const int nx = sh[1] - a0;
    for (int y = b0 + 1 + tid; y < e1; y += nth) {
      bool ok = true;
      for (int i = 0; i < nx && ok; ++i) ok = G[at(a0 + i, y, c0)] == k;
      if (!ok) atomicMin(&sh[2], y);
    }
    __syncthreads();
    const int ny = sh[2] - b0;
    for (int z = c0 + 1 + (tid / 32); z < e2; z += nth / 32) {  // a warp per slab
      bool ok = true;
      for (int p = tid & 31; p < nx * ny && ok; p += 32) ok = G[at(a0 + p % nx, b0 + p / nx, z)] == k;
      if (!__all_sync(0xffffffffu, ok) && (tid & 31) == 0) atomicMin(&sh[3], z);
    }
    __syncthreads();
    const int nz = sh[3] - c0;
    for (int p = tid; p < nx * ny * nz; p += nth) {
      const int x = p % nx, yz = p / nx;
      G[at(a0 + x, b0 + yz % ny, c0 + yz / ny)] = -2;
    }
    if (MODE != 0 && tid == 0 && (MODE == 1 || count < a.cap)) {
      int* r = out + 13 * (base + count);
      const int o = T.transfer ? 4 : 0;  // transfer boxes: lo in the patch's ghosted frame
      if (T.transfer) transfer_row(a, T, k, r);
      else ghost_row(a, T, k, r);
      r[4] = a0 + o;
      r[5] = b0 + o;
      r[6] = a.dim == 3 ? c0 + o : c0;
      r[7] = nx;
      r[8] = ny;
      r[9] = nz;
    }
    __syncthreads();
    ++count;
    pos = t0 + 1;
  }
  if (MODE != 1 && tid == 0) a.cnt[ti] = count;
}

// one task per CTA, its label grid (ids of type ET) in shared memory (transfer
// tasks: followed by the owner grid)
template <class ET, int MODE>
__global__ void __launch_bounds__(kBoxThreads) k_box_tasks_smem(BArgs a, const int* list, int n) {
  extern __shared__ __align__(16) unsigned char sraw[];
  ET* sg = (ET*)sraw;
  if ((int)blockIdx.x >= n) return;
  const int ti = list[blockIdx.x];
  const BTask& T = a.T[ti];
  if (T.transfer) {
    const int tot = T.ex[0] * T.ex[1] * T.ex[2];
    transfer_fill(a, ti, sg, sg + (tot + 15) / 16 * 16);
  } else {
    ghost_scatter(a, ti, sg);
  }
  block_merge<MODE>(a, ti, sg);
}

// the one-pass rows of every task to their places in the cell and face lists
__global__ void k_box_compact(BArgs a, int nt) {
  const int ti = blockIdx.x;
  if (ti >= nt) return;
  const long long n = 13LL * a.cnt[ti];
  const int* src = a.scratch + 13LL * ti * a.cap;
  int* dst = (a.T[ti].d < 0 ? a.out_cells : a.out_faces) + 13LL * a.first[ti];
  for (long long i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// large tasks: labels into their global grids, then one warp per task merges
__global__ void k_box_label_global(BArgs a, const int* list, int n) {
  for (int k = blockIdx.y; k < n; k += gridDim.y) {
    const int ti = list[k];
    const BTask& T = a.T[ti];
    const int tot = T.ex[0] * T.ex[1] * T.ex[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
      const int id = label_of(a, T, t);
      if (id == -3) atomicMin(a.err, ((unsigned long long)ti << 32) | (unsigned long long)t);
      a.G[T.go + t] = id < 0 ? -1 : id;
    }
  }
}

template <int MODE>
__global__ void k_box_merge_global(BArgs a, const int* list, int n) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= n) return;  // the whole warp
  const int ti = list[k];
  warp_merge<MODE>(a, ti, a.G + a.T[ti].go);
}

// closure mask of the footprints of the listed transfer cell tasks
__global__ void k_closure_mask(BArgs a, const int* list, const long long* moff, int n, unsigned char* mask) {
  const int k = blockIdx.y;
  if (k >= n) return;
  const BTask& T = a.T[list[k]];
  const BPatch& P = a.P[T.q];
  int nc[3];
  for (int e = 0; e < 3; ++e) nc[e] = e < a.dim ? P.n[e] / 2 : 1;
  const int tot = nc[0] * nc[1] * nc[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    int c[3] = {t % nc[0], (t / nc[0]) % nc[1], t / (nc[0] * nc[1])};
    for (int e = 0; e < a.dim; ++e) c[e] += P.lo[e] / 2;
    mask[moff[k] + t] = closure_cell(a, T, c, LoopOwner{a, T}) ? 1 : 0;
  }
}

// ---- host tables

inline void patch_table(const amrmhd::Hierarchy& H, std::vector<BPatch>& out) {
  out.assign(H.p.size(), BPatch());
  for (size_t q = 0; q < H.p.size(); ++q) {
    for (int d = 0; d < 3; ++d) { out[q].lo[d] = H.p[q].lo[d]; out[q].n[d] = H.p[q].n[d]; out[q].ext[d] = H.p[q].ext[d]; }
    out[q].level = H.p[q].level;
  }
}

inline int shift_code(const int* s) { return (s[0] + 1) + 3 * (s[1] + 1) + 9 * (s[2] + 1); }

// the coarse candidates of patch q: its parents and their neighbours, ascending
inline std::vector<int> coarse_candidates(const amrmhd::Hierarchy& H, int q) {
  std::vector<int> cc;
  for (int par : H.parents[q]) {
    cc.push_back(par);
    for (const amrmhd::Nbr& x : H.nbr[par]) cc.push_back(x.q);
  }
  std::sort(cc.begin(), cc.end());
  cc.erase(std::unique(cc.begin(), cc.end()), cc.end());
  return cc;
}

// Ghost tasks of the patches of levels >= H.ghost_from: per patch its
// same-level neighbour entries (as listed) and the (coarse candidate, image)
// entries whose fine footprint meets the patch's ghosted box, in the host
// builder's order (candidate ascending, then z, y, x image).
inline void ghost_tasks(const amrmhd::Hierarchy& H, std::vector<BTask>& T, std::vector<int>& pairs) {
  const int dim = H.dim;
  for (int q = 0; q < (int)H.p.size(); ++q) {
    const amrmhd::HPatch& hp = H.p[q];
    if (hp.level < H.ghost_from) continue;
    const int l = hp.level;
    const int s0 = (int)pairs.size() / 2;
    for (const amrmhd::Nbr& x : H.nbr[q]) {
      pairs.push_back(x.q);
      pairs.push_back(shift_code(x.s));
    }
    const int s1 = (int)pairs.size() / 2;
    if (l > 0)
      for (int cq : coarse_candidates(H, q)) {
        const amrmhd::HPatch& C = H.p[cq];
        int wr[3];
        for (int e = 0; e < 3; ++e) wr[e] = (e < dim && H.per[e]) ? 1 : 0;
        for (int wz = -wr[2]; wz <= wr[2]; ++wz)
          for (int wy = -wr[1]; wy <= wr[1]; ++wy)
            for (int wx = -wr[0]; wx <= wr[0]; ++wx) {
              const int w[3] = {wx, wy, wz};
              bool meet = true;
              for (int e = 0; e < dim; ++e) {
                const int aux = w[e] * H.N(l, e);
                // footprint [2 lo - aux, 2 hi + 1 - aux) against the ghosted box [lo - 4, hi + 5)
                if (2 * C.hi[e] + 1 - aux <= hp.lo[e] - 4 || 2 * C.lo[e] - aux >= hp.hi[e] + 5) meet = false;
              }
              if (meet) {
                pairs.push_back(cq);
                pairs.push_back(shift_code(w));
              }
            }
      }
    const int p1 = (int)pairs.size() / 2;
    for (int d = -1; d < dim; ++d) {
      BTask t;
      t.q = q;
      t.d = d;
      t.s0 = s0;
      t.s1 = s1;
      t.p0 = s1;
      t.p1 = p1;
      t.touches = 0;
      t.transfer = 0;
      t.go = -1;
      for (int e = 0; e < 3; ++e) {
        t.ex[e] = e < dim ? hp.n[e] + 8 + (e == d ? 1 : 0) : 1;
        t.g0[e] = e < dim ? hp.lo[e] - 4 : 0;
        if (e < dim && !H.per[e] && (t.g0[e] < 0 || t.g0[e] + t.ex[e] - 1 > (e == d ? H.N(l, e) : H.N(l, e) - 1)))
          t.touches = 1;
      }
      T.push_back(t);
    }
  }
}

// Transfer tasks of level lf of Hn: per new patch the old level-lf (patch,
// shift) entries meeting the patch grown by 2 fine cells (old id ascending,
// then z, y, x shift) and its coarse candidates.
inline void transfer_tasks(const amrmhd::Hierarchy& Hn, const amrmhd::Hierarchy& Ho, int lf, std::vector<BTask>& T,
                           std::vector<int>& pairs, std::vector<int>& ids) {
  const int dim = Hn.dim;
  const int B = 16;  // bins of 16 fine cells over the old level
  int N[3], nb[3];
  for (int e = 0; e < 3; ++e) {
    N[e] = Hn.N(lf, e);
    nb[e] = e < dim ? (N[e] + B - 1) / B : 1;
  }
  std::vector<std::vector<int>> bins((size_t)nb[0] * nb[1] * nb[2]);
  if (Ho.nlev > lf)
    for (int oq : Ho.level_patches[lf]) {
      int b0[3], b1[3];
      for (int e = 0; e < 3; ++e) {
        b0[e] = e < dim ? Ho.p[oq].lo[e] / B : 0;
        b1[e] = e < dim ? (Ho.p[oq].hi[e] - 1) / B : 0;
      }
      for (int z = b0[2]; z <= b1[2]; ++z)
        for (int y = b0[1]; y <= b1[1]; ++y)
          for (int x = b0[0]; x <= b1[0]; ++x) bins[((size_t)z * nb[1] + y) * nb[0] + x].push_back(oq);
    }
  int wr[3];
  for (int e = 0; e < 3; ++e) wr[e] = (e < dim && Hn.per[e]) ? 1 : 0;
  for (int q : Hn.level_patches[lf]) {
    const amrmhd::HPatch& hp = Hn.p[q];
    std::vector<int> oc;
    for (int sz = -wr[2]; sz <= wr[2]; ++sz)
      for (int sy = -wr[1]; sy <= wr[1]; ++sy)
        for (int sx = -wr[0]; sx <= wr[0]; ++sx) {
          const int sh[3] = {sx, sy, sz};
          int a0[3] = {0, 0, 0}, a1[3] = {0, 0, 0};
          bool empty = false;
          for (int e = 0; e < dim; ++e) {
            const int lo = std::max(hp.lo[e] - 2 - sh[e] * N[e], 0), hi = std::min(hp.hi[e] + 2 - sh[e] * N[e], N[e]);
            if (hi <= lo) { empty = true; break; }
            a0[e] = lo / B;
            a1[e] = (hi - 1) / B;
          }
          if (empty) continue;
          for (int z = a0[2]; z <= a1[2]; ++z)
            for (int y = a0[1]; y <= a1[1]; ++y)
              for (int x = a0[0]; x <= a1[0]; ++x)
                for (int oq : bins[((size_t)z * nb[1] + y) * nb[0] + x]) oc.push_back(oq);
        }
    std::sort(oc.begin(), oc.end());
    oc.erase(std::unique(oc.begin(), oc.end()), oc.end());
    const int s0 = (int)pairs.size() / 2;
    for (int oq : oc) {
      const amrmhd::HPatch& O = Ho.p[oq];
      for (int sz = -wr[2]; sz <= wr[2]; ++sz)
        for (int sy = -wr[1]; sy <= wr[1]; ++sy)
          for (int sx = -wr[0]; sx <= wr[0]; ++sx) {
            const int sh[3] = {sx, sy, sz};
            bool meet = true;
            for (int e = 0; e < dim; ++e)
              if (O.hi[e] + sh[e] * N[e] <= hp.lo[e] - 2 || O.lo[e] + sh[e] * N[e] >= hp.hi[e] + 2) meet = false;
            if (meet) {
              pairs.push_back(oq);
              pairs.push_back(shift_code(sh));
            }
          }
    }
    const int s1 = (int)pairs.size() / 2;
    const std::vector<int> cc = coarse_candidates(Hn, q);
    const int p0 = (int)ids.size();
    ids.insert(ids.end(), cc.begin(), cc.end());
    const int p1 = (int)ids.size();
    for (int d = -1; d < dim; ++d) {
      BTask t;
      t.q = q;
      t.d = d;
      t.s0 = s0;
      t.s1 = s1;
      t.p0 = p0;
      t.p1 = p1;
      t.touches = 0;
      t.transfer = 1;
      t.go = -1;
      for (int e = 0; e < 3; ++e) {
        t.ex[e] = e < dim ? hp.n[e] + (e == d ? 1 : 0) : 1;
        t.g0[e] = e < dim ? hp.lo[e] : 0;
      }
      T.push_back(t);
    }
  }
}

// the largest label id a task can produce
inline long long max_id(const BTask& t) {
  const long long ns = t.s1 - t.s0, np = t.p1 - t.p0;
  return t.transfer ? ns + 8 * np : ns + np + 27;
}

}  // namespace amrbx

namespace amrapi {

namespace {

long long box_now_us() {
  return std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// AMRMHD_REGRID_TRACE set in the environment: the builder's phases on stderr
bool box_trace() {
  static const bool on = std::getenv("AMRMHD_REGRID_TRACE") != nullptr;
  return on;
}

constexpr size_t kBoxSmem = 200 * 1024;  // label grid bytes of a task labelled in shared memory

// Runs box tasks (ghost or transfer) on the device and returns the boxes of the
// cell tasks and of the face tasks in task order; with closure (transfer), the
// closure mask of every cell task's coarse footprint. *bad gets the first task
// and position without a source (or -1).
amrmhd_status run_box_tasks(amrmhd_ctx* ctx, cudaStream_t st, const amrmhd::Hierarchy& H,
                            const std::vector<amrbx::BPatch>& P, const std::vector<amrbx::BPatch>* PO, int have_old,
                            std::vector<amrbx::BTask>& T, const std::vector<int>& pairs, const std::vector<int>& ids,
                            std::vector<int32_t>& cells, std::vector<int32_t>& faces, std::vector<uint8_t>* closure,
                            std::vector<long long>* closure_off, long long* bad, const char* what) {
  using namespace amrbx;
  cells.clear();
  faces.clear();
  *bad = -1;
  const int nt = (int)T.size();
  if (!nt) return AMRMHD_OK;
  const long long tt0 = box_now_us();
  // tasks labelled in shared memory with 8-bit ids, with 16-bit ids, and the
  // large ones in global memory
  std::vector<int> s8, s16, large;
  long long gtot = 0, need8 = 1, need16 = 1;
  for (int i = 0; i < nt; ++i) {
    const long long tot = (long long)T[i].ex[0] * T[i].ex[1] * T[i].ex[2];
    long long need = tot;
    if (T[i].transfer) {  // the owner grid over the patch grown by 2 fine cells
      long long gw = 1;
      for (int e = 0; e < H.dim; ++e) gw *= P[T[i].q].n[e] + 4;
      need = (tot + 15) / 16 * 16 + gw;
    }
    const long long mid = std::max<long long>(max_id(T[i]), T[i].s1 - T[i].s0);
    if (mid < 127 && need <= (long long)kBoxSmem) {
      s8.push_back(i);
      need8 = std::max(need8, need);
    } else if (mid < 32767 && 2 * need <= (long long)kBoxSmem) {
      s16.push_back(i);
      need16 = std::max(need16, need);
    } else {
      large.push_back(i);
      T[i].go = gtot;
      gtot += tot;
    }
  }
  std::vector<int> ctask;
  std::vector<long long> moff;
  long long mtot = 0;
  if (closure)
    for (int i = 0; i < nt; ++i)
      if (T[i].d < 0) {
        ctask.push_back(i);
        moff.push_back(mtot);
        long long v = 1;
        for (int e = 0; e < H.dim; ++e) v *= P[T[i].q].n[e] / 2;
        mtot += v;
      }
  const int cap = 256;  // rows per task kept by the one-pass merge
  std::vector<char> img;
  auto put = [&](const void* src, size_t bytes) {
    const size_t o = (img.size() + 255) / 256 * 256;
    img.resize(o + bytes);
    if (bytes) std::memcpy(img.data() + o, src, bytes);
    return o;
  };
  const size_t oP = put(P.data(), sizeof(BPatch) * P.size()),
               oPO = put(PO ? PO->data() : nullptr, sizeof(BPatch) * (PO ? PO->size() : 0)),
               oT = put(T.data(), sizeof(BTask) * nt), oPr = put(pairs.data(), sizeof(int) * pairs.size()),
               oI = put(ids.data(), sizeof(int) * ids.size()), o8 = put(s8.data(), sizeof(int) * s8.size()),
               o16 = put(s16.data(), sizeof(int) * s16.size()), oL = put(large.data(), sizeof(int) * large.size()),
               oCT = put(ctask.data(), sizeof(int) * ctask.size()), oMO = put(moff.data(), sizeof(long long) * moff.size());
  const size_t in_bytes = img.size();
  size_t o = (in_bytes + 255) / 256 * 256;
  auto reserve = [&](size_t bytes) { const size_t r = o; o = (o + bytes + 255) / 256 * 256; return r; };
  const size_t oG = reserve(sizeof(int) * gtot), oCnt = reserve(sizeof(long long) * nt),
               oFirst = reserve(sizeof(long long) * nt), oErr = reserve(sizeof(unsigned long long)),
               oMask = reserve((size_t)mtot), oScr = reserve(sizeof(int) * 13 * (size_t)cap * nt);
  // scratch from the stream-ordered allocator (no device-wide synchronisation on free)
  char* dev = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dev, o, st);
  if (e != cudaSuccess) return fail(ctx, AMRMHD_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  int* dout = nullptr;
  auto done = [&](amrmhd_status s, const std::string& m) {
    cudaFreeAsync(dev, st);
    if (dout) cudaFreeAsync(dout, st);
    return s == AMRMHD_OK ? s : fail(ctx, s, m);
  };
  e = cudaMemcpyAsync(dev, img.data(), in_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev + oErr, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  BArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dim = H.dim;
  for (int d = 0; d < 3; ++d) {
    a.base[d] = H.base[d];
    a.per[d] = H.per[d] ? 1 : 0;
    a.bc[d][0] = H.bc[d][0];
    a.bc[d][1] = H.bc[d][1];
  }
  a.P = (const BPatch*)(dev + oP);
  a.PO = (const BPatch*)(dev + oPO);
  a.have_old = have_old;
  a.T = (const BTask*)(dev + oT);
  a.pairs = (const int*)(dev + oPr);
  a.ids = (const int*)(dev + oI);
  a.G = (int*)(dev + oG);
  a.cnt = (long long*)(dev + oCnt);
  a.first = (const long long*)(dev + oFirst);
  a.err = (unsigned long long*)(dev + oErr);
  a.scratch = (int*)(dev + oScr);
  a.cap = cap;
  // the kernels' shared-memory limit, once per process (thread-safe static initialisation)
  static const bool attr = [] {
    for (auto f : {k_box_tasks_smem<signed char, 0>, k_box_tasks_smem<signed char, 1>, k_box_tasks_smem<signed char, 2>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBoxSmem);
    for (auto f : {k_box_tasks_smem<short, 0>, k_box_tasks_smem<short, 1>, k_box_tasks_smem<short, 2>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBoxSmem);
    return true;
  }();
  (void)attr;
  long long lmax = 0;
  for (int i : large) lmax = std::max(lmax, (long long)T[i].ex[0] * T[i].ex[1] * T[i].ex[2]);
  const dim3 lg((unsigned)std::min<long long>((lmax + 255) / 256, 64), (unsigned)std::min<size_t>(large.size(), 65535));
  const int WPB = 4;
  const size_t sm8 = (size_t)need8, sm16 = 2 * (size_t)need16;
  auto launch = [&](auto mode) {
    constexpr int M = decltype(mode)::value;
    if (!s8.empty())
      k_box_tasks_smem<signed char, M><<<(unsigned)s8.size(), kBoxThreads, sm8, st>>>(a, (const int*)(dev + o8), (int)s8.size());
    if (!s16.empty())
      k_box_tasks_smem<short, M><<<(unsigned)s16.size(), kBoxThreads, sm16, st>>>(a, (const int*)(dev + o16), (int)s16.size());
    if (!large.empty()) {
      k_box_label_global<<<lg, 256, 0, st>>>(a, (const int*)(dev + oL), (int)large.size());
      k_box_merge_global<M><<<(unsigned)((large.size() + WPB - 1) / WPB), 32 * WPB, 0, st>>>(a, (const int*)(dev + oL), (int)large.size());
    }
    ctx->launches += (s8.empty() ? 0 : 1) + (s16.empty() ? 0 : 1) + (large.empty() ? 0 : 2);
  };
  // one pass: count every task's boxes and keep up to cap of them
  const long long tt1 = box_now_us();
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (box_trace()) {
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], st);
  }
  launch(std::integral_constant<int, 2>());
  if (box_trace()) cudaEventRecord(ev[1], st);
  if (closure && mtot) {
    k_closure_mask<<<dim3(8, (unsigned)ctask.size()), 256, 0, st>>>(a, (const int*)(dev + oCT),
                                                                   (const long long*)(dev + oMO), (int)ctask.size(),
                                                                   (unsigned char*)(dev + oMask));
    ctx->launches += 1;
  }
  std::vector<long long> cnt(nt);
  unsigned long long err = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), a.cnt, sizeof(long long) * nt, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, a.err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && closure) {
    closure->resize((size_t)mtot);
    if (mtot) e = cudaMemcpyAsync(closure->data(), dev + oMask, (size_t)mtot, cudaMemcpyDeviceToHost, st);
    *closure_off = moff;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const long long tt2 = box_now_us();
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string(what) + " (count): " + cudaGetErrorString(e));
  if (err != ~0ull) {
    *bad = (long long)err;
    return done(AMRMHD_OK, "");
  }
  std::vector<long long> first(nt);
  long long nc = 0, nf = 0;
  bool over = false;
  for (int i = 0; i < nt; ++i) {
    long long& acc = T[i].d < 0 ? nc : nf;
    first[i] = acc;
    acc += cnt[i];
    over = over || cnt[i] > cap;
  }
  e = cudaMallocAsync((void**)&dout, sizeof(int) * 13 * std::max<long long>(nc + nf, 1), st);
  if (e != cudaSuccess) { dout = nullptr; return done(AMRMHD_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e)); }
  a.out_cells = dout;
  a.out_faces = dout + 13 * nc;
  e = cudaMemcpyAsync(dev + oFirst, first.data(), sizeof(long long) * nt, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  if (over) {
    // a task with more boxes than the one-pass rows: label again and write every box in place
    launch(std::integral_constant<int, 1>());
  } else {
    k_box_compact<<<nt, 128, 0, st>>>(a, nt);
    ctx->launches += 1;
  }
  cells.resize(13 * (size_t)nc);
  faces.resize(13 * (size_t)nf);
  e = cudaGetLastError();
  if (e == cudaSuccess && nc) e = cudaMemcpyAsync(cells.data(), a.out_cells, sizeof(int) * 13 * nc, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && nf) e = cudaMemcpyAsync(faces.data(), a.out_faces, sizeof(int) * 13 * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(AMRMHD_ECUDA, std::string(what) + " (emit): " + cudaGetErrorString(e));
  if (box_trace()) {
    float kms = 0.f;
    cudaEventElapsedTime(&kms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    std::fprintf(stderr, "amrmhd %s: %d tasks (%zu + %zu in shared memory, %zu global): host tables %lld us, "
                 "label and merge to sync %lld us (kernels %.0f us), placement to sync %lld us, %lld + %lld boxes\n",
                 what, nt, s8.size(), s16.size(), large.size(), tt1 - tt0, tt2 - tt1, 1e3 * kms, box_now_us() - tt2,
                 nc, nf);
  }
  return done(AMRMHD_OK, "");
}

}  // namespace

// The ghost-fill boxes of the patches of levels >= H.ghost_from, built on the
// device into H.ghost_box_cells and H.ghost_box_faces (host copies: the bind
// step turns them into fill records).
amrmhd_status device_ghost_boxes(amrmhd_ctx* ctx) {
  using namespace amrbx;
  amrmhd::Hierarchy& H = ctx->H;
  H.ghost_rows_ready = false;
  std::vector<BPatch> P;
  std::vector<BTask> T;
  std::vector<int> pairs, ids;
  long long bad = -1;
  patch_table(H, P);
  ghost_tasks(H, T, pairs);
  amrmhd_status s = run_box_tasks(ctx, ctx->stream, H, P, nullptr, 0, T, pairs, ids, H.ghost_box_cells,
                                  H.ghost_box_faces, nullptr, nullptr, &bad, "ghost maps");
  if (s != AMRMHD_OK || bad < 0) return s;
  // a ghost position without a source: the host builder's messages
  const BTask& t = T[bad >> 32];
  int x[3];
  decode(t, bad & 0xffffffffll, x);
  const int g[3] = {t.g0[0] + x[0], t.g0[1] + x[1], t.g0[2] + x[2]};
  H.ghost_box_cells.clear();
  H.ghost_box_faces.clear();
  if (H.p[t.q].level == 0)
    return fail(ctx, AMRMHD_EINVAL, t.d < 0 ? "level-0 ghost cell without a source" : "level-0 ghost face without a source");
  return fail(ctx, AMRMHD_ENEST,
              t.d < 0 ? "no parent-level source for the ghost cell (" + std::to_string(g[0]) + ", " + std::to_string(g[1]) +
                            ", " + std::to_string(g[2]) + ") of patch " + std::to_string(t.q)
                      : "no parent-level source for the ghost face (" + std::to_string(t.d) + "; " +
                            std::to_string(g[0]) + ", " + std::to_string(g[1]) + ", " + std::to_string(g[2]) +
                            ") of patch " + std::to_string(t.q));
}

// The transfer maps of level lf of the new hierarchy Hn from the old hierarchy
// Ho, built on the device: the rows of amrmhd::transfer_maps (the cell and face
// boxes of every new patch, and the closure rows).
amrmhd_status device_transfer_maps(amrmhd_ctx* ctx, const amrmhd::Hierarchy& Hn, const amrmhd::Hierarchy& Ho, int lf,
                                   cudaStream_t st, std::vector<int32_t>& cells, std::vector<int32_t>& faces,
                                   std::vector<int32_t>& closure) {
  using namespace amrbx;
  std::vector<BPatch> P, PO;
  std::vector<BTask> T;
  std::vector<int> pairs, ids;
  long long bad = -1;
  patch_table(Hn, P);
  patch_table(Ho, PO);
  transfer_tasks(Hn, Ho, lf, T, pairs, ids);
  std::vector<uint8_t> mask;
  std::vector<long long> moff;
  amrmhd_status s = run_box_tasks(ctx, st, Hn, P, &PO, Ho.nlev > lf, T, pairs, ids, cells, faces, &mask, &moff, &bad,
                                  "transfer maps");
  if (s != AMRMHD_OK) return s;
  if (bad >= 0) return fail(ctx, AMRMHD_EINVAL, "regrid: transfer map without a source");
  closure.clear();
  int k = 0;
  for (const BTask& t : T) {
    if (t.d >= 0) continue;
    const amrmhd::HPatch& hp = Hn.p[t.q];
    int nc[3];
    for (int e = 0; e < 3; ++e) nc[e] = e < Hn.dim ? hp.n[e] / 2 : 1;
    const uint8_t* m = mask.data() + moff[k++];
    for (int z = 0; z < nc[2]; ++z)
      for (int y = 0; y < nc[1]; ++y)
        for (int x = 0; x < nc[0]; ++x, ++m)
          if (*m) {
            closure.push_back(t.q);
            closure.push_back(Hn.loc(t.q, hp.lo[0] + 2 * x, hp.lo[1] + 2 * y, Hn.dim == 3 ? hp.lo[2] + 2 * z : 0));
          }
  }
  return AMRMHD_OK;
}

}  // namespace amrapi
