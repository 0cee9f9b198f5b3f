// Oracle: plain, slow FP64 CPU implementation of the AMR ideal-MHD advance of
// every patch on every refinement level with extended ghost zones.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the CPU-baseline
// leg of the benchmark may build, load or call this code; the product path
// (the CUDA library and its binding) never does, and shares no code with it.
//
// What it computes, and where that comes from:
//  * Patches, levels, ratio R = 2, nesting of every level above 0 inside the
//    next coarser one (Sec. 2).
//  * Levels advance in the recursive order 0,1,2,2,1,2,2 with the operations
//    (P)rolongate, (A)dvance, (S)ynchronize = reflux, (R)estrict (Sec. 4).
//  * Extended ghost zones decouple the levels (Abstract, Sec. 1): the ghost
//    shell of width 4 = R x reach 2 of a level above 0 is prolonged once per
//    parent step from the parent's state at the start of that step; sub-step 1
//    updates the interior plus 2 ghost layers, sub-step 2 the interior.
//    Same-level ghosts are refreshed before every sub-step (reading R7).
//  * The per-cell numerics (not in the paper) follow readings R1-R5 in
//    mhd_core.hpp; prolongation, reflux, restriction and CFL follow R6-R9.
//
// Representation: unlike the patch-based product path, each level is one
// array over the whole periodic domain at that level's resolution. The
// level's region is the union of its patch interiors; a cell's ghost value in
// any patch is either another patch's interior value or a prolonged value, both
// of which are the single global value here, so the union of all patches'
// ghosted boxes behaves exactly like the band of width 4 around the region.
// This keeps the oracle free of any patch bookkeeping.
//
// Boundaries: periodic, or (per dimension) a fixed inflow state on one side
// and zero-gradient outflow on the other (reading R17). A non-periodic
// dimension carries a margin of 4 cells outside the domain, filled by the
// boundary conditions before every sub-step.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ad.hpp"
#include "mhd_core.hpp"

namespace oracle {

static const int G = 4;  // ghost width

struct Patch { int level, lo[3], hi[3]; };

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2 };

// Value type R: double for the forward oracle; the differentiation types of
// oracle/adjoint.cpp (a reverse-mode tape entry, a forward-mode tangent) for the
// adjoint pins.
template <class R> struct LevelT {
  int N[3] = {1, 1, 1};  // cells per dimension
  int M[3] = {0, 0, 0};  // margin (4 in a non-periodic dimension)
  int X[3] = {1, 1, 1};  // storage extent: N (periodic) or N + 2M + 1
  bool per[3] = {true, true, true};
  double dx[3] = {1, 1, 1}, idx[3] = {1, 1, 1};
  size_t ncell = 0;
  std::vector<R> u[NFIELD];      // cell fields and face fields, index (k*Ny + j)*Nx + i
  std::vector<R> start[NFIELD];  // state at the start of the latest sub-step
  std::vector<int8_t> dist;           // Chebyshev distance to the region, -1 if > 4
  std::vector<int8_t> cov;            // cell covered by the next finer level
  // work arrays
  std::vector<R> W[NFIELD], Wh[NFIELD], S[3][NFIELD], ref[3], F[3][NFIELD], E[3];
  std::vector<int8_t> tmask;          // target distance map used by one advance
  // registers of this level's C/F boundary with its parent (indexed on the parent level)
  std::vector<R> rflux[3][NFIELD];    // per parent face: fine time-integrated flux (S1 + S2)
  std::vector<R> rcoarse[3][NFIELD];  // per parent face: coarse time-integrated flux C
  std::vector<R> remf[3], remfc[3];   // the same for the EMF of parent edges
  std::vector<int8_t> cf_face[3], cf_edge[3];
};

template <class R> struct SimT {
  int dim = 2;
  int base[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  double gamma = 5.0 / 3.0, cfl = 0.4;
  double eps = 1e-12;
  int nlev = 1;
  std::vector<Patch> patches;
  std::vector<LevelT<R>> lev;
  long long cell_updates = 0;
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  double inflow[NFIELD] = {0, 0, 0, 0, 0, 0, 0, 0};
  int flags = 0;  // test-only switches: bit 0 skips the cell reflux (a planted
                  // mistake); bit 1 replaces minmod by the unlimited centred slope;
                  // bit 2 plants an off-by-one in the high-side boundary faces;
                  // bit 3 skips the divergence-free closure of the regrid;
                  // bits 4-6 plant mistakes in the half-step predictor (controls
                  // of its pins): bit 4 p div v for gamma p div v in the pressure
                  // row; bit 5 the sign of the B_t dv_z/dz terms of the induction
                  // rows flipped; bit 6 the dp/dz term of the z-momentum row
                  // dropped (bits 5 and 6 touch the z direction only)
};

// ---------------------------------------------------------------- indexing
static inline int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
template <class LV> static inline int mapi(const LV& L, int d, int i) { return L.per[d] ? wrapi(i, L.N[d]) : i + L.M[d]; }
template <class LV> static inline size_t at(const LV& L, int i, int j, int k) {
  return ((size_t)mapi(L, 2, k) * L.X[1] + mapi(L, 1, j)) * L.X[0] + mapi(L, 0, i);
}
// cell (i,j,k) stored (margin included)?
template <class LV> static inline bool in_storage(const LV& L, int i, int j, int k) {
  const int o[3] = {i, j, k};
  for (int d = 0; d < 3; ++d)
    if (!L.per[d] && (o[d] < -L.M[d] || o[d] >= L.N[d] + L.M[d])) return false;
  return true;
}
template <class LV> static inline bool in_domain(const LV& L, int i, int j, int k) {
  const int o[3] = {i, j, k};
  for (int d = 0; d < 3; ++d)
    if (!L.per[d] && (o[d] < 0 || o[d] >= L.N[d])) return false;
  return true;
}
template <class LV> static inline size_t atd(const LV& L, int i, int j, int k, int d, int s) {
  int o[3] = {i, j, k};
  o[d] += s;
  return at(L, o[0], o[1], o[2]);
}
// cells of the domain
template <class LV, class F> static void for_cells(const LV& L, F f) {
  for (int k = 0; k < L.N[2]; ++k)
    for (int j = 0; j < L.N[1]; ++j)
      for (int i = 0; i < L.N[0]; ++i) f(i, j, k);
}
// cells of the domain and of the margins
template <class LV, class F> static void for_all(const LV& L, F f) {
  for (int k = -L.M[2]; k < L.N[2] + L.M[2]; ++k)
    for (int j = -L.M[1]; j < L.N[1] + L.M[1]; ++j)
      for (int i = -L.M[0]; i < L.N[0] + L.M[0]; ++i) f(i, j, k);
}
// positions of the d-faces of the domain (the face at the high end of a
// non-periodic dimension included; periodic faces wrap)
template <class LV, class F> static void for_face_pos(const LV& L, int d, F f) {
  int hi[3] = {L.N[0], L.N[1], L.N[2]};
  if (!L.per[d]) hi[d] += 1;
  for (int k = 0; k < hi[2]; ++k)
    for (int j = 0; j < hi[1]; ++j)
      for (int i = 0; i < hi[0]; ++i) f(i, j, k);
}
// positions of the c-edges of the domain
template <class LV, class F> static void for_edge_pos(const LV& L, int c, F f) {
  int hi[3] = {L.N[0], L.N[1], L.N[2]};
  for (int e = 0; e < 3; ++e)
    if (e != c && !L.per[e]) hi[e] += 1;
  for (int k = 0; k < hi[2]; ++k)
    for (int j = 0; j < hi[1]; ++j)
      for (int i = 0; i < hi[0]; ++i) f(i, j, k);
}

// Cell-field list: in 3D rho, m, E; in 2D also Bz, which is cell-centred and
// advanced by its fluxes there.
template <class R> static int cell_fields(const SimT<R>& S, int* f) {
  int n = 0;
  f[n++] = RHO; f[n++] = MX; f[n++] = MY; f[n++] = MZ; f[n++] = EN;
  if (S.dim == 2) f[n++] = BZ;
  return n;
}
template <class R> static inline bool is_face_field(const SimT<R>& S, int f) { return f == BX || f == BY || (f == BZ && S.dim == 3); }

// Chebyshev dilation of a distance map (0 = seed) up to 4, with periodic wrap.
template <class R> static void dilate(const SimT<R>& S, const LevelT<R>& L, std::vector<int8_t>& d) {
  const int kz = S.dim == 3 ? 1 : 0;
  for (int r = 1; r <= G; ++r) {
    std::vector<int8_t> nd = d;
    for_all(L, [&](int i, int j, int k) {
      size_t q = at(L, i, j, k);
      if (d[q] >= 0) return;
      for (int c = -kz; c <= kz; ++c)
        for (int b = -1; b <= 1; ++b)
          for (int a = -1; a <= 1; ++a)
            if (in_storage(L, i + a, j + b, k + c) && d[at(L, i + a, j + b, k + c)] == r - 1) {
              nd[q] = (int8_t)r;
              return;
            }
    });
    d.swap(nd);
  }
}

// ---------------------------------------------------------------- setup
template <class R> static int validate_and_build(SimT<R>& S) {
  // Sec. 2: levels l>0 nested in level l-1 with ratio 2; patches aligned to
  // parent cells; no same-level overlap; level 0 tiles the domain.
  S.lev.assign(S.nlev, LevelT<R>());
  for (int l = 0; l < S.nlev; ++l) {
    LevelT<R>& L = S.lev[l];
    for (int d = 0; d < 3; ++d) {
      L.N[d] = d < S.dim ? (S.base[d] << l) : 1;
      L.dx[d] = d < S.dim ? (S.hi[d] - S.lo[d]) / L.N[d] : 1.0;
      L.idx[d] = 1.0 / L.dx[d];
      L.per[d] = d >= S.dim || S.bc[d][0] == BC_PERIODIC;
      L.M[d] = L.per[d] ? 0 : G;
      L.X[d] = L.per[d] ? L.N[d] : L.N[d] + 2 * G + 1;
    }
    L.ncell = (size_t)L.X[0] * L.X[1] * L.X[2];
    for (int f = 0; f < NFIELD; ++f) { L.u[f].assign(L.ncell, 0.0); L.start[f].assign(L.ncell, 0.0); }
    L.dist.assign(L.ncell, -1);
    L.cov.assign(L.ncell, 0);
  }
  for (const Patch& p : S.patches) {
    if (p.level < 0 || p.level >= S.nlev) return -1;
    LevelT<R>& L = S.lev[p.level];
    for (int d = 0; d < 3; ++d) {
      int lo = p.lo[d], hi = p.hi[d];
      if (d >= S.dim) { if (lo != 0 || hi != 1) return -1; continue; }
      if (lo < 0 || hi > L.N[d] || hi <= lo) return -1;
      if (p.level > 0 && ((lo & 1) || (hi & 1))) return -1;
    }
    for (int k = p.lo[2]; k < p.hi[2]; ++k)
      for (int j = p.lo[1]; j < p.hi[1]; ++j)
        for (int i = p.lo[0]; i < p.hi[0]; ++i) {
          size_t q = at(L, i, j, k);
          if (L.dist[q] == 0) return -3;  // same-level overlap
          L.dist[q] = 0;
        }
  }
  {
    bool tiled = true;
    for_cells(S.lev[0], [&](int i, int j, int k) {
      if (S.lev[0].dist[at(S.lev[0], i, j, k)] != 0) tiled = false;
    });
    if (!tiled) return -1;  // level 0 must tile the domain
  }
  for (int l = 1; l < S.nlev; ++l) {
    LevelT<R>& F = S.lev[l];
    LevelT<R>& C = S.lev[l - 1];
    // covered coarse cells and proper nesting (R11): every coarse cell within
    // Chebyshev distance 3 of a covered cell lies in the coarse region.
    for_cells(F, [&](int i, int j, int k) {
      if (F.dist[at(F, i, j, k)] == 0) C.cov[at(C, i >> 1, j >> 1, k >> 1)] = 1;
    });
    bool ok = true;
    const int kz = S.dim == 3 ? 3 : 0;
    for_cells(C, [&](int i, int j, int k) {
      if (!C.cov[at(C, i, j, k)]) return;
      for (int c = -kz; c <= kz; ++c)
        for (int b = -3; b <= 3; ++b)
          for (int a = -3; a <= 3; ++a)
            if (in_domain(C, i + a, j + b, k + c) && C.dist[at(C, i + a, j + b, k + c)] != 0) ok = false;
    });
    if (!ok) return -2;
  }
  for (int l = 0; l < S.nlev; ++l) dilate(S, S.lev[l], S.lev[l].dist);
  // C/F faces and edges of level l (>0) on its parent level.
  for (int l = 1; l < S.nlev; ++l) {
    LevelT<R>& F = S.lev[l];
    LevelT<R>& C = S.lev[l - 1];
    for (int d = 0; d < 3; ++d) {
      F.cf_face[d].assign(C.ncell, 0);
      F.cf_edge[d].assign(C.ncell, 0);
      for (int f = 0; f < NFIELD; ++f) { F.rflux[d][f].assign(C.ncell, 0.0); F.rcoarse[d][f].assign(C.ncell, 0.0); }
      F.remf[d].assign(C.ncell, 0.0);
      F.remfc[d].assign(C.ncell, 0.0);
    }
    // a C/F face lies between a covered and an uncovered cell of the domain; a
    // C/F edge has 1..3 covered cells around it (cells outside the domain count
    // as uncovered)
    for (int d = 0; d < S.dim; ++d)
      for_face_pos(C, d, [&](int i, int j, int k) {
        int m[3] = {i, j, k};
        m[d] -= 1;
        if (!in_domain(C, i, j, k) || !in_domain(C, m[0], m[1], m[2])) return;
        size_t q = at(C, i, j, k);
        if (C.cov[at(C, m[0], m[1], m[2])] != C.cov[q]) F.cf_face[d][q] = 1;
      });
    for (int c = 0; c < 3; ++c) {
      if (S.dim == 2 && c != 2) continue;
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      for_edge_pos(C, c, [&](int i, int j, int k) {
        int n = 0;
        for (int sb = -1; sb <= 0; ++sb)
          for (int sa = -1; sa <= 0; ++sa) {
            int p[3] = {i, j, k};
            p[a] += sa;
            p[b] += sb;
            if (in_domain(C, p[0], p[1], p[2])) n += C.cov[at(C, p[0], p[1], p[2])];
          }
        if (n >= 1 && n <= 3) F.cf_edge[c][at(C, i, j, k)] = 1;
      });
    }
  }
  return 0;
}

template <class R> static void alloc_work(const SimT<R>& S, LevelT<R>& L) {
  if (L.W[0].size() == L.ncell) return;
  for (int f = 0; f < NFIELD; ++f) {
    L.W[f].assign(L.ncell, 0.0); L.Wh[f].assign(L.ncell, 0.0);
    for (int d = 0; d < 3; ++d) { L.S[d][f].assign(L.ncell, 0.0); L.F[d][f].assign(L.ncell, 0.0); }
  }
  for (int d = 0; d < 3; ++d) { L.ref[d].assign(L.ncell, 0.0); L.E[d].assign(L.ncell, 0.0); }
  (void)S;
}

// ---------------------------------------------------------------- advance
template <class R> static inline void cell_bc(const SimT<R>& S, const LevelT<R>& L, int i, int j, int k, R* bc) {
  size_t q = at(L, i, j, k);
  bc[0] = 0.5 * (L.u[BX][q] + L.u[BX][atd(L, i, j, k, 0, 1)]);
  bc[1] = 0.5 * (L.u[BY][q] + L.u[BY][atd(L, i, j, k, 1, 1)]);
  bc[2] = S.dim == 3 ? 0.5 * (L.u[BZ][q] + L.u[BZ][atd(L, i, j, k, 2, 1)]) : L.u[BZ][q];
}

template <class R> static void prim_at(const SimT<R>& S, const LevelT<R>& L, int i, int j, int k, R* w) {
  size_t q = at(L, i, j, k);
  R u[5] = {L.u[RHO][q], L.u[MX][q], L.u[MY][q], L.u[MZ][q], L.u[EN][q]};
  R bc[3];
  cell_bc(S, L, i, j, k, bc);
  cons_to_prim<R>(u, bc, R(S.gamma - 1.0), w);
}

// One level update with time step dt of the target cell set T = {dist_t <= 0}
// where dist_t is L.tmask (Chebyshev distance to the target, -1 beyond 4):
// W on T+2, predictor on T+1, fluxes between T+1 cells, EMFs at edges whose 4
// cells are in T+1, then cells of T and faces touching T are updated.
template <class R> static void advance_masked(SimT<R>& S, LevelT<R>& L, double dt) {
  alloc_work(S, L);
  const int dim = S.dim;
  const std::vector<int8_t>& tm = L.tmask;
  auto in = [&](size_t q, int r) { return tm[q] >= 0 && tm[q] <= r; };
  // the same test for a cell given by coordinates (false outside the storage)
  auto inc = [&](int i, int j, int k, int r) { return in_storage(L, i, j, k) && in(at(L, i, j, k), r); };
  const double gamma = S.gamma;
  // primitives
  for_all(L, [&](int i, int j, int k) {
    size_t q = at(L, i, j, k);
    if (!in(q, 2)) return;
    R w[8];
    prim_at(S, L, i, j, k, w);
    for (int f = 0; f < 8; ++f) L.W[f][q] = w[f];
  });
  // slopes and half-step predictor (R1, R2)
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = 0.5 * dt * L.idx[d];
  for_all(L, [&](int i, int j, int k) {
    size_t q = at(L, i, j, k);
    if (!in(q, 1)) return;
    R w[8], s[3][8];
    for (int f = 0; f < 8; ++f) w[f] = L.W[f][q];
    for (int d = 0; d < dim; ++d) {
      size_t qm = atd(L, i, j, k, d, -1), qp = atd(L, i, j, k, d, 1);
      for (int f = 0; f < 8; ++f) {
        if (f == BX + d) s[d][f] = L.u[BX + d][qp] - L.u[BX + d][q];
        else if (S.flags & 2) s[d][f] = 0.5 * ((w[f] - L.W[f][qm]) + (L.W[f][qp] - w[f]));
        else s[d][f] = minmod(w[f] - L.W[f][qm], L.W[f][qp] - w[f]);
        L.S[d][f][q] = s[d][f];
      }
    }
    R ir = R(1.0) / w[0];
    R wh[8];
    for (int f = 0; f < 8; ++f) wh[f] = w[f];
    for (int d = 0; d < dim; ++d) {
      R dw[8];
      prim_rhs<R>(w, s[d], d, R(gamma), ir, dw);
      if (S.flags & 16) dw[4] = dw[4] - R(gamma - 1.0) * w[4] * s[d][1 + d];  // planted mistake (control)
      if ((S.flags & 32) && d == 2) {                                          // planted mistake (control)
        dw[5 + 0] = dw[5 + 0] - R(2.0) * w[5 + 0] * s[d][1 + d];
        dw[5 + 1] = dw[5 + 1] - R(2.0) * w[5 + 1] * s[d][1 + d];
      }
      if ((S.flags & 64) && d == 2) dw[1 + d] = dw[1 + d] - s[d][4] * ir;     // planted mistake (control)
      for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h[d] * dw[f];
    }
    for (int f = 0; f < 8; ++f) L.Wh[f][q] = wh[f];
    // cell-centre reference EMF -(v x B) at the half step (R5)
    L.ref[0][q] = wh[3] * wh[6] - wh[2] * wh[7];
    L.ref[1][q] = wh[1] * wh[7] - wh[3] * wh[5];
    L.ref[2][q] = wh[2] * wh[5] - wh[1] * wh[6];
  });
  // HLLD fluxes at d-faces (R3, R4); face stored at the cell on its high side
  for (int d = 0; d < dim; ++d) {
    const int t = (d + 1) % 3, u = (d + 2) % 3;
    for_all(L, [&](int i, int j, int k) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      if (!inc(i, j, k, 1) || !inc(m[0], m[1], m[2], 1)) return;
      size_t qr = at(L, i, j, k), ql = at(L, m[0], m[1], m[2]);
      R wl[8], wr[8];
      for (int f = 0; f < 8; ++f) {
        wl[f] = L.Wh[f][ql] + 0.5 * L.S[d][f][ql];
        wr[f] = L.Wh[f][qr] - 0.5 * L.S[d][f][qr];
      }
      R bn = 0.5 * (wl[5 + d] + wr[5 + d]);
      R rl[7] = {wl[0], wl[1 + d], wl[1 + t], wl[1 + u], wl[4], wl[5 + t], wl[5 + u]};
      R rr[7] = {wr[0], wr[1 + d], wr[1 + t], wr[1 + u], wr[4], wr[5 + t], wr[5 + u]};
      R fr[7];
      hlld<R>(rl, rr, bn, R(gamma), R(S.eps), fr);
      L.F[d][RHO][qr] = fr[0];
      L.F[d][MX + d][qr] = fr[1];
      L.F[d][MX + t][qr] = fr[2];
      L.F[d][MX + u][qr] = fr[3];
      L.F[d][EN][qr] = fr[4];
      L.F[d][BX + t][qr] = fr[5];
      L.F[d][BX + u][qr] = fr[6];
      L.F[d][BX + d][qr] = 0.0;
    });
  }
  // edge EMFs (R5): E_c at the edge (a-1/2, b-1/2), stored at cell (a, b)
  for (int c = 0; c < 3; ++c) {
    if (dim == 2 && c != 2) continue;
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    for_all(L, [&](int i, int j, int k) {
      int o[3] = {i, j, k}, oa[3] = {i, j, k}, ob[3] = {i, j, k};
      o[a] -= 1; o[b] -= 1;
      oa[a] -= 1;
      ob[b] -= 1;
      if (!inc(i, j, k, 1) || !inc(oa[0], oa[1], oa[2], 1) || !inc(ob[0], ob[1], ob[2], 1) ||
          !inc(o[0], o[1], o[2], 1))
        return;
      size_t q11 = at(L, i, j, k);
      size_t q01 = at(L, oa[0], oa[1], oa[2]);
      size_t q10 = at(L, ob[0], ob[1], ob[2]);
      size_t q00 = at(L, o[0], o[1], o[2]);
      // E_c on an a-face is -F_a[B_b]; on a b-face it is +F_b[B_a].
      R ea_hi = -L.F[a][BX + b][q11], ea_lo = -L.F[a][BX + b][q10];
      R eb_hi = L.F[b][BX + a][q11], eb_lo = L.F[b][BX + a][q01];
      L.E[c][q11] = gs_edge_emf(ea_lo, ea_hi, eb_lo, eb_hi, L.ref[c][q00], L.ref[c][q10],
                                L.ref[c][q01], L.ref[c][q11], L.F[a][RHO][q10], L.F[a][RHO][q11],
                                L.F[b][RHO][q01], L.F[b][RHO][q11]);
    });
  }
  // updates: new values into Wh storage reused as the output buffer
  int cf[6];
  const int ncf = cell_fields(S, cf);
  double dtd[3];
  for (int d = 0; d < 3; ++d) dtd[d] = dt * L.idx[d];
  std::vector<R> nu[NFIELD];
  for (int f = 0; f < NFIELD; ++f) nu[f] = L.u[f];
  for_all(L, [&](int i, int j, int k) {
    size_t q = at(L, i, j, k);
    // cell update
    if (in(q, 0)) {
      if (L.dist[q] == 0) S.cell_updates++;
      for (int n = 0; n < ncf; ++n) {
        int f = cf[n];
        R v = L.u[f][q];
        for (int d = 0; d < dim; ++d) v = v - dtd[d] * (L.F[d][f][atd(L, i, j, k, d, 1)] - L.F[d][f][q]);
        nu[f][q] = v;
      }
    }
    // face updates: d-face stored at q (between q-e_d and q)
    for (int d = 0; d < dim; ++d) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      if (!in(q, 0) && !inc(m[0], m[1], m[2], 0)) continue;
      R v = L.u[BX + d][q];
      if (dim == 2) {
        if (d == 0) v = v - dtd[1] * (L.E[2][atd(L, i, j, k, 1, 1)] - L.E[2][q]);
        else        v = v + dtd[0] * (L.E[2][atd(L, i, j, k, 0, 1)] - L.E[2][q]);
      } else {
        if (d == 0) {
          v = v - dtd[1] * (L.E[2][atd(L, i, j, k, 1, 1)] - L.E[2][q]);
          v = v + dtd[2] * (L.E[1][atd(L, i, j, k, 2, 1)] - L.E[1][q]);
        } else if (d == 1) {
          v = v - dtd[2] * (L.E[0][atd(L, i, j, k, 2, 1)] - L.E[0][q]);
          v = v + dtd[0] * (L.E[2][atd(L, i, j, k, 0, 1)] - L.E[2][q]);
        } else {
          v = v - dtd[0] * (L.E[1][atd(L, i, j, k, 0, 1)] - L.E[1][q]);
          v = v + dtd[1] * (L.E[0][atd(L, i, j, k, 1, 1)] - L.E[0][q]);
        }
      }
      nu[BX + d][q] = v;
    }
  });
  for (int f = 0; f < NFIELD; ++f) L.u[f].swap(nu[f]);
}

// ---------------------------------------------------------------- prolongation (R8)
// Conserved cell fields: minmod-limited linear, children average to the parent.
// Face B: fine faces on coarse faces = coarse face + minmod transverse slopes;
// fine faces inside a coarse cell from the divergence-free quadratic
// reconstruction (Balsara 2001): mean of the two bracketing fine faces plus
// (dx_n/8) sum over the transverse t of (d/dn-slope of B_t on the high t-face
// - the same on the low t-face) / dx_t.
template <class R> static R prolong_cell(const SimT<R>& S, const LevelT<R>& C, int f, int ci, int cj, int ck, int oa, int ob, int oc) {
  const std::vector<R>& u = C.start[f];
  size_t q = at(C, ci, cj, ck);
  R v = u[q];
  const int off[3] = {oa, ob, oc};
  R r = u[q];
  for (int d = 0; d < S.dim; ++d) {
    R sl = minmod(u[q] - u[atd(C, ci, cj, ck, d, -1)], u[atd(C, ci, cj, ck, d, 1)] - u[q]);
    r = r + sl * (off[d] ? 0.25 : -0.25);
  }
  (void)v;
  return r;
}

// Fine value of B_n on the coarse n-face stored at coarse cell (ci,cj,ck),
// at the fine sub-face with transverse offsets given by fine parities.
template <class R> static R prolong_coincident(const SimT<R>& S, const LevelT<R>& C, int n, int ci, int cj, int ck, const int* par) {
  const std::vector<R>& b = C.start[BX + n];
  size_t q = at(C, ci, cj, ck);
  R v = b[q];
  for (int d = 0; d < S.dim; ++d) {
    if (d == n) continue;
    R sl = minmod(b[q] - b[atd(C, ci, cj, ck, d, -1)], b[atd(C, ci, cj, ck, d, 1)] - b[q]);
    v = v + sl * (par[d] ? 0.25 : -0.25);
  }
  return v;
}

// Transverse slope along direction d of B_t on the coarse t-face stored at (ci,cj,ck).
template <class R> static R face_slope(const LevelT<R>& C, int t, int d, int ci, int cj, int ck) {
  const std::vector<R>& b = C.start[BX + t];
  size_t q = at(C, ci, cj, ck);
  return minmod(b[q] - b[atd(C, ci, cj, ck, d, -1)], b[atd(C, ci, cj, ck, d, 1)] - b[q]);
}

// Fine n-face at fine index (fi,fj,fk) (position fi-1/2 etc. along n).
template <class R> static R prolong_face(const SimT<R>& S, const LevelT<R>& C, const LevelT<R>& F, int n, int fi, int fj, int fk) {
  int fidx[3] = {fi, fj, fk};
  int cidx[3], par[3];
  for (int d = 0; d < 3; ++d) {
    if (d < S.dim) { cidx[d] = fidx[d] >> 1; par[d] = fidx[d] & 1; }
    else { cidx[d] = 0; par[d] = 0; }
  }
  if (!par[n]) return prolong_coincident(S, C, n, cidx[0], cidx[1], cidx[2], par);
  // interior face of coarse cell cidx: bracketing coincident fine faces
  int hi[3] = {cidx[0], cidx[1], cidx[2]};
  hi[n] += 1;
  R lo_v = prolong_coincident(S, C, n, cidx[0], cidx[1], cidx[2], par);
  R hi_v = prolong_coincident(S, C, n, hi[0], hi[1], hi[2], par);
  R corr = 0.0;
  for (int t = 0; t < S.dim; ++t) {
    if (t == n) continue;
    int th[3] = {cidx[0], cidx[1], cidx[2]};
    th[t] += 1;
    R s_hi = face_slope(C, t, n, th[0], th[1], th[2]);
    R s_lo = face_slope(C, t, n, cidx[0], cidx[1], cidx[2]);
    corr = corr + (C.dx[n] / C.dx[t]) * (s_hi - s_lo);
  }
  (void)F;
  return 0.5 * (lo_v + hi_v) + 0.125 * corr;
}

// P: fill the band (1 <= dist <= 4) of level l from level l-1's start state.
template <class R> static void prolong_band(SimT<R>& S, int l) {
  LevelT<R>& F = S.lev[l];
  const LevelT<R>& C = S.lev[l - 1];
  int cf[6];
  const int ncf = cell_fields(S, cf);
  for_cells(F, [&](int i, int j, int k) {
    size_t q = at(F, i, j, k);
    if (F.dist[q] >= 1) {
      for (int n = 0; n < ncf; ++n)
        F.u[cf[n]][q] = prolong_cell(S, C, cf[n], i >> 1, j >> 1, S.dim == 3 ? k >> 1 : 0, i & 1, j & 1, S.dim == 3 ? (k & 1) : 0);
    }
  });
  // d-face between cells q-e_d and q of the domain closure: prolonged if not
  // owned (no adjacent region cell) and adjacent to a band cell
  for (int d = 0; d < S.dim; ++d)
    for_face_pos(F, d, [&](int i, int j, int k) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      int8_t dd = in_storage(F, i, j, k) ? F.dist[at(F, i, j, k)] : -1;
      int8_t dm = in_storage(F, m[0], m[1], m[2]) ? F.dist[at(F, m[0], m[1], m[2])] : -1;
      if (dd == 0 || dm == 0) return;
      if (dd < 0 && dm < 0) return;
      F.u[BX + d][at(F, i, j, k)] = prolong_face(S, C, F, d, i, j, k);
    });
}

// Physical boundaries (R17): margin cells and faces outside the domain. Cells
// copy the nearest domain cell (zero-gradient outflow) or take the inflow
// state; a face whose normal index lies beyond the boundary face copies that
// boundary face, a face of a margin cell along another dimension copies the
// face of the nearest domain cell; inflow faces take the inflow field.
template <class R> static bool outside_kind(const SimT<R>& S, const LevelT<R>& L, const int* o, int* clamped) {
  bool inflow = false;
  for (int d = 0; d < 3; ++d) {
    clamped[d] = o[d];
    if (L.per[d]) continue;
    if (o[d] < 0) { clamped[d] = 0; inflow |= S.bc[d][0] == BC_INFLOW; }
    else if (o[d] >= L.N[d]) { clamped[d] = L.N[d] - 1; inflow |= S.bc[d][1] == BC_INFLOW; }
  }
  return inflow;
}

template <class R> static void fill_bc(SimT<R>& S, int l) {
  LevelT<R>& L = S.lev[l];
  bool any = false;
  for (int d = 0; d < S.dim; ++d) any |= !L.per[d];
  if (!any) return;
  int cf[6];
  const int ncf = cell_fields(S, cf);
  for_all(L, [&](int i, int j, int k) {
    const int o[3] = {i, j, k};
    if (in_domain(L, i, j, k)) return;
    int c[3];
    const bool inflow = outside_kind(S, L, o, c);
    size_t q = at(L, i, j, k), qs = at(L, c[0], c[1], c[2]);
    for (int n = 0; n < ncf; ++n) L.u[cf[n]][q] = inflow ? R(S.inflow[cf[n]]) : L.u[cf[n]][qs];
  });
  for (int d = 0; d < S.dim; ++d) {
    // d-face positions of the storage: along a non-periodic d one beyond the cells
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      lo[e] = -L.M[e];
      hi[e] = L.N[e] + L.M[e] + ((e == d && !L.per[e]) ? 1 : 0);
    }
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          const int o[3] = {i, j, k};
          bool out = false, inflow = false;
          int c[3] = {i, j, k};
          for (int e = 0; e < 3; ++e) {
            if (L.per[e]) continue;
            const int top = e == d ? L.N[e] : L.N[e] - 1;
            if (o[e] < 0) { out = true; c[e] = 0; inflow |= S.bc[e][0] == BC_INFLOW; }
            else if (o[e] > top) {
              out = true;
              // bit 2 of flags: a planted off-by-one (the high-side normal face
              // copies the face one cell inside) for the mirror-pair control
              c[e] = (e == d && (S.flags & 4)) ? top - 1 : top;
              inflow |= S.bc[e][1] == BC_INFLOW;
            }
          }
          if (!out) continue;
          L.u[BX + d][at(L, i, j, k)] = inflow ? R(S.inflow[BX + d]) : L.u[BX + d][at(L, c[0], c[1], c[2])];
        }
  }
}

// ---------------------------------------------------------------- registers, reflux, restriction (R9)
template <class R> static void record_coarse_registers(SimT<R>& S, int l, double dt) {
  LevelT<R>& C = S.lev[l];
  LevelT<R>& F = S.lev[l + 1];
  int cf[6];
  const int ncf = cell_fields(S, cf);
  for (int d = 0; d < S.dim; ++d)
    for (size_t q = 0; q < C.ncell; ++q) {
      if (!F.cf_face[d][q]) continue;
      for (int n = 0; n < ncf; ++n) { F.rflux[d][cf[n]][q] = 0.0; F.rcoarse[d][cf[n]][q] = dt * C.F[d][cf[n]][q]; }
    }
  for (int c = 0; c < 3; ++c) {
    if (S.dim == 2 && c != 2) continue;
    for (size_t q = 0; q < C.ncell; ++q)
      if (F.cf_edge[c][q]) { F.remf[c][q] = 0.0; F.remfc[c][q] = dt * C.E[c][q]; }
  }
}

// Pairwise sum of 2, 4 or 8 values in the given order: ((v0+v1)+(v2+v3))+...
// (R9: exact for equal values, so uniform states stay bitwise uniform).
template <class V> static V tree_sum(const V* v, int n) {
  if (n == 1) return v[0];
  if (n == 2) return v[0] + v[1];
  if (n == 4) return (v[0] + v[1]) + (v[2] + v[3]);
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}

// Fine side of the registers after one fine sub-step of dt: per C/F coarse
// face R += (dt 2^-(dim-1)) * tree_sum(fine sub-face fluxes in z,y,x order);
// per C/F coarse edge R += (dt 2^-(dim-2)) * tree_sum(fine sub-edges along it).
template <class R> static void add_fine_registers(SimT<R>& S, int l, double dt) {
  LevelT<R>& F = S.lev[l];
  LevelT<R>& C = S.lev[l - 1];
  int cf[6];
  const int ncf = cell_fields(S, cf);
  const double af = dt * (S.dim == 3 ? 0.25 : 0.5);
  const double ae = dt * (S.dim == 3 ? 0.5 : 1.0);
  for (int d = 0; d < S.dim; ++d)
    for_face_pos(C, d, [&](int i, int j, int k) {
      size_t q = at(C, i, j, k);
      if (!F.cf_face[d][q]) return;
      size_t qf[4];
      int m = 0;
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1)
          for (int c0 = 0; c0 < 2; ++c0) {
            int o[3] = {c0, c1, c2};
            if (o[d] != 0) continue;
            if (S.dim == 2 && c2 != 0) continue;
            qf[m++] = at(F, 2 * i + o[0], 2 * j + o[1], S.dim == 3 ? 2 * k + o[2] : 0);
          }
      for (int n = 0; n < ncf; ++n) {
        R v[4];
        for (int s = 0; s < m; ++s) v[s] = F.F[d][cf[n]][qf[s]];
        F.rflux[d][cf[n]][q] += af * tree_sum(v, m);
      }
    });
  for (int c = 0; c < 3; ++c) {
    if (S.dim == 2 && c != 2) continue;
    for_edge_pos(C, c, [&](int i, int j, int k) {
      size_t q = at(C, i, j, k);
      if (!F.cf_edge[c][q]) return;
      int nsub = S.dim == 3 ? 2 : 1;
      R v[2];
      for (int sidx = 0; sidx < nsub; ++sidx) {
        int o[3] = {2 * i, 2 * j, S.dim == 3 ? 2 * k : 0};
        o[c] += sidx;
        v[sidx] = F.E[c][at(F, o[0], o[1], o[2])];
      }
      F.remf[c][q] += ae * tree_sum(v, nsub);
    });
  }
}

template <class R> static void restrict_cell(const SimT<R>& S, LevelT<R>& C, const LevelT<R>& F, int i, int j, int k, double wc) {
  int cf[6];
  const int ncf = cell_fields(S, cf);
  const int kz = S.dim == 3 ? 2 : 1;
  size_t q = at(C, i, j, k);
  for (int n = 0; n < ncf; ++n) {
    R v[8];
    int m = 0;
    for (int c = 0; c < kz; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) v[m++] = F.u[cf[n]][at(F, 2 * i + a, 2 * j + b, S.dim == 3 ? 2 * k + c : 0)];
    C.u[cf[n]][q] = tree_sum(v, m) * wc;
  }
}

template <class R> static void restrict_face(const SimT<R>& S, LevelT<R>& C, const LevelT<R>& F, int d, int i, int j, int k, double wf) {
  const int kz = S.dim == 3 ? 2 : 1;
  R v[4];
  int m = 0;
  for (int c = 0; c < kz; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        int o[3] = {a, b, c};
        if (o[d] != 0) continue;
        v[m++] = F.u[BX + d][at(F, 2 * i + o[0], 2 * j + o[1], S.dim == 3 ? 2 * k + o[2] : 0)];
      }
  C.u[BX + d][at(C, i, j, k)] = tree_sum(v, m) * wf;
}

template <class R> static void reflux_and_restrict(SimT<R>& S, int l) {
  // level l is the fine level; corrections go to level l-1
  LevelT<R>& F = S.lev[l];
  LevelT<R>& C = S.lev[l - 1];
  int cf[6];
  const int ncf = cell_fields(S, cf);
  // S: cell reflux on uncovered coarse cells, faces in order x-,x+,y-,y+,z-,z+
  for_cells(C, [&](int i, int j, int k) {
    size_t q = at(C, i, j, k);
    if (C.cov[q] || (S.flags & 1)) return;
    for (int d = 0; d < S.dim; ++d) {
      size_t qlo = q, qhi = atd(C, i, j, k, d, 1);
      if (F.cf_face[d][qlo])
        for (int n = 0; n < ncf; ++n)
          C.u[cf[n]][q] = C.u[cf[n]][q] + (F.rflux[d][cf[n]][qlo] - F.rcoarse[d][cf[n]][qlo]) * C.idx[d];
      if (F.cf_face[d][qhi])
        for (int n = 0; n < ncf; ++n)
          C.u[cf[n]][q] = C.u[cf[n]][q] - (F.rflux[d][cf[n]][qhi] - F.rcoarse[d][cf[n]][qhi]) * C.idx[d];
    }
  });
  // EMF correction on uncovered coarse faces adjacent to C/F edges (a cell
  // outside the domain counts as uncovered)
  auto covered = [&](int i, int j, int k) { return in_domain(C, i, j, k) && C.cov[at(C, i, j, k)]; };
  for (int d = 0; d < S.dim; ++d)
    for_face_pos(C, d, [&](int i, int j, int k) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      if (covered(i, j, k) || covered(m[0], m[1], m[2])) return;
      size_t q = at(C, i, j, k);
      R v = C.u[BX + d][q];
      auto add = [&](int c, int si, int sj, int sk, double coef) {
        int e[3] = {i + si, j + sj, k + sk};
        size_t qe = at(C, e[0], e[1], e[2]);
        if (in_storage(C, e[0], e[1], e[2]) && F.cf_edge[c][qe]) v = v + coef * (F.remf[c][qe] - F.remfc[c][qe]);
      };
      if (S.dim == 2) {
        if (d == 0) { add(2, 0, 0, 0, C.idx[1]); add(2, 0, 1, 0, -C.idx[1]); }
        else        { add(2, 0, 0, 0, -C.idx[0]); add(2, 1, 0, 0, C.idx[0]); }
      } else if (d == 0) {
        add(2, 0, 0, 0, C.idx[1]); add(2, 0, 1, 0, -C.idx[1]);
        add(1, 0, 0, 0, -C.idx[2]); add(1, 0, 0, 1, C.idx[2]);
      } else if (d == 1) {
        add(0, 0, 0, 0, C.idx[2]); add(0, 0, 0, 1, -C.idx[2]);
        add(2, 0, 0, 0, -C.idx[0]); add(2, 1, 0, 0, C.idx[0]);
      } else {
        add(1, 0, 0, 0, C.idx[0]); add(1, 1, 0, 0, -C.idx[0]);
        add(0, 0, 0, 0, -C.idx[1]); add(0, 0, 1, 0, C.idx[1]);
      }
      C.u[BX + d][q] = v;
    });
  // R: restriction of covered cells and of faces in the closure of the fine
  // region: pairwise sums in z,y,x child order times 2^-dim (2^-(dim-1)).
  const double wc = S.dim == 3 ? 0.125 : 0.25;
  const double wf = S.dim == 3 ? 0.25 : 0.5;
  for_cells(C, [&](int i, int j, int k) {
    if (C.cov[at(C, i, j, k)]) restrict_cell(S, C, F, i, j, k, wc);
  });
  for (int d = 0; d < S.dim; ++d)
    for_face_pos(C, d, [&](int i, int j, int k) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      if (!covered(i, j, k) && !covered(m[0], m[1], m[2])) return;
      restrict_face(S, C, F, d, i, j, k, wf);
    });
}

// ---------------------------------------------------------------- CFL (R6)
template <class R> static double level_rate(const SimT<R>& S, const LevelT<R>& L) {
  double m = 0.0;
  for_cells(L, [&](int i, int j, int k) {
    size_t q = at(L, i, j, k);
    if (L.dist[q] != 0) return;
    double w[8];
    prim_at(S, L, i, j, k, w);
    if (!(w[0] > 0.0) || !(w[4] > 0.0)) { m = NAN; return; }
    double r = 0.0;
    for (int d = 0; d < S.dim; ++d) {
      int t = (d + 1) % 3, u = (d + 2) % 3;
      double cf = fast_speed(w[0], w[4], w[5 + d], w[5 + t], w[5 + u], S.gamma);
      r = r + (fabs(w[1 + d]) + cf) * L.idx[d];
    }
    if (std::isnan(m)) return;
    if (std::isnan(r)) m = NAN;
    else if (r > m) m = r;
  });
  return m;
}

template <class R> static double cfl_dt(const SimT<R>& S) {
  double mmax = 0.0;
  double scale = 1.0;
  for (int l = 0; l < S.nlev; ++l) {
    double m = level_rate(S, S.lev[l]) * scale;
    if (std::isnan(m)) return NAN;
    if (m > mmax) mmax = m;
    scale *= 0.5;
  }
  return S.cfl / mmax;
}

// ---------------------------------------------------------------- recursion (Sec. 4)
template <class R> static void level_substep(SimT<R>& S, int l, int s, double dt) {
  LevelT<R>& L = S.lev[l];
  const int w = (l == 0) ? 0 : (s == 1 ? 2 : 0);
  if (l > 0 && s == 1) prolong_band(S, l);  // P
  fill_bc(S, l);
  for (int f = 0; f < NFIELD; ++f) L.start[f] = L.u[f];
  L.tmask.assign(L.ncell, -1);
  for (size_t q = 0; q < L.ncell; ++q)
    if (L.dist[q] >= 0 && L.dist[q] <= w) L.tmask[q] = 0;
  dilate(S, L, L.tmask);
  advance_masked(S, L, dt);  // A
  if (l > 0) add_fine_registers(S, l, dt);
  if (l + 1 < S.nlev) {
    record_coarse_registers(S, l, dt);
    level_substep(S, l + 1, 1, dt * 0.5);
    level_substep(S, l + 1, 2, dt * 0.5);
    reflux_and_restrict(S, l + 1);  // S and R
  }
}

// ---------------------------------------------------------------- regrid (reading R18)
// Every level above 0 is rebuilt from the flags of the level below, coarse to
// fine: flag, buffer by 2 cells, mark the aligned blocks of 4 x 4 (x 4) level-l
// cells holding a buffered flag, keep the blocks whose 3-cell surroundings lie
// in the level-l region (proper nesting), merge them greedily in z,y,x order
// into boxes of at most 4 blocks per side, refine the boxes by 2. New fine data
// are copied from the old fine level where it covered the parent cell, else
// prolonged; fine faces on a coarse face next to copied data are copied, and the
// interior faces of a prolonged coarse cell then get the smallest correction
// that makes every child divergence-free.
using Level = LevelT<double>;
using Sim = SimT<double>;

static const int RG_B = 4;     // block edge in parent cells
static const int RG_MAXB = 4;  // blocks per box side at most

static bool rg_old(const Sim& S, int l, int ci, int cj, int ck) {
  // coarse cell (ci,cj,ck) of level l covered by the old level l+1
  if (S.nlev <= l + 1) return false;
  const Level& F = S.lev[l + 1];
  if (!in_domain(S.lev[l], ci, cj, ck)) return false;
  return F.dist[at(F, 2 * ci, 2 * cj, S.dim == 3 ? 2 * ck : 0)] == 0;
}

// least-norm correction of the interior faces of a coarse cell so that every
// child has zero discrete divergence; faces ordered d, then transverse children
// in z,y,x order; r: child divergences (children in z,y,x order)
static void rg_closure(int dim, const double* idx, const double* r, double* delta) {
  const int nc = dim == 3 ? 8 : 4;
  const int nt = dim == 3 ? 4 : 2;
  const int nf = dim * nt;
  double M[8][12] = {};
  int f = 0;
  for (int d = 0; d < dim; ++d)
    for (int t = 0; t < nt; ++t, ++f) {
      // transverse child offsets of this face
      int o[3] = {0, 0, 0}, b = 0;
      for (int e = 0; e < dim; ++e) {
        if (e == d) continue;
        o[e] = (t >> b) & 1;
        ++b;
      }
      int lo[3] = {o[0], o[1], o[2]}, hi[3] = {o[0], o[1], o[2]};
      lo[d] = 0;
      hi[d] = 1;
      const int clo = lo[0] + 2 * lo[1] + 4 * lo[2], chi = hi[0] + 2 * hi[1] + 4 * hi[2];
      M[clo][f] += idx[d];   // the face is the high face of the low child
      M[chi][f] -= idx[d];   // and the low face of the high child
    }
  // (M M^T + 1 1^T) y = -r, delta = M^T y
  double A[8][9];
  for (int i = 0; i < nc; ++i) {
    for (int j = 0; j < nc; ++j) {
      double s = 1.0;
      for (int k = 0; k < nf; ++k) s += M[i][k] * M[j][k];
      A[i][j] = s;
    }
    A[i][nc] = -r[i];
  }
  for (int c = 0; c < nc; ++c) {
    int piv = c;
    for (int i = c + 1; i < nc; ++i)
      if (std::fabs(A[i][c]) > std::fabs(A[piv][c])) piv = i;
    for (int j = 0; j <= nc; ++j) std::swap(A[c][j], A[piv][j]);
    for (int i = 0; i < nc; ++i) {
      if (i == c) continue;
      const double m = A[i][c] / A[c][c];
      for (int j = c; j <= nc; ++j) A[i][j] -= m * A[c][j];
    }
  }
  double y[8];
  for (int i = 0; i < nc; ++i) y[i] = A[i][nc] / A[i][i];
  for (int k = 0; k < nf; ++k) {
    double s = 0.0;
    for (int i = 0; i < nc; ++i) s += M[i][k] * y[i];
    delta[k] = s;
  }
}

// flags of level l of N: region cells with max_d |rho(i+1) - rho(i-1)| / (2 rho) > theta
static std::vector<int8_t> rg_flags(const Sim& N, int l, double theta) {
  const Level& L = N.lev[l];
  std::vector<int8_t> fl(L.ncell, -1);  // 0 = flagged
  for_cells(L, [&](int i, int j, int k) {
    const size_t q = at(L, i, j, k);
    if (L.dist[q] != 0) return;
    const double r = L.u[RHO][q];
    double m = 0.0;
    for (int d = 0; d < N.dim; ++d) {
      const double g = std::fabs(L.u[RHO][atd(L, i, j, k, d, 1)] - L.u[RHO][atd(L, i, j, k, d, -1)]) / (2.0 * r);
      if (g > m) m = g;
    }
    if (m > theta) fl[q] = 0;
  });
  return fl;
}

// new level l+1 boxes (fine coordinates) from the flag map fl of level l of N
static std::vector<Patch> rg_boxes(const Sim& N, int l, const std::vector<int8_t>& fl) {
  const Level& L = N.lev[l];
  const int dim = N.dim;
  // buffer of 2 cells (Chebyshev), inside the domain and the level region
  const int kz = dim == 3 ? 1 : 0;
  std::vector<char> buf(L.ncell, 0);
  for_cells(L, [&](int i, int j, int k) {
    if (fl[at(L, i, j, k)] != 0) return;
    for (int c = -2 * kz; c <= 2 * kz; ++c)
      for (int b = -2; b <= 2; ++b)
        for (int a = -2; a <= 2; ++a) {
          if (!in_domain(L, i + a, j + b, k + c)) continue;
          const size_t q = at(L, i + a, j + b, k + c);
          if (L.dist[q] == 0) buf[q] = 1;
        }
  });
  int nb[3];
  for (int d = 0; d < 3; ++d) nb[d] = d < dim ? L.N[d] / RG_B : 1;
  const size_t nblk = (size_t)nb[0] * nb[1] * nb[2];
  std::vector<char> ok(nblk, 0);
  auto bidx = [&](int a, int b, int c) { return ((size_t)c * nb[1] + b) * nb[0] + a; };
  for (int bk = 0; bk < nb[2]; ++bk)
    for (int bj = 0; bj < nb[1]; ++bj)
      for (int bi = 0; bi < nb[0]; ++bi) {
        const int lo[3] = {bi * RG_B, bj * RG_B, dim == 3 ? bk * RG_B : 0};
        const int hi[3] = {lo[0] + RG_B, lo[1] + RG_B, dim == 3 ? lo[2] + RG_B : 1};
        bool want = false;
        for (int k = lo[2]; k < hi[2]; ++k)
          for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) want |= buf[at(L, i, j, k)] != 0;
        if (!want) continue;
        bool allowed = true;
        const int g = 3;
        for (int k = lo[2] - g * kz; k < hi[2] + g * kz && allowed; ++k)
          for (int j = lo[1] - g; j < hi[1] + g && allowed; ++j)
            for (int i = lo[0] - g; i < hi[0] + g && allowed; ++i) {
              if (!in_domain(L, i, j, k)) continue;
              if (L.dist[at(L, i, j, k)] != 0) allowed = false;
            }
        if (allowed) ok[bidx(bi, bj, bk)] = 1;
      }
  std::vector<Patch> out;
  for (int bk = 0; bk < nb[2]; ++bk)
    for (int bj = 0; bj < nb[1]; ++bj)
      for (int bi = 0; bi < nb[0]; ++bi) {
        if (!ok[bidx(bi, bj, bk)]) continue;
        int nx = 1, ny = 1, nz = 1;
        while (nx < RG_MAXB && bi + nx < nb[0] && ok[bidx(bi + nx, bj, bk)]) ++nx;
        auto row_ok = [&](int b, int c) {
          for (int t = 0; t < nx; ++t)
            if (!ok[bidx(bi + t, b, c)]) return false;
          return true;
        };
        while (ny < RG_MAXB && bj + ny < nb[1] && row_ok(bj + ny, bk)) ++ny;
        if (dim == 3) {
          auto slab_ok = [&](int c) {
            for (int u = 0; u < ny; ++u)
              if (!row_ok(bj + u, c)) return false;
            return true;
          };
          while (nz < RG_MAXB && bk + nz < nb[2] && slab_ok(bk + nz)) ++nz;
        }
        for (int c = 0; c < nz; ++c)
          for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) ok[bidx(bi + a, bj + b, bk + c)] = 0;
        Patch p;
        p.level = l + 1;
        p.lo[0] = 2 * RG_B * bi; p.hi[0] = 2 * RG_B * (bi + nx);
        p.lo[1] = 2 * RG_B * bj; p.hi[1] = 2 * RG_B * (bj + ny);
        p.lo[2] = dim == 3 ? 2 * RG_B * bk : 0;
        p.hi[2] = dim == 3 ? 2 * RG_B * (bk + nz) : 1;
        out.push_back(p);
      }
  return out;
}

// band fill of level l of N (prolongation from l-1 and boundaries), then start = u
static void rg_fill(Sim& N, int l) {
  if (l > 0) {
    for (int f = 0; f < NFIELD; ++f) N.lev[l - 1].start[f] = N.lev[l - 1].u[f];
    prolong_band(N, l);
  }
  fill_bc(N, l);
  for (int f = 0; f < NFIELD; ++f) N.lev[l].start[f] = N.lev[l].u[f];
}

// level l+1 of N from the old simulation S and level l of N
static void rg_transfer(const Sim& S, Sim& N, int l) {
  const int dim = N.dim;
  const Level& C = N.lev[l];
  Level& F = N.lev[l + 1];
  const Level* O = S.nlev > l + 1 ? &S.lev[l + 1] : nullptr;
  int cf[6];
  const int ncf = cell_fields(N, cf);
  for_cells(F, [&](int i, int j, int k) {
    const size_t q = at(F, i, j, k);
    if (F.dist[q] != 0) return;
    if (rg_old(S, l, i >> 1, j >> 1, k >> 1)) {
      for (int n = 0; n < ncf; ++n) F.u[cf[n]][q] = O->u[cf[n]][at(*O, i, j, k)];
    } else {
      for (int n = 0; n < ncf; ++n)
        F.u[cf[n]][q] = prolong_cell(N, C, cf[n], i >> 1, j >> 1, dim == 3 ? k >> 1 : 0, i & 1, j & 1,
                                     dim == 3 ? (k & 1) : 0);
    }
  });
  // faces in the closure of the new region
  for (int d = 0; d < dim; ++d)
    for_face_pos(F, d, [&](int i, int j, int k) {
      int m[3] = {i, j, k};
      m[d] -= 1;
      const bool rq = in_storage(F, i, j, k) && F.dist[at(F, i, j, k)] == 0;
      const bool rm = in_storage(F, m[0], m[1], m[2]) && F.dist[at(F, m[0], m[1], m[2])] == 0;
      if (!rq && !rm) return;
      const int pq[3] = {i >> 1, j >> 1, dim == 3 ? k >> 1 : 0};
      const int pm[3] = {m[0] >> 1, m[1] >> 1, dim == 3 ? m[2] >> 1 : 0};
      const bool interior = pq[d] == pm[d];
      const bool copy = interior ? rg_old(S, l, pq[0], pq[1], pq[2])
                                 : (rg_old(S, l, pq[0], pq[1], pq[2]) || rg_old(S, l, pm[0], pm[1], pm[2]));
      const size_t q = at(F, i, j, k);
      if (copy) F.u[BX + d][q] = O->u[BX + d][at(*O, i, j, k)];
      else F.u[BX + d][q] = prolong_face(N, C, F, d, i, j, k);
    });
  // divergence-free closure of prolonged coarse cells touching copied faces
  // (bit 3 of flags skips it: a planted mistake for the div B control)
  if (N.flags & 8) return;
  for_cells(C, [&](int ci, int cj, int ck) {
    const int f0[3] = {2 * ci, 2 * cj, dim == 3 ? 2 * ck : 0};
    if (F.dist[at(F, f0[0], f0[1], f0[2])] != 0) return;  // not in the new fine region
    if (rg_old(S, l, ci, cj, ck)) return;
    bool touches = false;
    for (int d = 0; d < dim; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int nbc[3] = {ci, cj, ck};
        nbc[d] += s;
        touches |= rg_old(S, l, nbc[0], nbc[1], nbc[2]);
      }
    if (!touches) return;
    const int nc = dim == 3 ? 8 : 4;
    double r[8];
    for (int c = 0; c < nc; ++c) {
      const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
      const int x = f0[0] + o[0], y = f0[1] + o[1], z = dim == 3 ? f0[2] + o[2] : 0;
      double div = 0.0;
      for (int d = 0; d < dim; ++d)
        div += (F.u[BX + d][atd(F, x, y, z, d, 1)] - F.u[BX + d][at(F, x, y, z)]) * F.idx[d];
      r[c] = div;
    }
    double delta[12];
    rg_closure(dim, F.idx, r, delta);
    const int nt = dim == 3 ? 4 : 2;
    int fi = 0;
    for (int d = 0; d < dim; ++d)
      for (int t = 0; t < nt; ++t, ++fi) {
        int o[3] = {0, 0, 0}, b = 0;
        for (int e = 0; e < dim; ++e) {
          if (e == d) continue;
          o[e] = (t >> b) & 1;
          ++b;
        }
        o[d] = 1;  // the interior face is the low face of the high child
        F.u[BX + d][at(F, f0[0] + o[0], f0[1] + o[1], dim == 3 ? f0[2] + o[2] : 0)] += delta[fi];
      }
  });
}

}  // namespace oracle

// ================================================================ C API
using namespace oracle;

extern "C" {

void* oc_new(int dim, const int* base, const double* lo, const double* hi, int nlev, double gamma, double cfl) {
  Sim* s = new Sim();
  s->dim = dim;
  for (int d = 0; d < 3; ++d) {
    s->base[d] = d < dim ? base[d] : 1;
    s->lo[d] = lo[d];
    s->hi[d] = hi[d];
  }
  s->nlev = nlev;
  s->gamma = gamma;
  s->cfl = cfl;
  return s;
}

// bc: 6 ints (x-low, x-high, y-low, y-high, z-low, z-high): 0 periodic,
// 1 outflow, 2 inflow; a dimension is periodic only with both sides 0.
// inflow: the conserved inflow state (rho, mx, my, mz, E, Bx, By, Bz).
void* oc_new2(int dim, const int* base, const double* lo, const double* hi, int nlev, double gamma, double cfl,
              const int* bc, const double* inflow) {
  Sim* s = (Sim*)oc_new(dim, base, lo, hi, nlev, gamma, cfl);
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 2; ++e) s->bc[d][e] = d < dim ? bc[2 * d + e] : 0;
  for (int f = 0; f < NFIELD; ++f) s->inflow[f] = inflow[f];
  return s;
}

void oc_free(void* h) { delete (Sim*)h; }

// patches: n x 7 int32 (level, lo0, lo1, lo2, hi0, hi1, hi2). 0 ok, -1 invalid,
// -2 nesting violated, -3 same-level overlap.
int oc_set_patches(void* h, const int* p, int n) {
  Sim* s = (Sim*)h;
  s->patches.clear();
  for (int i = 0; i < n; ++i) {
    Patch q;
    q.level = p[7 * i];
    for (int d = 0; d < 3; ++d) { q.lo[d] = p[7 * i + 1 + d]; q.hi[d] = p[7 * i + 4 + d]; }
    s->patches.push_back(q);
  }
  return validate_and_build(*s);
}

// Whole-level arrays, x fastest. Cell fields: (Nz, Ny, Nx). Face field along
// d: one extra entry along d (entry N_d repeats entry 0 on output, ignored on input).
static void field_shape(const Sim& s, int level, int field, int* n) {
  const Level& L = s.lev[level];
  for (int d = 0; d < 3; ++d) n[d] = L.N[d];
  if (is_face_field(s, field)) n[field - BX] += 1;
}

long long oc_field_size(void* h, int level, int field) {
  Sim* s = (Sim*)h;
  int n[3];
  field_shape(*s, level, field, n);
  return (long long)n[0] * n[1] * n[2];
}

int oc_set_field(void* h, int level, int field, const double* a) {
  Sim* s = (Sim*)h;
  Level& L = s->lev[level];
  int n[3];
  field_shape(*s, level, field, n);
  // a periodic dimension stores the face at N as the face at 0; a bounded one
  // stores both domain faces
  int m[3];
  for (int d = 0; d < 3; ++d) m[d] = L.per[d] ? L.N[d] : n[d];
  for (int k = 0; k < m[2]; ++k)
    for (int j = 0; j < m[1]; ++j)
      for (int i = 0; i < m[0]; ++i) L.u[field][at(L, i, j, k)] = a[((size_t)k * n[1] + j) * n[0] + i];
  return 0;
}

int oc_get_field(void* h, int level, int field, double* a) {
  Sim* s = (Sim*)h;
  Level& L = s->lev[level];
  int n[3];
  field_shape(*s, level, field, n);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) a[((size_t)k * n[1] + j) * n[0] + i] = L.u[field][at(L, i, j, k)];
  return 0;
}

double oc_cfl_dt(void* h) { return cfl_dt(*(Sim*)h); }

// One coarse step (all levels, recursive order). dt0 <= 0: use the CFL dt.
double oc_step(void* h, double dt0) {
  Sim* s = (Sim*)h;
  if (!(dt0 > 0)) dt0 = cfl_dt(*s);
  level_substep(*s, 0, 1, dt0);
  return dt0;
}

long long oc_cell_updates(void* h) { return ((Sim*)h)->cell_updates; }

// The clustering alone: new level l+1 boxes from the given flagged level-l
// cells (x, y, z triples; cells outside the level-l region are ignored).
int oc_regrid_boxes(void* h, int l, const int* flags, long long nflags, int* out, int cap, int* n) {
  Sim* s = (Sim*)h;
  const Level& L = s->lev[l];
  std::vector<int8_t> fl(L.ncell, -1);
  for (long long f = 0; f < nflags; ++f) {
    const int* c = flags + 3 * f;
    if (!in_domain(L, c[0], c[1], c[2])) continue;
    const size_t q = at(L, c[0], c[1], c[2]);
    if (L.dist[q] == 0) fl[q] = 0;
  }
  std::vector<Patch> b = rg_boxes(*s, l, fl);
  if ((int)b.size() > cap) return -4;
  *n = (int)b.size();
  for (int i = 0; i < *n; ++i) {
    out[7 * i] = b[i].level;
    for (int d = 0; d < 3; ++d) { out[7 * i + 1 + d] = b[i].lo[d]; out[7 * i + 4 + d] = b[i].hi[d]; }
  }
  return 0;
}

// Regrid (reading R18) with density-gradient threshold theta: every level
// above 0 is rebuilt, coarse to fine, up to max_levels levels; the first level
// left without boxes ends the hierarchy. out: the new patch list (n x 7, as
// oc_set_patches, levels ascending, level 0 first), *n its length. Returns 0,
// -4 if cap is too small.
int oc_regrid(void* h, double theta, int max_levels, int* out, int cap, int* n) {
  Sim* s = (Sim*)h;
  Sim* N = new Sim();
  N->dim = s->dim;
  for (int d = 0; d < 3; ++d) {
    N->base[d] = s->base[d]; N->lo[d] = s->lo[d]; N->hi[d] = s->hi[d];
    N->bc[d][0] = s->bc[d][0]; N->bc[d][1] = s->bc[d][1];
  }
  N->gamma = s->gamma; N->cfl = s->cfl; N->eps = s->eps; N->flags = s->flags;
  for (int f = 0; f < NFIELD; ++f) N->inflow[f] = s->inflow[f];
  std::vector<Patch> ps;
  for (const Patch& p : s->patches)
    if (p.level == 0) ps.push_back(p);
  N->patches = ps;
  N->nlev = 1;
  validate_and_build(*N);
  for (int f = 0; f < NFIELD; ++f) N->lev[0].u[f] = s->lev[0].u[f];
  for (int l = 0; l + 1 < max_levels; ++l) {
    rg_fill(*N, l);
    std::vector<Patch> nb = rg_boxes(*N, l, rg_flags(*N, l, theta));
    if (nb.empty()) break;
    // the new hierarchy with one more level; earlier levels keep their data
    Sim* M = new Sim(*N);
    M->patches.insert(M->patches.end(), nb.begin(), nb.end());
    M->nlev = l + 2;
    validate_and_build(*M);
    for (int q = 0; q <= l; ++q)
      for (int f = 0; f < NFIELD; ++f) M->lev[q].u[f] = N->lev[q].u[f];
    rg_fill(*M, l);
    rg_transfer(*s, *M, l);
    delete N;
    N = M;
  }
  if ((int)N->patches.size() > cap) { delete N; return -4; }
  *n = (int)N->patches.size();
  for (int i = 0; i < *n; ++i) {
    const Patch& p = N->patches[i];
    out[7 * i] = p.level;
    for (int d = 0; d < 3; ++d) { out[7 * i + 1 + d] = p.lo[d]; out[7 * i + 4 + d] = p.hi[d]; }
  }
  N->cell_updates = s->cell_updates;
  *s = *N;
  delete N;
  return 0;
}

// Test-only planted mistakes (controls showing that a pin can fail).
void oc_set_flags(void* h, int flags) { ((Sim*)h)->flags = flags; }

// Region (dist == 0) and covered masks of a level, as int8 over (Nz, Ny, Nx).
int oc_get_masks(void* h, int level, signed char* dist, signed char* cov) {
  Sim* s = (Sim*)h;
  Level& L = s->lev[level];
  size_t o = 0;
  for (int k = 0; k < L.N[2]; ++k)
    for (int j = 0; j < L.N[1]; ++j)
      for (int i = 0; i < L.N[0]; ++i, ++o) {
        const size_t q = at(L, i, j, k);
        dist[o] = L.dist[q];
        cov[o] = L.cov[q];
      }
  return 0;
}

// One single-level step of dt updating only the listed target cells (and
// their faces): targets are (i,j,k) triples on level 0 of a one-level sim.
// Used to check sampled outputs of large runs one by one.
int oc_step_targets(void* h, double dt, const int* ijk, int n) {
  Sim* s = (Sim*)h;
  Level& L = s->lev[0];
  L.tmask.assign(L.ncell, -1);
  for (int m = 0; m < n; ++m) L.tmask[at(L, ijk[3 * m], ijk[3 * m + 1], ijk[3 * m + 2])] = 0;
  dilate(*s, L, L.tmask);
  advance_masked(*s, L, dt);
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------- adjoint pins
// A copy of the simulation s (configuration, hierarchy, state) with value type
// R; the domain entries of every level's state (those oc_set_field writes)
// become the independent variables through make_input.
template <class R, class MakeInput>
static SimT<R>* clone_as(const Sim& s, MakeInput make_input) {
  SimT<R>* a = new SimT<R>();
  a->dim = s.dim;
  for (int d = 0; d < 3; ++d) {
    a->base[d] = s.base[d];
    a->lo[d] = s.lo[d];
    a->hi[d] = s.hi[d];
    a->bc[d][0] = s.bc[d][0];
    a->bc[d][1] = s.bc[d][1];
  }
  a->gamma = s.gamma;
  a->cfl = s.cfl;
  a->eps = s.eps;
  a->nlev = s.nlev;
  a->patches = s.patches;
  a->flags = s.flags;
  for (int f = 0; f < NFIELD; ++f) a->inflow[f] = s.inflow[f];
  validate_and_build(*a);
  size_t off = 0;
  for (int l = 0; l < s.nlev; ++l) {
    const Level& L = s.lev[l];
    LevelT<R>& A = a->lev[l];
    for (int f = 0; f < NFIELD; ++f) {
      for (size_t q = 0; q < L.ncell; ++q) A.u[f][q] = R(L.u[f][q]);
      int n[3];
      field_shape(s, l, f, n);
      int m[3];
      for (int d = 0; d < 3; ++d) m[d] = L.per[d] ? L.N[d] : n[d];
      for (int k = 0; k < m[2]; ++k)
        for (int j = 0; j < m[1]; ++j)
          for (int i = 0; i < m[0]; ++i) {
            const size_t q = at(L, i, j, k);
            A.u[f][q] = make_input(L.u[f][q], off + ((size_t)k * n[1] + j) * n[0] + i);
          }
      off += (size_t)n[0] * n[1] * n[2];
    }
  }
  return a;
}

// Visits every level-array entry (the oc_get_field layout, levels then fields,
// periodic face copies included) with its storage value.
template <class R, class Visit> static void visit_state(const Sim& s, const SimT<R>& a, Visit visit) {
  size_t off = 0;
  for (int l = 0; l < s.nlev; ++l) {
    const LevelT<R>& A = a.lev[l];
    for (int f = 0; f < NFIELD; ++f) {
      int n[3];
      field_shape(s, l, f, n);
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) visit(A.u[f][at(A, i, j, k)], off + ((size_t)k * n[1] + j) * n[0] + i);
      off += (size_t)n[0] * n[1] * n[2];
    }
  }
}

extern "C" {

long long oc_state_size(void* h) {
  Sim* s = (Sim*)h;
  long long t = 0;
  for (int l = 0; l < s->nlev; ++l)
    for (int f = 0; f < NFIELD; ++f) t += oc_field_size(h, l, f);
  return t;
}

// Reverse mode: lam0 = (dU_final/dU0)^T lam_final for nsteps coarse steps of the
// given dts (dt is a constant of the differentiated map). Both vectors hold
// every level array in the oc_get_field layout, levels then fields; the entry
// N of a periodic face array is the entry 0 (seeds at both add, and both
// receive the same adjoint). The simulation's own state is not changed.
long long oc_backward(void* h, int nsteps, const double* dts, const double* lam_final, double* lam0) {
  Sim* s = (Sim*)h;
  Tape& T = tape();
  T.clear();
  std::vector<int32_t> input_node((size_t)oc_state_size(h), -1);
  SimT<Rev>* a = clone_as<Rev>(*s, [&](double v, size_t pos) {
    Rev r(v);
    r.i = T.input();
    input_node[pos] = r.i;
    return r;
  });
  for (int i = 0; i < nsteps; ++i) level_substep(*a, 0, 1, dts[i]);
  std::vector<double> adj(T.size(), 0.0);
  visit_state(*s, *a, [&](const Rev& r, size_t pos) {
    if (r.i >= 0) adj[r.i] += lam_final[pos];
  });
  const long long nodes = (long long)T.size();
  T.sweep(adj);
  // every output entry reads the adjoint of the storage input behind it
  SimT<Rev>* b = clone_as<Rev>(*s, [&](double v, size_t pos) {
    Rev r(v);
    r.i = input_node[pos];
    return r;
  });
  visit_state(*s, *b, [&](const Rev& r, size_t pos) { lam0[pos] = r.i >= 0 ? adj[r.i] : 0.0; });
  delete a;
  delete b;
  T.clear();
  std::vector<int32_t>().swap(T.pa);
  std::vector<int32_t>().swap(T.pb);
  std::vector<double>().swap(T.da);
  std::vector<double>().swap(T.db);
  return nodes;
}

// Forward mode: jv = (dU_final/dU0) v0, same layouts (entries N of periodic
// face arrays are ignored in v0, as in oc_set_field).
int oc_tangent(void* h, int nsteps, const double* dts, const double* v0, double* jv) {
  Sim* s = (Sim*)h;
  SimT<Tan>* a = clone_as<Tan>(*s, [&](double v, size_t pos) { return Tan(v, v0[pos]); });
  for (int i = 0; i < nsteps; ++i) level_substep(*a, 0, 1, dts[i]);
  visit_state(*s, *a, [&](const Tan& t, size_t pos) { jv[pos] = t.d; });
  delete a;
  return 0;
}

// Transposed Jacobians of single formulas by the tape (Rev): gx = J^T g.
// The HLLD flux (R4) with x = (ql[7], qr[7], bn).
void oc_hlld_vjp(const double* x, double gamma, double eps, const double* g, double* gx) {
  Tape& T = tape();
  T.clear();
  Rev in[15];
  for (int i = 0; i < 15; ++i) {
    in[i] = Rev(x[i]);
    in[i].i = T.input();
  }
  Rev f[7];
  hlld<Rev>(in, in + 7, in[14], Rev(gamma), Rev(eps), f);
  std::vector<double> adj(T.size(), 0.0);
  for (int o = 0; o < 7; ++o)
    if (f[o].i >= 0) adj[f[o].i] += g[o];
  T.sweep(adj);
  for (int i = 0; i < 15; ++i) gx[i] = adj[in[i].i];
  T.clear();
}

// The half-step predictor of one cell (R1): wh = w - sum_d h_d A_d(w) s_d with
// x = (w[8], s_0[8], .., s_{dim-1}[8]), as the advance forms it.
}  // extern "C"
template <class R> static void predict_cell(int dim, const R* x, double gamma, const double* h, R* wh) {
  const R* w = x;
  R ir = R(1.0) / w[0];
  for (int f = 0; f < 8; ++f) wh[f] = w[f];
  for (int d = 0; d < dim; ++d) {
    R dw[8];
    prim_rhs<R>(w, x + 8 + 8 * d, d, R(gamma), ir, dw);
    for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h[d] * dw[f];
  }
}
extern "C" {
void oc_predict(int dim, const double* x, double gamma, const double* h, double* wh) {
  predict_cell<double>(dim, x, gamma, h, wh);
}
void oc_predict_vjp(int dim, const double* x, double gamma, const double* h, const double* g, double* gx) {
  Tape& T = tape();
  T.clear();
  const int nin = 8 + 8 * dim;
  Rev in[32];
  for (int i = 0; i < nin; ++i) {
    in[i] = Rev(x[i]);
    in[i].i = T.input();
  }
  Rev wh[8];
  predict_cell<Rev>(dim, in, gamma, h, wh);
  std::vector<double> adj(T.size(), 0.0);
  for (int o = 0; o < 8; ++o)
    if (wh[o].i >= 0) adj[wh[o].i] += g[o];
  T.sweep(adj);
  for (int i = 0; i < nin; ++i) gx[i] = adj[in[i].i];
  T.clear();
}

// Stand-alone kernels for pins.
void oc_hlld(const double* ql, const double* qr, double bn, double gamma, double eps, double* f) {
  hlld(ql, qr, bn, gamma, eps, f);
}
void oc_flux(const double* q, double bn, double gamma, double* f) {
  double u[7];
  mhd_flux(q, bn, 1.0 / (gamma - 1.0), f, u);
}
double oc_minmod(double a, double b) { return minmod(a, b); }
// a3: conservative -> primitive recovery of one cell, u = (rho, mx, my, mz, E),
// bc = cell-centred B; w = (rho, vx, vy, vz, p, Bx, By, Bz)
void oc_recover(const double* u, const double* bc, double gamma, double* w) {
  cons_to_prim<double>(u, bc, gamma - 1.0, w);
}
double oc_fast_speed(double rho, double p, double bn, double bt, double bu, double gamma) {
  return fast_speed(rho, p, bn, bt, bu, gamma);
}
double oc_gs_edge(const double* a) {
  return gs_edge_emf(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8], a[9], a[10], a[11]);
}

// Prolongation of one coarse cell's children from a (2*1+1)^dim coarse block
// given as whole-level arrays of a one-level sim: writes the 2^dim children
// cell values of every cell field and all fine faces of the coarse cell into
// a fine scratch sim built by the caller (same domain, base doubled).
int oc_prolong_all(void* hc, void* hf) {
  Sim* c = (Sim*)hc;
  Sim* f = (Sim*)hf;
  Level& C = c->lev[0];
  Level& F = f->lev[0];
  for (int fl = 0; fl < NFIELD; ++fl) C.start[fl] = C.u[fl];
  int cf[6];
  const int ncf = cell_fields(*c, cf);
  for_cells(F, [&](int i, int j, int k) {
    size_t q = at(F, i, j, k);
    for (int n = 0; n < ncf; ++n)
      F.u[cf[n]][q] = prolong_cell(*c, C, cf[n], i >> 1, j >> 1, c->dim == 3 ? k >> 1 : 0, i & 1, j & 1, c->dim == 3 ? (k & 1) : 0);
    for (int d = 0; d < c->dim; ++d) F.u[BX + d][q] = prolong_face(*c, C, F, d, i, j, k);
  });
  return 0;
}

// Restriction of a fine one-level sim onto a coarse one-level sim (all cells
// covered): the R operation alone.
int oc_restrict_all(void* hc, void* hf) {
  Sim* c = (Sim*)hc;
  Sim* f = (Sim*)hf;
  Level& C = c->lev[0];
  Level& F = f->lev[0];
  const double wc = c->dim == 3 ? 0.125 : 0.25;
  const double wf = c->dim == 3 ? 0.25 : 0.5;
  for_cells(C, [&](int i, int j, int k) {
    restrict_cell(*c, C, F, i, j, k, wc);
    for (int d = 0; d < c->dim; ++d) restrict_face(*c, C, F, d, i, j, k, wf);
  });
  return 0;
}

}  // extern "C"
