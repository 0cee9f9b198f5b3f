// Algorithmic floating-point operation count of one cell update, obtained by
// running the oracle's templated per-cell formulas (mhd_core.hpp) with a
// counting scalar type. TEST INFRASTRUCTURE ONLY (see amr_oracle.cpp).
//
// Counted: +, -, *, /, sqrt (one each); negation, fabs, comparisons and
// selections are not counted. Per cell update the algorithm needs, once:
// the recovery of the cell, its slopes, its half-step predictor, its face
// states, the HLLD flux at its dim low faces, its reference EMF, the GS EMF
// at its low edges, and the flux-difference and curl updates. Halo
// recomputation of a patch-based implementation is not algorithmic work.
#include <cstdint>
#include <random>

#include "mhd_core.hpp"

namespace oracle {

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
static long long g_ops = 0;
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
inline Cnt sqrt(Cnt a) { ++g_ops; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }

}  // namespace oracle

using namespace oracle;

extern "C" {

// Count of one conservative-to-primitive recovery (a pin: 19 by hand).
long long oc_flops_recovery() {
  Cnt u[5] = {Cnt(1.1), Cnt(0.2), Cnt(-0.1), Cnt(0.05), Cnt(12.0)}, bc[3] = {Cnt(0.5), Cnt(0.6), Cnt(0.7)}, w[8];
  g_ops = 0;
  cons_to_prim(u, bc, Cnt(2.0 / 3.0), w);
  return g_ops;
}

// Average count over nsample random subsonic face/cell states around
// rho ~ 1, |v| < 0.5, p in [0.1, 10], |B| ~ 0.6 (the blast workload's range).
double oc_flops_per_cell_update(int dim, int nsample, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const Cnt gamma(5.0 / 3.0), gm1(2.0 / 3.0), eps(1e-12);
  long long tot = 0;
  for (int s = 0; s < nsample; ++s) {
    auto state = [&](Cnt* w) {
      w[0] = 1.0 + 0.5 * U(rng); w[1] = 0.5 * U(rng); w[2] = 0.5 * U(rng); w[3] = 0.5 * U(rng);
      w[4] = 5.05 + 4.95 * U(rng); w[5] = 0.6 + 0.2 * U(rng); w[6] = 0.6 + 0.2 * U(rng); w[7] = 0.6 + 0.2 * U(rng);
    };
    g_ops = 0;
    // recovery: B_c means (3 x 2), then cons_to_prim
    Cnt u[5] = {Cnt(1.1), Cnt(0.2), Cnt(-0.1), Cnt(0.05), Cnt(12.0)};
    Cnt bl[3] = {Cnt(0.5), Cnt(0.6), Cnt(0.7)}, br[3] = {Cnt(0.55), Cnt(0.58), Cnt(0.71)};
    Cnt bc[3], w[8];
    for (int d = 0; d < 3; ++d) bc[d] = Cnt(0.5) * (bl[d] + br[d]);
    cons_to_prim(u, bc, gm1, w);
    // slopes: per direction 7 limited components (2 differences each) + the normal B difference
    Cnt sl[3][8];
    for (int d = 0; d < dim; ++d)
      for (int f = 0; f < 8; ++f) {
        Cnt a = w[f] - Cnt(w[f].v * 0.98), b = Cnt(w[f].v * 1.01) - w[f];
        if (f == BX + d) { sl[d][f] = b; g_ops--; }  // the normal B slope is one difference
        else sl[d][f] = minmod(a, b);
      }
    // predictor
    Cnt ir = Cnt(1) / w[0], wh[8], dw[8];
    for (int f = 0; f < 8; ++f) wh[f] = w[f];
    for (int d = 0; d < dim; ++d) {
      prim_rhs(w, sl[d], d, gamma, ir, dw);
      for (int f = 0; f < 8; ++f) wh[f] = wh[f] - Cnt(0.01) * dw[f];
    }
    // face states of the cell (2 per direction)
    for (int d = 0; d < dim; ++d)
      for (int f = 0; f < 8; ++f) { Cnt a = wh[f] + Cnt(0.5) * sl[d][f]; Cnt b = wh[f] - Cnt(0.5) * sl[d][f]; (void)a; (void)b; }
    // HLLD at the dim low faces (normal field = mean of the two face states)
    for (int d = 0; d < dim; ++d) {
      Cnt wl[8], wr[8];
      state(wl);
      state(wr);
      Cnt bn = Cnt(0.5) * (wl[5] + wr[5]);
      Cnt ql[7] = {wl[0], wl[1], wl[2], wl[3], wl[4], wl[6], wl[7]};
      Cnt qr[7] = {wr[0], wr[1], wr[2], wr[3], wr[4], wr[6], wr[7]};
      Cnt f7[7];
      hlld(ql, qr, bn, gamma, eps, f7);
    }
    // reference EMF (3 components in 3D, 1 in 2D; 3 ops each)
    g_ops += dim == 3 ? 9 : 3;
    // GS edge EMFs at the low edges
    const int nedge = dim == 3 ? 3 : 1;
    for (int e = 0; e < nedge; ++e) {
      Cnt a[12];
      for (int k = 0; k < 8; ++k) a[k] = Cnt(0.1 * U(rng));
      for (int k = 8; k < 12; ++k) a[k] = Cnt(U(rng));
      gs_edge_emf(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8], a[9], a[10], a[11]);
    }
    // updates: cell fields (sub, mul, sub per direction) and the dim faces (two terms each)
    const int ncf = dim == 3 ? 5 : 6;
    g_ops += (long long)ncf * dim * 3;
    g_ops += dim == 3 ? 3 * 2 * 3 : 2 * 1 * 3;
    tot += g_ops;
  }
  return (double)tot / nsample;
}

}  // extern "C"
