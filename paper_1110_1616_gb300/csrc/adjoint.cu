// Discrete adjoint of the AMR level advance: the exact transpose of the
// linearised forward map of whole coarse steps for a fixed dt sequence
// (dt is a constant, not differentiated), with checkpoints every k coarse steps
// and recomputation inside each segment. C-ABI: amrmhd_step_dt, amrmhd_backward.
//
// Forward map of one level sub-step (Sec. 4: P, A, S, R), as the adjoint sees it:
//   X_l = fill(state_l, X_{l-1})         ghost copies, prolongation, boundaries
//   Y_l = advance(X_l)                   interior + w ghost layers
//   registers += dt F(X_l), dt E(X_l)    on the C/F faces and edges
//   (children), then Y_l = reflux_restrict(Y_l, registers, Y_{l+1})
// The reverse sweep visits the sub-steps in the opposite order and applies the
// transposes: of reflux/restriction (scatter to the registers and the fine
// level), of the advance stage by stage (update, EMF, HLLD, predictor and
// slopes, recovery), and of the fill (scatter-add of every copied or
// prolonged ghost value to its sources). The transposed Jacobians of the two
// costliest pointwise formulas (HLLD, the half-step predictor, the recovery)
// are written by hand (adjoint_local.cuh); that of the edge EMF comes from the
// same templated device formula as the forward evaluated with forward-mode
// dual numbers (dual numbers are also kept for HLLD and the predictor, as the
// cross-check of amrmhd_local_vjp); branches (minmod, HLLD cases, upwinding)
// take the forward's decisions. Adjoint arithmetic is FP64 in both precision modes, at the forward
// trajectory of the context's precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.hpp"
#include "mhd_device.cuh"
#include "adjoint_local.cuh"

// ------------------------------------------------------------------ dual numbers
namespace amrdev {

template <int K> struct Dn {
  double v;
  double d[K];
  __device__ __forceinline__ Dn() : v(0.0) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ Dn(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  friend __device__ __forceinline__ Dn operator+(const Dn& a, const Dn& b) {
    Dn r(a.v + b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
  }
  friend __device__ __forceinline__ Dn operator-(const Dn& a, const Dn& b) {
    Dn r(a.v - b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
  }
  friend __device__ __forceinline__ Dn operator-(const Dn& a) {
    Dn r(-a.v);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
  }
  friend __device__ __forceinline__ Dn operator*(const Dn& a, const Dn& b) {
    Dn r(a.v * b.v);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
  }
  friend __device__ __forceinline__ Dn operator/(const Dn& a, const Dn& b) {
    const double q = a.v / b.v, ib = 1.0 / b.v;
    Dn r(q);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - q * b.d[k]) * ib;
    return r;
  }
  friend __device__ __forceinline__ bool operator<(const Dn& a, const Dn& b) { return a.v < b.v; }
  friend __device__ __forceinline__ bool operator>(const Dn& a, const Dn& b) { return a.v > b.v; }
  friend __device__ __forceinline__ bool operator<=(const Dn& a, const Dn& b) { return a.v <= b.v; }
  friend __device__ __forceinline__ bool operator>=(const Dn& a, const Dn& b) { return a.v >= b.v; }
};
template <int K> __device__ __forceinline__ Dn<K> dsqrt(const Dn<K>& a) {
  const double r = sqrt(a.v);
  Dn<K> o(r);
  const double h = 0.5 / r;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] * h;
  return o;
}
template <int K> __device__ __forceinline__ Dn<K> dabs(const Dn<K>& a) {
  const double s = a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0);
  Dn<K> o(fabs(a.v));
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] * s;
  return o;
}
template <int K> struct Eps<Dn<K>> {
  static __device__ __forceinline__ Dn<K> v() { return Dn<K>(1e-12); }
};

// J^T g of fn: R^NIN -> R^NOUT at x, by forward-mode chunks of K tangents
template <int NIN, int NOUT, int K, class Fn>
__device__ __forceinline__ void vjp(const double* x, const double* g, double* gx, const Fn& fn) {
#pragma unroll 1
  for (int c0 = 0; c0 < NIN; c0 += K) {
    Dn<K> in[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
      in[i] = Dn<K>(x[i]);
      if (i >= c0 && i < c0 + K) in[i].d[i - c0] = 1.0;
    }
    Dn<K> out[NOUT];
    fn(in, out);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (c0 + k >= NIN) break;
      double s = 0.0;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) s += g[o] * out[o].d[k];
      gx[c0 + k] = s;
    }
  }
}

}  // namespace amrdev

namespace amradj {
using namespace amrk;
using namespace amrdev;

constexpr int TPB = 256;
__host__ __device__ __forceinline__ int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

struct AdjArgs {
  const DPatch* P;   // patch table with the adjoint workspace's scratch offsets
  const int* ids;
  int npatch;
  int maxn[3];
  const void* X;     // the filled forward state of the level (T), by P.off
  const void* scr;   // forward stage arrays recomputed from X (T), by P.soff
  double* lam;       // adjoint of the advanced state
  double* lamx;      // adjoint accumulator of the filled state X
  double* lscr;      // adjoint stage arrays, by P.soff
  const double* dtp;
  double dtscale;
  double idx[3];
  double gamma;
  int w;
};

struct AdjRows {
  const DPatch* P;
  const int* rows;
  long long nrows;
  double* lam;        // adjoint of the level the rows write (fill: the level; reflux: the coarse level)
  double* lamf;       // reflux/restriction: adjoint of the fine level
  double* lamc;       // prolongation: adjoint accumulator of the coarse filled state
  const void* Xc;     // prolongation: coarse filled state (T)
  double* lscr;       // register seeds
  double* lR;         // adjoint of R = (S1 + S2) - C per C/F face row (x 6), rows of this level
  double* lRE;        // the same per C/F edge row
  const double* dtp;
  double dtscale;
  double idx[3];      // coarse 1/dx
  double ratio[3][3]; // coarse dx_n / dx_t
  int substep;
};

__device__ __forceinline__ int lidx(const DPatch& P, int i, int j, int k) { return i + P.ext[0] * (j + P.ext[1] * k); }
template <int DIM> __device__ __forceinline__ int stride_of(const DPatch& P, int d) {
  return d == 0 ? 1 : (d == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
}
template <int DIM>
__device__ __forceinline__ bool region_cell(const DPatch& P, int m, int t, int& i, int& j, int& k) {
  const int rx = P.n[0] + 2 * m, ry = P.n[1] + 2 * m, rz = DIM == 3 ? P.n[2] + 2 * m : 1;
  if (t >= rx * ry * rz) return false;
  i = 4 - m + t % rx;
  j = 4 - m + (t / rx) % ry;
  k = DIM == 3 ? 4 - m + t / (rx * ry) : 0;
  return true;
}
// storage coordinates of local index L
__device__ __forceinline__ void coords(const DPatch& P, int L, int* c) {
  c[0] = L % P.ext[0];
  c[1] = (L / P.ext[0]) % P.ext[1];
  c[2] = L / (P.ext[0] * P.ext[1]);
}
// cell in the update region (interior widened by w)?
template <int DIM> __device__ __forceinline__ bool in_upd(const DPatch& P, int w, const int* c) {
#pragma unroll
  for (int e = 0; e < DIM; ++e)
    if (c[e] < 4 - w || c[e] >= P.n[e] + 4 + w) return false;
  return true;
}
// d-face updated by the advance: normal index in [4-w, n+4+w], transverse in [4-w, n+4+w)
template <int DIM> __device__ __forceinline__ bool face_upd(const DPatch& P, int w, int d, const int* c) {
#pragma unroll
  for (int e = 0; e < DIM; ++e) {
    const int hi = P.n[e] + 4 + w + (e == d ? 1 : 0);
    if (c[e] < 4 - w || c[e] >= hi) return false;
  }
  return true;
}
__device__ __forceinline__ void aadd(double* p, double v) {
  if (v != 0.0) atomicAdd(p, v);
}
template <class T, int DIM> struct CF {
  static constexpr int N = DIM == 3 ? 5 : 6;
  static __device__ __forceinline__ int f(int n) { return n < 5 ? n : BZ; }
};

// ------------------------------------------------------------------ advance transpose
// update: cells of region w are the identity plus flux differences
template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_adj_update_cells(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    a.lamx[P.off + f * P.fs + L] += a.lam[P.off + f * P.fs + L];
  }
}

// updated d-faces: identity; the flux seeds of the same faces (cell-field
// fluxes feed the two adjacent cells of region w)
template <class T, int DIM, int D> __global__ void __launch_bounds__(TPB) k_adj_faces(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  const int w = a.w;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : (e == D ? P.n[e] + 2 * w + 1 : P.n[e] + 2 * w + 2);
  const int t = blockIdx.x * TPB + threadIdx.x;
  if (t >= r[0] * r[1] * r[2]) return;
  int c[3] = {t % r[0], (t / r[0]) % r[1], t / (r[0] * r[1])};
#pragma unroll
  for (int e = 0; e < 3; ++e) c[e] = e >= DIM ? 0 : c[e] + (e == D ? 4 - w : 3 - w);
  const int L = lidx(P, c[0], c[1], c[2]);
  const int sd = stride_of<DIM>(P, D);
  if (face_upd<DIM>(P, w, D, c)) a.lamx[P.off + (BX + D) * P.fs + L] += a.lam[P.off + (BX + D) * P.fs + L];
  int cm[3] = {c[0], c[1], c[2]};
  cm[D] -= 1;
  const bool hi_in = in_upd<DIM>(P, w, c), lo_in = in_upd<DIM>(P, w, cm);
  const double dtd = *a.dtp * a.dtscale * a.idx[D];
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    double g = 0.0;
    if (hi_in) g += a.lam[P.off + f * P.fs + L];
    if (lo_in) g -= a.lam[P.off + f * P.fs + L - sd];
    a.lscr[P.soff + (SC_F + 8 * D + f) * P.fs + L] = dtd * g;
  }
}

// edge EMF seeds from the curl update of the adjacent updated faces
template <class T, int DIM, int C> __global__ void __launch_bounds__(TPB) k_adj_emf_seed(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  const int w = a.w;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : (e == C ? P.n[e] + 2 * w : P.n[e] + 2 * w + 1);
  const int t = blockIdx.x * TPB + threadIdx.x;
  if (t >= r[0] * r[1] * r[2]) return;
  int c[3] = {t % r[0], (t / r[0]) % r[1], t / (r[0] * r[1])};
#pragma unroll
  for (int e = 0; e < 3; ++e) c[e] = e >= DIM ? 0 : c[e] + 4 - w;
  const int L = lidx(P, c[0], c[1], c[2]);
  const double dt = *a.dtp * a.dtscale;
  const double dtd[3] = {dt * a.idx[0], dt * a.idx[1], dt * a.idx[2]};
  // face (d) at the edge's cell shifted by -1 along s (s < 0: not shifted)
  auto lam_face = [&](int d, int s) -> double {
    int cc[3] = {c[0], c[1], c[2]};
    int LL = L;
    if (s >= 0) {
      cc[s] -= 1;
      LL -= stride_of<DIM>(P, s);
    }
    return face_upd<DIM>(P, w, d, cc) ? a.lam[P.off + (BX + d) * P.fs + LL] : 0.0;
  };
  double g;
  if (C == 2) {
    g = dtd[1] * (lam_face(0, -1) - lam_face(0, 1)) + dtd[0] * (lam_face(1, 0) - lam_face(1, -1));
  } else if (C == 1) {
    g = dtd[2] * (lam_face(0, 2) - lam_face(0, -1)) + dtd[0] * (lam_face(2, -1) - lam_face(2, 0));
  } else {
    g = dtd[2] * (lam_face(1, -1) - lam_face(1, 2)) + dtd[1] * (lam_face(2, 1) - lam_face(2, -1));
  }
  a.lscr[P.soff + (SC_E + C) * P.fs + L] = g;
}

struct GsFn {
  double fa_lo, fa_hi, fb_lo, fb_hi;
  template <class V> __device__ __forceinline__ void operator()(const V* x, V* y) const {
    y[0] = gs_emf<V>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], V(fa_lo), V(fa_hi), V(fb_lo), V(fb_hi));
  }
};

// edge EMF: E = GS(ea_lo, ea_hi, eb_lo, eb_hi, r00, r10, r01, r11; mass-flux signs)
template <class T, int DIM, int C> __global__ void __launch_bounds__(TPB) k_adj_emf(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  const int w = a.w;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : (e == C ? P.n[e] + 2 * w : P.n[e] + 2 * w + 1);
  const int t = blockIdx.x * TPB + threadIdx.x;
  if (t >= r[0] * r[1] * r[2]) return;
  int c[3] = {t % r[0], (t / r[0]) % r[1], t / (r[0] * r[1])};
#pragma unroll
  for (int e = 0; e < 3; ++e) c[e] = e >= DIM ? 0 : c[e] + 4 - w;
  constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
  const int L = lidx(P, c[0], c[1], c[2]);
  const long long fs = P.fs;
  const double g = a.lscr[P.soff + (SC_E + C) * fs + L];
  if (g == 0.0) return;
  const int sa = stride_of<DIM>(P, A), sb = stride_of<DIM>(P, B);
  const T* S = (const T*)a.scr + P.soff;
  const T* Fa = S + (SC_F + 8 * A) * fs;
  const T* Fb = S + (SC_F + 8 * B) * fs;
  const T* R = S + (SC_REF + C) * fs;
  const int q11 = L, q01 = L - sa, q10 = L - sb, q00 = L - sa - sb;
  const double x[8] = {-(double)Fa[(BX + B) * fs + q10], -(double)Fa[(BX + B) * fs + q11],
                       (double)Fb[(BX + A) * fs + q01],  (double)Fb[(BX + A) * fs + q11],
                       (double)R[q00], (double)R[q10], (double)R[q01], (double)R[q11]};
  GsFn fn{(double)Fa[q10], (double)Fa[q11], (double)Fb[q01], (double)Fb[q11]};
  double gx[8];
  vjp<8, 1, 8>(x, &g, gx, fn);
  double* lF = a.lscr + P.soff;
  aadd(lF + (SC_F + 8 * A + BX + B) * fs + q10, -gx[0]);
  aadd(lF + (SC_F + 8 * A + BX + B) * fs + q11, -gx[1]);
  aadd(lF + (SC_F + 8 * B + BX + A) * fs + q01, gx[2]);
  aadd(lF + (SC_F + 8 * B + BX + A) * fs + q11, gx[3]);
  aadd(lF + (SC_REF + C) * fs + q00, gx[4]);
  aadd(lF + (SC_REF + C) * fs + q10, gx[5]);
  aadd(lF + (SC_REF + C) * fs + q01, gx[6]);
  aadd(lF + (SC_REF + C) * fs + q11, gx[7]);
}

struct HlldFn {
  double gamma;
  template <class V> __device__ __forceinline__ void operator()(const V* x, V* y) const {
    hlld_flux<V>(x, x + 7, x[14], V(gamma), y);
  }
};

// HLLD at d-faces: inputs the rotated predicted face states and the mean normal field
template <class T, int DIM, int D> __global__ void __launch_bounds__(TPB) k_adj_flux(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  const int w = a.w;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : (e == D ? P.n[e] + 2 * w + 1 : P.n[e] + 2 * w + 2);
  const int t = blockIdx.x * TPB + threadIdx.x;
  if (t >= r[0] * r[1] * r[2]) return;
  int c[3] = {t % r[0], (t / r[0]) % r[1], t / (r[0] * r[1])};
#pragma unroll
  for (int e = 0; e < 3; ++e) c[e] = e >= DIM ? 0 : c[e] + (e == D ? 4 - w : 3 - w);
  const int L = lidx(P, c[0], c[1], c[2]);
  const int Ll = L - stride_of<DIM>(P, D);
  const long long fs = P.fs;
  constexpr int n = D, tt = (D + 1) % 3, uu = (D + 2) % 3;
  double* lS = a.lscr + P.soff;
  const double* lF = lS + (SC_F + 8 * D) * fs + L;
  const double g[7] = {lF[RHO * fs], lF[(MX + n) * fs], lF[(MX + tt) * fs], lF[(MX + uu) * fs],
                       lF[EN * fs], lF[(BX + tt) * fs], lF[(BX + uu) * fs]};
  bool any = false;
#pragma unroll
  for (int o = 0; o < 7; ++o) any |= g[o] != 0.0;
  if (!any) return;
  const T* S = (const T*)a.scr + P.soff;
  T wl[8], wr[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    wl[f] = S[(SC_WH + f) * fs + Ll] + T(0.5) * S[(SC_S + 8 * D + f) * fs + Ll];
    wr[f] = S[(SC_WH + f) * fs + L] - T(0.5) * S[(SC_S + 8 * D + f) * fs + L];
  }
  const T bn = T(0.5) * (wl[5 + n] + wr[5 + n]);
  // local Jacobian in the forward's compute type T (FP32 in mixed precision)
  const T x[15] = {wl[0], wl[1 + n], wl[1 + tt], wl[1 + uu], wl[4], wl[5 + tt], wl[5 + uu],
                   wr[0], wr[1 + n], wr[1 + tt], wr[1 + uu], wr[4], wr[5 + tt], wr[5 + uu], bn};
  T gt[7], gx[15];
#pragma unroll
  for (int o = 0; o < 7; ++o) gt[o] = (T)g[o];
  hlld_vjp<T>(x, gt, (T)a.gamma, gx);
  double gl[8], gr[8];
  gl[0] = gx[0]; gl[1 + n] = gx[1]; gl[1 + tt] = gx[2]; gl[1 + uu] = gx[3]; gl[4] = gx[4];
  gl[5 + tt] = gx[5]; gl[5 + uu] = gx[6]; gl[5 + n] = 0.5 * gx[14];
  gr[0] = gx[7]; gr[1 + n] = gx[8]; gr[1 + tt] = gx[9]; gr[1 + uu] = gx[10]; gr[4] = gx[11];
  gr[5 + tt] = gx[12]; gr[5 + uu] = gx[13]; gr[5 + n] = 0.5 * gx[14];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    aadd(lS + (SC_WH + f) * fs + Ll, gl[f]);
    aadd(lS + (SC_S + 8 * D + f) * fs + Ll, 0.5 * gl[f]);
    aadd(lS + (SC_WH + f) * fs + L, gr[f]);
    aadd(lS + (SC_S + 8 * D + f) * fs + L, -0.5 * gr[f]);
  }
}

// half-step predictor wh = w - sum_d h_d A_d(w) s_d as a function of (w, s)
template <int DIM> struct PredFn {
  double gamma, h[3];
  template <class V> __device__ __forceinline__ void operator()(const V* x, V* y) const {
    const V* w = x;
    const V ir = V(1.0) / w[0];
    const V g = V(gamma);
    V wh[8], dw[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = w[f];
    prim_terms<V, 0>(w, x + 8, g, ir, dw);
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = wh[f] - V(h[0]) * dw[f];
    prim_terms<V, 1>(w, x + 16, g, ir, dw);
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = wh[f] - V(h[1]) * dw[f];
    if (DIM == 3) {
      prim_terms<V, 2>(w, x + 24, g, ir, dw);
#pragma unroll
      for (int f = 0; f < 8; ++f) wh[f] = wh[f] - V(h[2]) * dw[f];
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) y[f] = wh[f];
  }
};

template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_adj_predict(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w + 1, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const long long fs = P.fs;
  const T* S = (const T*)a.scr + P.soff;
  double* lS = a.lscr + P.soff;
  double gwh[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) gwh[f] = lS[(SC_WH + f) * fs + L];
  {  // reference EMF -(v x B) at the half step
    const double r0 = lS[(SC_REF + 0) * fs + L], r1 = lS[(SC_REF + 1) * fs + L], r2 = lS[(SC_REF + 2) * fs + L];
    double wh[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = (double)S[(SC_WH + f) * fs + L];
    gwh[3] += r0 * wh[6] - r1 * wh[5];
    gwh[6] += r0 * wh[3] - r2 * wh[1];
    gwh[2] += -r0 * wh[7] + r2 * wh[5];
    gwh[7] += -r0 * wh[2] + r1 * wh[1];
    gwh[1] += r1 * wh[7] - r2 * wh[6];
    gwh[5] += -r1 * wh[3] + r2 * wh[2];
  }
  constexpr int NIN = 8 + 8 * DIM;
  // local Jacobian in the forward's compute type T (FP32 in mixed precision)
  T x[NIN], gxt[NIN], gt[8];
  double gx[NIN];
#pragma unroll
  for (int f = 0; f < 8; ++f) x[f] = S[(SC_W + f) * fs + L];
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int f = 0; f < 8; ++f) x[8 + 8 * d + f] = S[(SC_S + 8 * d + f) * fs + L];
  bool any = false;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    any |= gwh[f] != 0.0;
    gt[f] = (T)gwh[f];
  }
  const double dt = *a.dtp * a.dtscale;
  T h[3];
  for (int d = 0; d < 3; ++d) h[d] = (T)(0.5 * dt * a.idx[d]);
  if (any) {
    predict_vjp<DIM, T>(x, gt, (T)a.gamma, h, gxt);
#pragma unroll
    for (int q = 0; q < NIN; ++q) gx[q] = (double)gxt[q];
  } else {
#pragma unroll
    for (int q = 0; q < NIN; ++q) gx[q] = 0.0;
  }
  // W of the cell
  double* lW = lS + SC_W * fs;
#pragma unroll
  for (int f = 0; f < 8; ++f) aadd(lW + f * fs + L, gx[f]);
  // slopes: stored slope adjoint plus the predictor's
  const T* W = S + SC_W * fs;
  const T* U = (const T*)a.X + P.off;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = stride_of<DIM>(P, d);
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      const double gs = gx[8 + 8 * d + f] + lS[(SC_S + 8 * d + f) * fs + L];
      if (gs == 0.0) continue;
      if (f == BX + d) {  // face difference of the normal field
        aadd(a.lamx + P.off + (BX + d) * P.fs + L + sd, gs);
        aadd(a.lamx + P.off + (BX + d) * P.fs + L, -gs);
        continue;
      }
      const T wc = W[f * fs + L];
      const T aa = wc - W[f * fs + L - sd], bb = W[f * fs + L + sd] - wc;
      int br = 0;  // minmod branch of the forward: 1 = a, 2 = b, 0 = zero
      if (aa > T(0) && bb > T(0)) br = (aa <= bb) ? 1 : 2;
      else if (aa < T(0) && bb < T(0)) br = (aa >= bb) ? 1 : 2;
      if (br == 1) {
        aadd(lW + f * fs + L, gs);
        aadd(lW + f * fs + L - sd, -gs);
      } else if (br == 2) {
        aadd(lW + f * fs + L + sd, gs);
        aadd(lW + f * fs + L, -gs);
      }
    }
  }
  (void)U;
}

// recovery W(U) on region w+2; cell-centred B from the two faces
template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_adj_prim(AdjArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w + 2, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const long long fs = P.fs;
  const double* lW = a.lscr + P.soff + SC_W * fs;
  double g[8];
  bool any = false;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    g[f] = lW[f * fs + L];
    any |= g[f] != 0.0;
  }
  if (!any) return;
  const T* U = (const T*)a.X + P.off;
  double x[8];
#pragma unroll
  for (int f = 0; f < 5; ++f) x[f] = (double)U[f * fs + L];
  x[5] = 0.5 * ((double)U[5 * fs + L] + (double)U[5 * fs + L + 1]);
  x[6] = 0.5 * ((double)U[6 * fs + L] + (double)U[6 * fs + L + P.ext[0]]);
  if (DIM == 3) x[7] = 0.5 * ((double)U[7 * fs + L] + (double)U[7 * fs + L + P.ext[0] * P.ext[1]]);
  else x[7] = (double)U[7 * fs + L];
  double gx[8];
  recover_vjp(x, g, a.gamma - 1.0, gx);
  double* lx = a.lamx + P.off;
#pragma unroll
  for (int f = 0; f < 5; ++f) aadd(lx + f * fs + L, gx[f]);
  aadd(lx + 5 * fs + L, 0.5 * gx[5]);
  aadd(lx + 5 * fs + L + 1, 0.5 * gx[5]);
  aadd(lx + 6 * fs + L, 0.5 * gx[6]);
  aadd(lx + 6 * fs + L + P.ext[0], 0.5 * gx[6]);
  if (DIM == 3) {
    aadd(lx + 7 * fs + L, 0.5 * gx[7]);
    aadd(lx + 7 * fs + L + P.ext[0] * P.ext[1], 0.5 * gx[7]);
  } else {
    aadd(lx + 7 * fs + L, gx[7]);
  }
}

// ------------------------------------------------------------------ register seeds
// coarse side: C = dt F_c on the coarse face, R = (S1 + S2) - C  =>  dF_c -= dt lR
template <class T, int DIM> __global__ void k_adj_regc_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[1]];
  const int d = row[2], L = row[3];
  const double dt = *a.dtp * a.dtscale;
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n)
    aadd(a.lscr + P.soff + (SC_F + 8 * d + CF<T, DIM>::f(n)) * P.fs + L, -dt * a.lR[r * 6 + n]);
}
template <class T, int DIM> __global__ void k_adj_regc_edges(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[1]];
  const double dt = *a.dtp * a.dtscale;
  aadd(a.lscr + P.soff + (SC_E + row[2]) * P.fs + row[3], -dt * a.lRE[r]);
}
// fine side: S_s = dt 2^-(dim-1) tree sum of the sub-faces
template <class T, int DIM> __global__ void k_adj_regf_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[5]];
  const int d = row[2], L = row[6];
  const double af = *a.dtp * a.dtscale * (DIM == 3 ? 0.25 : 0.5);
  const int sx = 1, sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  int o[4] = {0, 0, 0, 0};
  int m;
  if (DIM == 2) {
    o[1] = d == 0 ? sy : sx;
    m = 2;
  } else {
    if (d == 0) { o[1] = sy; o[2] = sz; o[3] = sy + sz; }
    else if (d == 1) { o[1] = sx; o[2] = sz; o[3] = sx + sz; }
    else { o[1] = sx; o[2] = sy; o[3] = sx + sy; }
    m = 4;
  }
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const double g = af * a.lR[r * 6 + n];
    double* base = a.lscr + P.soff + (SC_F + 8 * d + CF<T, DIM>::f(n)) * P.fs + L;
    for (int s = 0; s < m; ++s) aadd(base + o[s], g);
  }
}
template <class T, int DIM> __global__ void k_adj_regf_edges(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[4]];
  const int c = row[2], L = row[5];
  const double dt = *a.dtp * a.dtscale;
  double* base = a.lscr + P.soff + (SC_E + c) * P.fs + L;
  if (DIM == 3) {
    const int sc = c == 0 ? 1 : (c == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
    const double g = dt * 0.5 * a.lRE[r];
    aadd(base, g);
    aadd(base + sc, g);
  } else {
    aadd(base, dt * a.lRE[r]);
  }
}

// ------------------------------------------------------------------ reflux / restriction transpose
template <class T, int DIM> __global__ void k_adj_restrict_cells(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 5 * r;
  const DPatch C = a.P[row[1]], F = a.P[row[3]];
  const int sy = F.ext[0], sz = F.ext[0] * F.ext[1];
  const double wc = DIM == 3 ? 0.125 : 0.25;
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    double* lc = a.lam + C.off + f * C.fs + row[2];
    const double g = *lc * wc;
    *lc = 0.0;
    double* lf = a.lamf + F.off + f * F.fs + row[4];
    aadd(lf, g);
    aadd(lf + 1, g);
    aadd(lf + sy, g);
    aadd(lf + sy + 1, g);
    if (DIM == 3) {
      aadd(lf + sz, g);
      aadd(lf + sz + 1, g);
      aadd(lf + sz + sy, g);
      aadd(lf + sz + sy + 1, g);
    }
  }
}
template <class T, int DIM> __global__ void k_adj_restrict_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch C = a.P[row[1]], F = a.P[row[4]];
  const int d = row[2];
  double* lc = a.lam + C.off + (BX + d) * C.fs + row[3];
  const double g = *lc * (DIM == 3 ? 0.25 : 0.5);
  *lc = 0.0;
  double* lf = a.lamf + F.off + (BX + d) * F.fs + row[5];
  const int sx = 1, sy = F.ext[0], sz = F.ext[0] * F.ext[1];
  if (DIM == 2) {
    aadd(lf, g);
    aadd(lf + (d == 0 ? sy : sx), g);
  } else {
    int o1, o2;
    if (d == 0) { o1 = sy; o2 = sz; }
    else if (d == 1) { o1 = sx; o2 = sz; }
    else { o1 = sx; o2 = sy; }
    aadd(lf, g);
    aadd(lf + o1, g);
    aadd(lf + o2, g);
    aadd(lf + o1 + o2, g);
  }
}
// reflux of uncovered coarse cells: U +/- R idx per slot (rows hold global C/F row numbers)
template <class T, int DIM> __global__ void k_adj_reflux_cells(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 9 * r;
  const DPatch P = a.P[row[1]];
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const double g = a.lam[P.off + CF<T, DIM>::f(n) * P.fs + row[2]];
    if (g == 0.0) continue;
    for (int slot = 0; slot < 2 * DIM; ++slot) {
      const int e = row[3 + slot];
      if (e < 0) continue;
      const double c = (slot & 1) ? -a.idx[slot >> 1] : a.idx[slot >> 1];
      aadd(a.lR + (long long)e * 6 + n, c * g);
    }
  }
}
// EMF correction of uncovered coarse faces: B += +e0/dx_t1 - e1/dx_t1 - e2/dx_t2 + e3/dx_t2
template <class T, int DIM> __global__ void k_adj_reflux_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 8 * r;
  const DPatch P = a.P[row[1]];
  const int d = row[2];
  const double g = a.lam[P.off + (BX + d) * P.fs + row[3]];
  if (g == 0.0) return;
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  for (int slot = 0; slot < 4; ++slot) {
    const int e = row[4 + slot];
    if (e < 0) continue;
    const double c = slot == 0 ? a.idx[t1] : slot == 1 ? -a.idx[t1] : slot == 2 ? -a.idx[t2] : a.idx[t2];
    aadd(a.lRE + e, c * g);
  }
}

// ------------------------------------------------------------------ fill transpose
template <class T, int DIM> __global__ void k_adj_same_cells(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 4 * r;
  const DPatch D = a.P[row[0]], S = a.P[row[2]];
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    double* ld = a.lam + D.off + f * D.fs + row[1];
    const double g = *ld;
    *ld = 0.0;
    aadd(a.lam + S.off + f * S.fs + row[3], g);
  }
}
template <class T, int DIM> __global__ void k_adj_same_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 5 * r;
  const DPatch D = a.P[row[0]], S = a.P[row[3]];
  const int f = BX + row[1];
  double* ld = a.lam + D.off + f * D.fs + row[2];
  const double g = *ld;
  *ld = 0.0;
  aadd(a.lam + S.off + f * S.fs + row[4], g);
}
template <class T, int DIM> __global__ void k_adj_bc_cells(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 5 * r;
  const DPatch D = a.P[row[0]];
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    double* ld = a.lam + D.off + f * D.fs + row[1];
    const double g = *ld;
    *ld = 0.0;
    if (row[2] == 2) aadd(a.lam + D.off + f * D.fs + row[4], g);
  }
}
template <class T, int DIM> __global__ void k_adj_bc_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch D = a.P[row[0]];
  const int f = BX + row[1];
  double* ld = a.lam + D.off + f * D.fs + row[2];
  const double g = *ld;
  *ld = 0.0;
  if (row[3] == 2) aadd(a.lam + D.off + f * D.fs + row[5], g);
}

// minmod(u0 - u[-s], u[s] - u0) scaled by c, transposed: adds g c dmm/du to the three values
template <class T>
__device__ __forceinline__ void mm_adj(const T* u, double* lu, int s, double gc) {
  const T u0 = u[0];
  const T aa = u0 - u[-s], bb = u[s] - u0;
  int br = 0;
  if (aa > T(0) && bb > T(0)) br = (aa <= bb) ? 1 : 2;
  else if (aa < T(0) && bb < T(0)) br = (aa >= bb) ? 1 : 2;
  if (br == 1) {
    aadd(lu, gc);
    aadd(lu - s, -gc);
  } else if (br == 2) {
    aadd(lu + s, gc);
    aadd(lu, -gc);
  }
}

template <int DIM> __device__ __forceinline__ void global_pos(const DPatch& P, int L, int* g) {
  int c[3];
  coords(P, L, c);
  g[0] = P.lo[0] + c[0] - 4;
  g[1] = P.lo[1] + c[1] - 4;
  g[2] = DIM == 3 ? P.lo[2] + c[2] - 4 : 0;
}

// prolonged cells: v = u0 + sum_d minmod-slope_d (+-1/4)
template <class T, int DIM> __global__ void k_adj_prolong_cells(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 4 * r;
  const DPatch D = a.P[row[0]], C = a.P[row[2]];
  int g[3];
  global_pos<DIM>(D, row[1], g);
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
#pragma unroll
  for (int n = 0; n < CF<T, DIM>::N; ++n) {
    const int f = CF<T, DIM>::f(n);
    double* ld = a.lam + D.off + f * D.fs + row[1];
    const double gv = *ld;
    *ld = 0.0;
    if (gv == 0.0) continue;
    const T* u = (const T*)a.Xc + C.off + f * C.fs + row[3];
    double* lu = a.lamc + C.off + f * C.fs + row[3];
    aadd(lu, gv);
#pragma unroll
    for (int d = 0; d < DIM; ++d) mm_adj<T>(u, lu, st[d], gv * ((g[d] & 1) ? 0.25 : -0.25));
  }
}

// B_n on the coarse n-face b prolonged to the fine sub-face with parities par, transposed
template <class T, int DIM>
__device__ __forceinline__ void coincident_adj(const T* b, double* lb, const int* st, int n, const int* par, double gv) {
  aadd(lb, gv);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (d == n) continue;
    mm_adj<T>(b, lb, st[d], gv * (par[d] ? 0.25 : -0.25));
  }
}

template <class T, int DIM> __global__ void k_adj_prolong_faces(AdjRows a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 5 * r;
  const DPatch D = a.P[row[0]], C = a.P[row[3]];
  const int n = row[1];
  double* ld = a.lam + D.off + (BX + n) * D.fs + row[2];
  const double gv = *ld;
  *ld = 0.0;
  if (gv == 0.0) return;
  int g[3];
  global_pos<DIM>(D, row[2], g);
  const int par[3] = {g[0] & 1, g[1] & 1, DIM == 3 ? (g[2] & 1) : 0};
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
  const T* cb = (const T*)a.Xc + C.off;
  double* lcb = a.lamc + C.off;
  const long long bo = (BX + n) * C.fs + row[4];
  if (!par[n]) {
    coincident_adj<T, DIM>(cb + bo, lcb + bo, st, n, par, gv);
    return;
  }
  coincident_adj<T, DIM>(cb + bo, lcb + bo, st, n, par, 0.5 * gv);
  coincident_adj<T, DIM>(cb + bo + st[n], lcb + bo + st[n], st, n, par, 0.5 * gv);
#pragma unroll
  for (int t = 0; t < DIM; ++t) {
    if (t == n) continue;
    const double c = 0.125 * a.ratio[n][t] * gv;
    const long long to = (BX + t) * C.fs + row[4];
    mm_adj<T>(cb + to + st[t], lcb + to + st[t], st[n], c);
    mm_adj<T>(cb + to, lcb + to, st[n], -c);
  }
}

// ------------------------------------------------------------------ packed adjoint I/O
template <int DIM>
__global__ void __launch_bounds__(TPB) k_lam_io(const DPatch* PP, const int* ids, double* lam, double* packed,
                                                const long long* poff, int field, int to_lam) {
  const int pid = ids[blockIdx.y];
  const DPatch P = PP[pid];
  const int fd = (field >= BX && !(DIM == 2 && field == BZ)) ? field - BX : -1;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : P.n[e] + (e == fd ? 1 : 0);
  const int t = blockIdx.x * TPB + threadIdx.x;
  if (t >= r[0] * r[1] * r[2]) return;
  const int i = t % r[0], j = (t / r[0]) % r[1], k = t / (r[0] * r[1]);
  const int L = lidx(P, i + 4, j + 4, DIM == 3 ? k + 4 : 0);
  double* s = lam + P.off + field * P.fs + L;
  double* q = packed + poff[pid] + t;
  if (to_lam) *s = *q;
  else *q = *s;
}

// ------------------------------------------------------------------ launch tables
struct AdjOps {
  void (*advance_t)(const AdjArgs&, cudaStream_t);
  void (*emf_flux_t)(const AdjArgs&, cudaStream_t);
  void (*pred_prim_t)(const AdjArgs&, cudaStream_t);
  void (*regc)(const AdjRows& faces, const AdjRows& edges, cudaStream_t);
  void (*regf)(const AdjRows& faces, const AdjRows& edges, cudaStream_t);
  void (*restrict_t)(const AdjRows& cells, const AdjRows& faces, cudaStream_t);
  void (*reflux_t)(const AdjRows& cells, const AdjRows& faces, cudaStream_t);
  void (*same_t)(const AdjRows& cells, const AdjRows& faces, cudaStream_t);
  void (*bc_t)(const AdjRows& cells, const AdjRows& faces, cudaStream_t);
  void (*prolong_t)(const AdjRows& cells, const AdjRows& faces, cudaStream_t);
  void (*lam_io)(const DPatch*, const int*, int, const int*, double*, double*, const long long*, int, int,
                 cudaStream_t);
};

template <class T, int DIM> struct AImpl {
  static dim3 grid(const AdjArgs& a, int m, int extra) {
    long long n = 1;
    for (int d = 0; d < DIM; ++d) n *= a.maxn[d] + 2 * m + extra;
    return dim3(cdiv(n, TPB), a.npatch);
  }
  static dim3 rgrid(long long n) { return dim3(cdiv(n, TPB)); }
  // update transpose: identity of cells and faces, flux and EMF seeds
  static void advance_t(const AdjArgs& a, cudaStream_t s) {
    k_adj_update_cells<T, DIM><<<grid(a, a.w, 0), TPB, 0, s>>>(a);
    k_adj_faces<T, DIM, 0><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    k_adj_faces<T, DIM, 1><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    if (DIM == 3) k_adj_faces<T, DIM, 2><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    if (DIM == 3) {
      k_adj_emf_seed<T, DIM, 0><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
      k_adj_emf_seed<T, DIM, 1><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
    }
    k_adj_emf_seed<T, DIM, 2><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
  }
  static void emf_flux_t(const AdjArgs& a, cudaStream_t s) {
    if (DIM == 3) {
      k_adj_emf<T, DIM, 0><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
      k_adj_emf<T, DIM, 1><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
    }
    k_adj_emf<T, DIM, 2><<<grid(a, a.w, 1), TPB, 0, s>>>(a);
    k_adj_flux<T, DIM, 0><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    k_adj_flux<T, DIM, 1><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    if (DIM == 3) k_adj_flux<T, DIM, 2><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
  }
  static void pred_prim_t(const AdjArgs& a, cudaStream_t s) {
    k_adj_predict<T, DIM><<<grid(a, a.w + 1, 0), TPB, 0, s>>>(a);
    k_adj_prim<T, DIM><<<grid(a, a.w + 2, 0), TPB, 0, s>>>(a);
  }
#define AMRADJ_PAIR(NAME, KC, KF)                                                   \
  static void NAME(const AdjRows& c, const AdjRows& f, cudaStream_t s) {            \
    if (c.nrows) KC<T, DIM><<<rgrid(c.nrows), TPB, 0, s>>>(c);                      \
    if (f.nrows) KF<T, DIM><<<rgrid(f.nrows), TPB, 0, s>>>(f);                      \
  }
  AMRADJ_PAIR(regc, k_adj_regc_faces, k_adj_regc_edges)
  AMRADJ_PAIR(regf, k_adj_regf_faces, k_adj_regf_edges)
  AMRADJ_PAIR(restrict_t, k_adj_restrict_cells, k_adj_restrict_faces)
  AMRADJ_PAIR(reflux_t, k_adj_reflux_cells, k_adj_reflux_faces)
  AMRADJ_PAIR(same_t, k_adj_same_cells, k_adj_same_faces)
  AMRADJ_PAIR(bc_t, k_adj_bc_cells, k_adj_bc_faces)
  AMRADJ_PAIR(prolong_t, k_adj_prolong_cells, k_adj_prolong_faces)
#undef AMRADJ_PAIR
  static void lam_io(const DPatch* P, const int* ids, int npatch, const int* maxn, double* lam, double* packed,
                     const long long* poff, int field, int to_lam, cudaStream_t s) {
    long long n = 1;
    for (int d = 0; d < DIM; ++d) n *= maxn[d] + 1;
    k_lam_io<DIM><<<dim3(cdiv(n, TPB), npatch), TPB, 0, s>>>(P, ids, lam, packed, poff, field, to_lam);
  }
  static const AdjOps* ops() {
    static const AdjOps o = {advance_t, emf_flux_t, pred_prim_t, regc, regf, restrict_t, reflux_t,
                             same_t, bc_t, prolong_t, lam_io};
    return &o;
  }
};

const AdjOps* adj_ops(bool fp32, int dim) {
  if (fp32) return dim == 3 ? AImpl<float, 3>::ops() : AImpl<float, 2>::ops();
  return dim == 3 ? AImpl<double, 3>::ops() : AImpl<double, 2>::ops();
}

// one thread per point: gx = J^T g of HLLD (WHICH 0; x = ql[7], qr[7], bn) or
// of the half-step predictor (WHICH 1; x = w[8], s_0[8], .., s_{DIM-1}[8]), by
// the hand-written transposes in FP64 (METHOD 0) or FP32 (METHOD 2, inputs
// rounded to FP32), or forward-mode dual numbers (METHOD 1)
template <int WHICH, int DIM, int METHOD>
__global__ void __launch_bounds__(TPB) k_local_vjp(long long n, const double* x, const double* g, double gamma,
                                                   double h0, double h1, double h2, double* gx) {
  const long long i = blockIdx.x * (long long)TPB + threadIdx.x;
  if (i >= n) return;
  constexpr int NIN = WHICH == 0 ? 15 : 8 + 8 * DIM;
  constexpr int NOUT = WHICH == 0 ? 7 : 8;
  double xi[NIN], gi[NOUT], o[NIN];
#pragma unroll
  for (int q = 0; q < NIN; ++q) xi[q] = x[i * NIN + q];
#pragma unroll
  for (int q = 0; q < NOUT; ++q) gi[q] = g[i * NOUT + q];
  float xf[NIN], gf[NOUT], of[NIN];
#pragma unroll
  for (int q = 0; q < NIN; ++q) xf[q] = (float)xi[q];
#pragma unroll
  for (int q = 0; q < NOUT; ++q) gf[q] = (float)gi[q];
  if (WHICH == 0) {
    if (METHOD == 0) hlld_vjp<double>(xi, gi, gamma, o);
    else if (METHOD == 1) vjp<NIN, NOUT, 5>(xi, gi, o, HlldFn{gamma});
    else hlld_vjp<float>(xf, gf, (float)gamma, of);
  } else {
    const double h[3] = {h0, h1, h2};
    const float hf[3] = {(float)h0, (float)h1, (float)h2};
    if (METHOD == 0) {
      predict_vjp<DIM, double>(xi, gi, gamma, h, o);
    } else if (METHOD == 2) {
      predict_vjp<DIM, float>(xf, gf, (float)gamma, hf, of);
    } else {
      PredFn<DIM> fn;
      fn.gamma = gamma;
      for (int d = 0; d < 3; ++d) fn.h[d] = h[d];
      vjp<NIN, NOUT, 8>(xi, gi, o, fn);
    }
  }
#pragma unroll
  for (int q = 0; q < NIN; ++q) gx[i * NIN + q] = METHOD == 2 ? (double)of[q] : o[q];
}

}  // namespace amradj

// ================================================================== host side
namespace amrapi {
using amrk::DPatch;

struct AdjWork {
  const amradj::AdjOps* ops = nullptr;
  size_t elem = 8;
  long long scr_elems = 0;
  std::vector<long long> soff;       // adjoint scratch offsets per patch
  std::vector<long long> lev_begin, lev_end;  // element range of each level in a state buffer
  DPatch* dP = nullptr;              // patch table with the adjoint scratch offsets
  double *lam = nullptr, *lamx = nullptr, *lscr = nullptr, *lR = nullptr, *lRE = nullptr, *d_dts = nullptr;
  void *fscr = nullptr, *tmp = nullptr;
  char *snaps = nullptr, *ckpts = nullptr;
  size_t snap_cap = 0, ckpt_cap = 0;
  long long dts_cap = 0;
  std::vector<size_t> slot_off;      // byte offset of each pre-order slot within one coarse step
  std::vector<int> slot_level;
  size_t step_bytes = 0;
  int rec_step = 0, rec_slot = 0;
  std::vector<void*> allocs;
  // the record of the last amrmhd_step_dt_ckpt: its steps, dt sequence (in
  // d_dts), checkpoints (the level buffers in use at each) and the state count
  // after it
  bool rec_valid = false;
  int rec_n = 0, rec_k = 0;
  std::vector<std::vector<int>> rec_cur;
  unsigned long long rec_version = 0;
};

void adj_free(amrmhd_ctx* ctx) {
  if (!ctx->adj) return;
  for (void* p : ctx->adj->allocs) cudaFree(p);
  if (ctx->adj->snaps) cudaFree(ctx->adj->snaps);
  if (ctx->adj->ckpts) cudaFree(ctx->adj->ckpts);
  if (ctx->adj->d_dts) cudaFree(ctx->adj->d_dts);
  delete ctx->adj;
  ctx->adj = nullptr;
}

namespace {

#define CUA(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, AMRMHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int subtree(int nlev, int l) { return (1 << (nlev - l)) - 1; }

// the level of every pre-order level-step slot of one coarse step
void preorder(int nlev, int l, std::vector<int>& out) {
  out.push_back(l);
  if (l + 1 < nlev) {
    preorder(nlev, l + 1, out);
    preorder(nlev, l + 1, out);
  }
}

amrmhd_status adj_setup(amrmhd_ctx* ctx) {
  if (ctx->adj) return AMRMHD_OK;
  amrmhd_status rst = upload_fill_rows(ctx);
  if (rst) return rst;
  AdjWork* A = new AdjWork();
  ctx->adj = A;
  const amrmhd::Hierarchy& H = ctx->H;
  const int np = (int)H.p.size();
  A->ops = amradj::adj_ops(ctx->cfg.precision == AMRMHD_MIXED, H.dim);
  A->elem = ctx->ops->elem;
  A->soff.assign(np, 0);
  long long sacc = 0;
  A->lev_begin.assign(H.nlev, 0);
  A->lev_end.assign(H.nlev, 0);
  for (int l = 0; l < H.nlev; ++l) {
    A->lev_begin[l] = ctx->off[H.level_patches[l].front()];
    for (int q : H.level_patches[l]) {
      A->soff[q] = sacc;
      sacc += amrk::SC_N * ctx->fs[q];
      A->lev_end[l] = std::max(A->lev_end[l], ctx->off[q] + 8 * ctx->fs[q]);
    }
  }
  A->scr_elems = sacc;
  std::vector<DPatch> hp(np);
  CUA(cudaMemcpy(hp.data(), ctx->dP, sizeof(DPatch) * np, cudaMemcpyDeviceToHost));
  for (int q = 0; q < np; ++q) hp[q].soff = A->soff[q];
  auto get = [&](size_t bytes, void** p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
    if (e == cudaSuccess) A->allocs.push_back(*p);
    return e;
  };
  CUA(get(sizeof(DPatch) * np, (void**)&A->dP));
  CUA(cudaMemcpy(A->dP, hp.data(), sizeof(DPatch) * np, cudaMemcpyHostToDevice));
  const size_t se = (size_t)ctx->state_elems;
  CUA(get(se * sizeof(double), (void**)&A->lam));
  CUA(get(se * sizeof(double), (void**)&A->lamx));
  CUA(get((size_t)sacc * sizeof(double), (void**)&A->lscr));
  CUA(get((size_t)sacc * A->elem, &A->fscr));
  CUA(get(se * A->elem, &A->tmp));
  CUA(get((size_t)std::max<int64_t>(ctx->ncf, 1) * 6 * sizeof(double), (void**)&A->lR));
  CUA(get((size_t)std::max<int64_t>(ctx->nce, 1) * sizeof(double), (void**)&A->lRE));
  preorder(H.nlev, 0, A->slot_level);
  A->slot_off.assign(A->slot_level.size(), 0);
  size_t o = 0;
  for (size_t i = 0; i < A->slot_level.size(); ++i) {
    const int l = A->slot_level[i];
    A->slot_off[i] = o;
    o += align256((size_t)(A->lev_end[l] - A->lev_begin[l]) * A->elem);
  }
  A->step_bytes = o;
  return AMRMHD_OK;
}

amrmhd_status adj_reserve(amrmhd_ctx* ctx, int steps_per_seg, int nseg, int n) {
  AdjWork* A = ctx->adj;
  const size_t snap = A->step_bytes * (size_t)steps_per_seg;
  if (snap > A->snap_cap) {
    if (A->snaps) cudaFree(A->snaps);
    A->snaps = nullptr;
    A->snap_cap = 0;
    CUA(cudaMalloc((void**)&A->snaps, snap));
    A->snap_cap = snap;
  }
  const size_t ck = align256((size_t)ctx->state_elems * A->elem) * (size_t)nseg;
  if (ck > A->ckpt_cap) {
    if (A->ckpts) cudaFree(A->ckpts);
    A->ckpts = nullptr;
    A->ckpt_cap = 0;
    CUA(cudaMalloc((void**)&A->ckpts, ck));
    A->ckpt_cap = ck;
  }
  if (n > A->dts_cap) {
    if (A->d_dts) cudaFree(A->d_dts);
    A->d_dts = nullptr;
    A->dts_cap = 0;
    CUA(cudaMalloc((void**)&A->d_dts, sizeof(double) * n));
    A->dts_cap = n;
  }
  return AMRMHD_OK;
}

// a level's snapshot, addressed like a state buffer (element offsets P.off)
const void* snap_base(amrmhd_ctx* ctx, int step, int slot) {
  AdjWork* A = ctx->adj;
  const int l = A->slot_level[slot];
  const char* p = A->snaps + (size_t)step * A->step_bytes + A->slot_off[slot];
  return p - (size_t)A->lev_begin[l] * A->elem;
}

void record_fill(amrmhd_ctx* ctx, int l, int) {
  AdjWork* A = ctx->adj;
  const int slot = A->rec_slot++;
  char* dst = A->snaps + (size_t)A->rec_step * A->step_bytes + A->slot_off[slot];
  const char* src = (const char*)state_buf(ctx, ctx->cur[l]) + (size_t)A->lev_begin[l] * A->elem;
  cudaMemcpyAsync(dst, src, (size_t)(A->lev_end[l] - A->lev_begin[l]) * A->elem, cudaMemcpyDeviceToDevice,
                  ctx->stream);
}

void save_ckpt(amrmhd_ctx* ctx, int seg, std::vector<int>& cur_saved) {
  AdjWork* A = ctx->adj;
  char* base = A->ckpts + align256((size_t)ctx->state_elems * A->elem) * (size_t)seg;
  for (int l = 0; l < ctx->H.nlev; ++l) {
    const size_t b = (size_t)A->lev_begin[l] * A->elem, n = (size_t)(A->lev_end[l] - A->lev_begin[l]) * A->elem;
    cudaMemcpyAsync(base + b, (char*)state_buf(ctx, ctx->cur[l]) + b, n, cudaMemcpyDeviceToDevice, ctx->stream);
  }
  cur_saved = ctx->cur;
}

void load_ckpt(amrmhd_ctx* ctx, int seg, const std::vector<int>& cur_saved) {
  AdjWork* A = ctx->adj;
  const char* base = A->ckpts + align256((size_t)ctx->state_elems * A->elem) * (size_t)seg;
  ctx->cur = cur_saved;
  for (int l = 0; l < ctx->H.nlev; ++l) {
    const size_t b = (size_t)A->lev_begin[l] * A->elem, n = (size_t)(A->lev_end[l] - A->lev_begin[l]) * A->elem;
    cudaMemcpyAsync((char*)state_buf(ctx, ctx->cur[l]) + b, base + b, n, cudaMemcpyDeviceToDevice, ctx->stream);
  }
}

// one forward coarse step with the prescribed dt0 (stored at d_dt)
void fwd_step(amrmhd_ctx* ctx, const double* d_dt) {
  cudaMemcpyAsync(ctx->d_scal, d_dt, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  int nl = 0;
  op_level_step(ctx, 0, 1, &nl);
  ctx->launches += nl;
}

amradj::AdjRows adj_rows(amrmhd_ctx* ctx, const DevList& L, int coarse_level) {
  amradj::AdjRows a;
  std::memset(&a, 0, sizeof(a));
  a.P = ctx->adj->dP;
  a.rows = L.p;
  a.nrows = L.n;
  a.lam = ctx->adj->lam;
  double dx[3];
  for (int d = 0; d < 3; ++d) {
    const int N = d < ctx->cfg.dim ? (ctx->cfg.base[d] << coarse_level) : 1;
    dx[d] = d < ctx->cfg.dim ? (ctx->cfg.hi[d] - ctx->cfg.lo[d]) / N : 1.0;
    a.idx[d] = 1.0 / dx[d];
  }
  for (int n = 0; n < 3; ++n)
    for (int t = 0; t < 3; ++t) a.ratio[n][t] = dx[n] / dx[t];
  return a;
}

struct Rev {
  amrmhd_ctx* ctx;
  int step;             // coarse step index within the segment (snapshot row)
  const double* d_dt;   // dt0 of this coarse step on the device
};

// transpose of reflux and restriction of fine level l onto level l-1
void adj_rr(const Rev& R, int l) {
  amrmhd_ctx* ctx = R.ctx;
  AdjWork* A = ctx->adj;
  const LevelDev& F = ctx->lev[l];
  // the register adjoints of this level's rows are rebuilt here
  if (F.cf_faces.n)
    cudaMemsetAsync(A->lR + F.cf_face0 * 6, 0, sizeof(double) * 6 * F.cf_faces.n, ctx->stream);
  if (F.cf_edges.n) cudaMemsetAsync(A->lRE + F.cf_edge0, 0, sizeof(double) * F.cf_edges.n, ctx->stream);
  amradj::AdjRows c = adj_rows(ctx, F.restrict_cells, l - 1), f = adj_rows(ctx, F.restrict_faces, l - 1);
  c.lamf = f.lamf = A->lam;
  A->ops->restrict_t(c, f, ctx->stream);
  // reflux rows hold global C/F row numbers
  c = adj_rows(ctx, F.reflux_cells, l - 1);
  f = adj_rows(ctx, F.emf_faces, l - 1);
  c.lR = f.lR = A->lR;
  c.lRE = f.lRE = A->lRE;
  A->ops->reflux_t(c, f, ctx->stream);
}

// transpose of one advance of level l, sub-step s, from the snapshot of its filled state
void adj_advance(const Rev& R, int l, int s, int slot) {
  amrmhd_ctx* ctx = R.ctx;
  AdjWork* A = ctx->adj;
  const LevelDev& L = ctx->lev[l];
  const int w = (l == 0) ? 0 : (s == 1 ? 2 : 0);
  const double dtscale = 1.0 / (double)(1 << l);
  const void* X = snap_base(ctx, R.step, slot);
  // forward stage arrays from the snapshot (the staged kernels; the output goes to a scratch buffer)
  amrk::LevelArgs fa = level_args(ctx, l, R.d_dt, dtscale, w);
  fa.P = A->dP;
  fa.cur = const_cast<void*>(X);
  fa.nxt = A->tmp;
  fa.scr = A->fscr;
  int nl = 0;
  ctx->ops->advance(fa, ctx->stream, &nl);
  ctx->launches += nl;
  // adjoint stage arrays of this level's patches start at zero
  {
    const int q0 = ctx->H.level_patches[l].front(), q1 = ctx->H.level_patches[l].back();
    const long long b = A->soff[q0], e = A->soff[q1] + amrk::SC_N * ctx->fs[q1];
    cudaMemsetAsync(A->lscr + b, 0, sizeof(double) * (size_t)(e - b), ctx->stream);
  }
  amradj::AdjArgs a;
  a.P = A->dP;
  a.ids = L.ids;
  a.npatch = L.npatch;
  for (int d = 0; d < 3; ++d) a.maxn[d] = L.maxn[d];
  a.X = X;
  a.scr = A->fscr;
  a.lam = A->lam;
  a.lamx = A->lamx;
  a.lscr = A->lscr;
  a.dtp = R.d_dt;
  a.dtscale = dtscale;
  level_idx(ctx, l, a.idx);
  a.gamma = ctx->cfg.gamma;
  a.w = w;
  A->ops->advance_t(a, ctx->stream);
  // register seeds: this level as the coarse side of level l+1, and as the fine side of level l
  if (l + 1 < ctx->H.nlev) {
    const LevelDev& F = ctx->lev[l + 1];
    amradj::AdjRows c = adj_rows(ctx, F.cf_faces, l), e = adj_rows(ctx, F.cf_edges, l);
    c.lscr = e.lscr = A->lscr;
    c.lR = e.lR = A->lR + F.cf_face0 * 6;
    c.lRE = e.lRE = A->lRE + F.cf_edge0;
    c.dtp = e.dtp = R.d_dt;
    c.dtscale = e.dtscale = dtscale;
    A->ops->regc(c, e, ctx->stream);
  }
  if (l > 0) {
    amradj::AdjRows c = adj_rows(ctx, L.cf_faces, l - 1), e = adj_rows(ctx, L.cf_edges, l - 1);
    c.lscr = e.lscr = A->lscr;
    c.lR = e.lR = A->lR + L.cf_face0 * 6;
    c.lRE = e.lRE = A->lRE + L.cf_edge0;
    c.dtp = e.dtp = R.d_dt;
    c.dtscale = e.dtscale = dtscale;
    c.substep = e.substep = s;
    A->ops->regf(c, e, ctx->stream);
  }
  A->ops->emf_flux_t(a, ctx->stream);
  A->ops->pred_prim_t(a, ctx->stream);
  // the level's adjoint now refers to its filled state
  const size_t b = (size_t)A->lev_begin[l], n = (size_t)(A->lev_end[l] - A->lev_begin[l]);
  cudaMemcpyAsync(A->lam + b, A->lamx + b, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  cudaMemsetAsync(A->lamx + b, 0, n * sizeof(double), ctx->stream);
}

// transpose of the ghost fill: boundaries, then prolongation (s = 1), then same-level copies
void adj_fill(const Rev& R, int l, int s, int parent_slot) {
  amrmhd_ctx* ctx = R.ctx;
  AdjWork* A = ctx->adj;
  const LevelDev& L = ctx->lev[l];
  amradj::AdjRows c = adj_rows(ctx, L.row_bc_cells, l), f = adj_rows(ctx, L.row_bc_faces, l);
  A->ops->bc_t(c, f, ctx->stream);
  if (s == 1 && l > 0) {
    c = adj_rows(ctx, L.row_prol_cells, l - 1);
    f = adj_rows(ctx, L.row_prol_faces, l - 1);
    c.lamc = f.lamc = A->lamx;
    c.Xc = f.Xc = snap_base(ctx, R.step, parent_slot);
    A->ops->prolong_t(c, f, ctx->stream);
  }
  c = adj_rows(ctx, L.row_same_cells, l);
  f = adj_rows(ctx, L.row_same_faces, l);
  A->ops->same_t(c, f, ctx->stream);
}

void adj_level_step(const Rev& R, int l, int s, int slot, int parent_slot) {
  const int nlev = R.ctx->H.nlev;
  if (l + 1 < nlev) {
    adj_rr(R, l + 1);
    const int c = subtree(nlev, l + 1);
    adj_level_step(R, l + 1, 2, slot + 1 + c, slot);
    adj_level_step(R, l + 1, 1, slot + 1, slot);
  }
  adj_advance(R, l, s, slot);
  adj_fill(R, l, s, parent_slot);
}

// packed adjoint of all 8 fields <-> the level adjoint buffers
void lam_io(amrmhd_ctx* ctx, double* packed, int to_lam) {
  AdjWork* A = ctx->adj;
  const amrmhd::Hierarchy& H = ctx->H;
  long long o = 0;
  for (int field = 0; field < 8; ++field) {
    const int kind = (field >= 5 && !(H.dim == 2 && field == 7)) ? field - 4 : 0;
    for (int l = 0; l < H.nlev; ++l) {
      const LevelDev& L = ctx->lev[l];
      A->ops->lam_io(A->dP, L.ids, L.npatch, L.maxn, A->lam, packed + o, ctx->d_poff[kind], field, to_lam,
                     ctx->stream);
    }
    o += ctx->ptotal[kind];
  }
}

}  // namespace
}  // namespace amrapi

using namespace amrapi;

extern "C" {

amrmhd_status amrmhd_step_dt(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq) {
  if (ctx) ++ctx->state_version;  // a recorded forward (amrmhd_step_dt_ckpt) no longer matches
  amrmhd_status st = check_bound(ctx);
  if (st) return st;
  if (n_coarse < 0 || (n_coarse > 0 && !dt_seq)) return fail(ctx, AMRMHD_EINVAL, "bad step count or dt sequence");
  for (int i = 0; i < n_coarse; ++i)
    if (!(dt_seq[i] > 0.0)) return fail(ctx, AMRMHD_EINVAL, "dt must be positive");
  st = adj_setup(ctx);
  if (st) return st;
  st = adj_reserve(ctx, 1, 1, std::max(n_coarse, 1));
  if (st) return st;
  AdjWork* A = ctx->adj;
  if (n_coarse) CUA(cudaMemcpyAsync(A->d_dts, dt_seq, sizeof(double) * n_coarse, cudaMemcpyHostToDevice, ctx->stream));
  for (int i = 0; i < n_coarse; ++i) fwd_step(ctx, A->d_dts + i);
  CUA(cudaStreamSynchronize(ctx->stream));
  CUA(cudaGetLastError());
  return AMRMHD_OK;
}

}  // extern "C"

namespace {

// The reverse sweep of amrmhd_backward over n_coarse steps of dt0 in A->d_dts,
// from the checkpoints saved every k steps (cur_at: the level buffers in use
// at each); leaves the context at the first checkpoint.
amrmhd_status adj_sweep(amrmhd_ctx* ctx, int n_coarse, int k, const std::vector<std::vector<int>>& cur_at,
                        const double* dL_dUfinal, double* dL_dU0) {
  AdjWork* A = ctx->adj;
  const int nseg = (n_coarse + k - 1) / k;
  // seed: the adjoint of the final state
  const size_t se = (size_t)ctx->state_elems;
  CUA(cudaMemsetAsync(A->lam, 0, se * sizeof(double), ctx->stream));
  CUA(cudaMemsetAsync(A->lamx, 0, se * sizeof(double), ctx->stream));
  lam_io(ctx, const_cast<double*>(dL_dUfinal), 1);
  // reverse sweep over the segments, each recomputed with its filled states recorded
  for (int seg = nseg - 1; seg >= 0; --seg) {
    load_ckpt(ctx, seg, cur_at[seg]);
    const int i0 = seg * k, i1 = std::min(n_coarse, i0 + k);
    ctx->after_fill = record_fill;
    for (int i = i0; i < i1; ++i) {
      A->rec_step = i - i0;
      A->rec_slot = 0;
      fwd_step(ctx, A->d_dts + i);
    }
    ctx->after_fill = nullptr;
    for (int i = i1 - 1; i >= i0; --i) {
      Rev R{ctx, i - i0, A->d_dts + i};
      adj_level_step(R, 0, 1, 0, -1);
    }
  }
  lam_io(ctx, dL_dU0, 0);
  // leave the context at the initial state
  load_ckpt(ctx, 0, cur_at[0]);
  ++ctx->state_version;
  A->rec_valid = false;
  CUA(cudaStreamSynchronize(ctx->stream));
  CUA(cudaGetLastError());
  return AMRMHD_OK;
}

amrmhd_status adj_check(amrmhd_ctx* ctx, int n_coarse, const double* dt_seq, int ckpt_every) {
  amrmhd_status st = check_bound(ctx);
  if (st) return st;
  if (n_coarse < 1 || !dt_seq || ckpt_every < 1) return fail(ctx, AMRMHD_EINVAL, "bad arguments");
  for (int i = 0; i < n_coarse; ++i)
    if (!(dt_seq[i] > 0.0)) return fail(ctx, AMRMHD_EINVAL, "dt must be positive");
  if (ctx->floor_rho > 0.0 || ctx->floor_p > 0.0)
    return fail(ctx, AMRMHD_ESTATE, "the adjoint does not differentiate floors: set them to 0");
  return AMRMHD_OK;
}

}  // namespace

extern "C" {

amrmhd_status amrmhd_backward(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq, int32_t ckpt_every,
                              const double* dL_dUfinal, double* dL_dU0) {
  amrmhd_status st = adj_check(ctx, n_coarse, dt_seq, ckpt_every);
  if (st) return st;
  if (!dL_dUfinal || !dL_dU0) return fail(ctx, AMRMHD_EINVAL, "bad arguments");
  st = adj_setup(ctx);
  if (st) return st;
  const int k = std::min<int>(ckpt_every, n_coarse);
  const int nseg = (n_coarse + k - 1) / k;
  st = adj_reserve(ctx, k, nseg, n_coarse);
  if (st) return st;
  AdjWork* A = ctx->adj;
  A->rec_valid = false;
  CUA(cudaMemcpyAsync(A->d_dts, dt_seq, sizeof(double) * n_coarse, cudaMemcpyHostToDevice, ctx->stream));
  // forward pass: checkpoints at the start of every segment (it stops at the
  // last segment's start: the sweep recomputes that segment from its checkpoint)
  std::vector<std::vector<int>> cur_at(nseg);
  for (int i = 0; i < n_coarse; ++i) {
    if (i % k == 0) save_ckpt(ctx, i / k, cur_at[i / k]);
    if (i / k == nseg - 1) break;
    fwd_step(ctx, A->d_dts + i);
  }
  return adj_sweep(ctx, n_coarse, k, cur_at, dL_dUfinal, dL_dU0);
}

amrmhd_status amrmhd_step_dt_ckpt(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq, int32_t ckpt_every) {
  amrmhd_status st = adj_check(ctx, n_coarse, dt_seq, ckpt_every);
  if (st) return st;
  st = adj_setup(ctx);
  if (st) return st;
  const int k = std::min<int>(ckpt_every, n_coarse);
  const int nseg = (n_coarse + k - 1) / k;
  st = adj_reserve(ctx, k, nseg, n_coarse);
  if (st) return st;
  AdjWork* A = ctx->adj;
  A->rec_valid = false;
  CUA(cudaMemcpyAsync(A->d_dts, dt_seq, sizeof(double) * n_coarse, cudaMemcpyHostToDevice, ctx->stream));
  A->rec_cur.assign(nseg, {});
  for (int i = 0; i < n_coarse; ++i) {
    if (i % k == 0) save_ckpt(ctx, i / k, A->rec_cur[i / k]);
    fwd_step(ctx, A->d_dts + i);
  }
  CUA(cudaStreamSynchronize(ctx->stream));
  CUA(cudaGetLastError());
  ++ctx->state_version;
  A->rec_valid = true;
  A->rec_n = n_coarse;
  A->rec_k = k;
  A->rec_version = ctx->state_version;
  return AMRMHD_OK;
}

amrmhd_status amrmhd_backward_recorded(amrmhd_ctx* ctx, const double* dL_dUfinal, double* dL_dU0) {
  amrmhd_status st = check_bound(ctx);
  if (st) return st;
  if (!dL_dUfinal || !dL_dU0) return fail(ctx, AMRMHD_EINVAL, "bad arguments");
  AdjWork* A = ctx->adj;
  if (!A || !A->rec_valid || A->rec_version != ctx->state_version)
    return fail(ctx, AMRMHD_ESTATE, "no recorded forward matches the current state (amrmhd_step_dt_ckpt)");
  if (ctx->floor_rho > 0.0 || ctx->floor_p > 0.0)
    return fail(ctx, AMRMHD_ESTATE, "the adjoint does not differentiate floors: set them to 0");
  const std::vector<std::vector<int>> cur_at = A->rec_cur;
  return adj_sweep(ctx, A->rec_n, A->rec_k, cur_at, dL_dUfinal, dL_dU0);
}

amrmhd_status amrmhd_local_vjp(int32_t which, int32_t dim, int64_t n, const double* x, const double* g, double gamma,
                               const double* h, int32_t method, double* gx) {
  if (which < 0 || which > 1 || (which == 1 && dim != 2 && dim != 3) || n < 0 || method < 0 || method > 2 ||
      (n > 0 && (!x || !g || !gx || (which == 1 && !h))) || !(gamma > 1.0))
    return AMRMHD_EINVAL;
  if (n == 0) return AMRMHD_OK;
  const int nin = which == 0 ? 15 : 8 + 8 * dim, nout = which == 0 ? 7 : 8;
  double *dx = nullptr, *dg = nullptr, *dgx = nullptr;
  amrmhd_status st = AMRMHD_OK;
  const double hh[3] = {which == 1 ? h[0] : 0.0, which == 1 ? h[1] : 0.0, which == 1 && dim == 3 ? h[2] : 0.0};
  if (cudaMalloc(&dx, sizeof(double) * n * nin) != cudaSuccess || cudaMalloc(&dg, sizeof(double) * n * nout) != cudaSuccess ||
      cudaMalloc(&dgx, sizeof(double) * n * nin) != cudaSuccess) {
    st = AMRMHD_ECUDA;
  } else if (cudaMemcpy(dx, x, sizeof(double) * n * nin, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dg, g, sizeof(double) * n * nout, cudaMemcpyHostToDevice) != cudaSuccess) {
    st = AMRMHD_ECUDA;
  } else {
    using namespace amradj;
    const unsigned nb = (unsigned)((n + TPB - 1) / TPB);
    const int key = which * 100 + (which == 1 ? dim : 0) * 10 + method;
#define AMRMHD_LVJP(W, D, M) \
  case W * 100 + (W == 1 ? D : 0) * 10 + M: \
    k_local_vjp<W, D, M><<<nb, TPB>>>(n, dx, dg, gamma, hh[0], hh[1], hh[2], dgx); \
    break;
    switch (key) {
      AMRMHD_LVJP(0, 3, 0)
      AMRMHD_LVJP(0, 3, 1)
      AMRMHD_LVJP(0, 3, 2)
      AMRMHD_LVJP(1, 2, 0)
      AMRMHD_LVJP(1, 2, 1)
      AMRMHD_LVJP(1, 2, 2)
      AMRMHD_LVJP(1, 3, 0)
      AMRMHD_LVJP(1, 3, 1)
      AMRMHD_LVJP(1, 3, 2)
      default: break;
    }
#undef AMRMHD_LVJP
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(gx, dgx, sizeof(double) * n * nin, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = AMRMHD_ECUDA;
  }
  cudaFree(dx);
  cudaFree(dg);
  cudaFree(dgx);
  return st;
}

}  // extern "C"
