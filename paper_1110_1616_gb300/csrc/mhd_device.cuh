// Device-side per-element formulas of the ideal-MHD advance, templated on the
// arithmetic type T (double for the FP64 path, float for the FP32 stencil of
// the mixed path). The evaluation order of every expression is the one the
// scheme fixes, so that the FP64 build without FMA contraction reproduces a
// plain FP64 implementation bit for bit.
//
// The paper names the hyperbolic advance of each grid (Abstract, Sec. 1) but not
// the scheme; the choices are:
//  * MUSCL-Hancock, unsplit, with the half-step predictor written in primitive
//    variables (the v div B term of the induction equation dropped).
//  * minmod(a, b): 0 unless a and b have the same strict sign, else the one of
//    smaller magnitude (a on a tie); a = backward, b = forward difference. The
//    slope of the normal B in its own direction is the face difference.
//  * HLLD (Miyoshi & Kusano 2005) with S_L = min(uL,uR) - max(cfL,cfR),
//    S_R = max(uL,uR) + max(cfL,cfR); degenerate star states when
//    |e| <= eps (|rho (S-u)(S-S_M)| + Bn^2); double-star states skipped when
//    Bn^2 <= eps p_T*; eps = 1e-12 in FP64 and 1e-6 in FP32; the normal field
//    is the mean of the two predicted face states' normal B.
//  * Edge EMFs: Gardiner & Stone upwinded average with the cell-centre
//    reference -(v x B) at the half step, upwinded by the face mass flux (the
//    mean of both sides when it is exactly 0).
#pragma once
#include <cuda_runtime.h>
#include "fp_bits.cuh"

namespace amrdev {

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7 };

template <class T> struct Eps;
template <> struct Eps<double> { static __device__ __forceinline__ double v() { return 1e-12; } };
template <> struct Eps<float> { static __device__ __forceinline__ float v() { return 1e-6f; } };

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }

template <class T> __device__ __forceinline__ T mm(T a, T b) {
  if (a > T(0) && b > T(0)) return (a <= b) ? a : b;
  if (a < T(0) && b < T(0)) return (a >= b) ? a : b;
  return T(0);
}

template <class T> __device__ __forceinline__ T tmaxd(T a, T b) { return a > b ? a : b; }
template <class T> __device__ __forceinline__ T tmind(T a, T b) { return a < b ? a : b; }

// square of the fast magnetosonic speed along a direction with normal field bn
template <class T> __device__ __forceinline__ T cfast2(T rho, T p, T bn, T bt, T bu, T gamma) {
  T irho = T(1) / rho;
  T gp = gamma * p;
  T b2 = bn * bn + bt * bt + bu * bu;
  T a = (gp + b2) * irho;
  T disc = a * a - T(4) * (gp * irho) * (bn * bn * irho);
  if (disc < T(0)) disc = T(0);
  return T(0.5) * (a + dsqrt(disc));
}
// fast magnetosonic speed along a direction with normal field bn
template <class T> __device__ __forceinline__ T cfast(T rho, T p, T bn, T bt, T bu, T gamma) {
  return dsqrt(cfast2(rho, p, bn, bt, bu, gamma));
}

// conservative -> primitive, always in FP64: p = (g-1)(E - m.m/(2 rho) - B.B/2)
__device__ __forceinline__ void recover(const double* u, const double* bc, double gm1, double* w) {
  double r = u[0];
  double ir = 1.0 / r;
  double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  double ke = 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);
  double me = 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
  w[0] = r; w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = gm1 * ((u[4] - ke) - me);
  w[5] = bc[0]; w[6] = bc[1]; w[7] = bc[2];
}

// Error-free FP32 transformations (Knuth two-sum, FMA two-product): a pair
// (hi, lo) represents hi + lo exactly or to ~2^-46 relative.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
// (ah, al) + (bh, bl)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  h = s + e;
  l = e - (h - s);
}
// (ah, al)^2
__device__ __forceinline__ void df_sq(float ah, float al, float& h, float& l) {
  float p, e;
  two_prod(ah, ah, p, e);
  e = fmaf(2.0f * ah, al, e);
  h = p + e;
  l = e - (h - p);
}

// Recovery of one cell from stored values in the working type T. For T =
// double this is recover() exactly. For the mixed path (T = float) the energy
// balance p = (g-1)(E - ke - me) is evaluated in FP64, with
// ke = |m|^2 / (2 rho) and me = |B_c|^2 / 2 formed from the FP32 inputs by
// error-free FP32 transformations (squares, sums, face means and the division
// by rho carried as hi + lo pairs, ~2^-46 relative), so that the FP64 pipe
// only does the final subtraction and the scaling, its operands widened and
// its result rounded to FP32 (nearest even) on the integer pipe (fp_bits.cuh);
// v = m / rho and B_c are FP32.
__device__ __forceinline__ void recover_t(const double* u, const double* bl, const double* br, double gm1, double* w) {
  double bc[3] = {0.5 * (bl[0] + br[0]), 0.5 * (bl[1] + br[1]), 0.5 * (bl[2] + br[2])};
  recover(u, bc, gm1, w);
}
__device__ __forceinline__ void recover_t(const float* u, const float* bl, const float* br, double gm1, float* w) {
  const float r = u[0];
  const float irf = 1.0f / r;
  // |m|^2 as a pair
  float mh, ml, th, tl;
  two_prod(u[1], u[1], mh, ml);
  two_prod(u[2], u[2], th, tl);
  df_add(mh, ml, th, tl, mh, ml);
  two_prod(u[3], u[3], th, tl);
  df_add(mh, ml, th, tl, mh, ml);
  // ke = 0.5 |m|^2 / rho as a pair: q = mh/r, remainder (mh - q r + ml)/r
  const float q = mh * irf;
  const float q1 = (fmaf(-q, r, mh) + ml) * irf;
  const float q2 = (fmaf(-q1, r, fmaf(-q, r, mh) + ml)) * irf;
  float kh, kl;
  two_sum(q, q1 + q2, kh, kl);
  // |bl + br|^2 summed over components as a pair (me = that / 8)
  float bh = 0.0f, blo = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float sh, se, qh, ql;
    two_sum(bl[c], br[c], sh, se);
    df_sq(sh, se, qh, ql);
    df_add(bh, blo, qh, ql, bh, blo);
  }
  // (ke + me) = 0.5 (kh, kl) + 0.125 (bh, blo): exact power-of-two scalings
  float eh, el;
  df_add(0.5f * kh, 0.5f * kl, 0.125f * bh, 0.125f * blo, eh, el);
  const double p = gm1 * (widen_bits(u[4]) - (widen_bits(eh) + widen_bits(el)));
  w[0] = r;
  w[1] = u[1] * irf;
  w[2] = u[2] * irf;
  w[3] = u[3] * irf;
  w[4] = narrow_bits(p);
  w[5] = 0.5f * (bl[0] + br[0]);
  w[6] = 0.5f * (bl[1] + br[1]);
  w[7] = 0.5f * (bl[2] + br[2]);
}

// floors of the recovery (reading 12): the density before the recovery, the
// pressure after it; each raise counted
template <class T> __device__ __forceinline__ void floor_density(T* u, double rho_min, unsigned long long* events) {
  if (rho_min > 0.0 && u[0] < (T)rho_min) {
    u[0] = (T)rho_min;
    atomicAdd(events, 1ull);
  }
}
template <class T> __device__ __forceinline__ void floor_pressure(T* w, double p_min, unsigned long long* events) {
  if (p_min > 0.0 && w[4] < (T)p_min) {
    w[4] = (T)p_min;
    atomicAdd(events, 1ull);
  }
}

// A_d(W) s for the primitive predictor, direction d (n = d, t = d+1, u = d+2 mod 3)
template <class T, int D> __device__ __forceinline__ void prim_terms(const T* w, const T* s, T gamma, T ir, T* dw) {
  constexpr int n = D, t = (D + 1) % 3, u = (D + 2) % 3;
  const T rho = w[0], p = w[4];
  const T vn = w[1 + n];
  const T bn = w[5 + n], bt = w[5 + t], bu = w[5 + u];
  dw[0] = vn * s[0] + rho * s[1 + n];
  dw[1 + n] = vn * s[1 + n] + (s[4] + bt * s[5 + t] + bu * s[5 + u]) * ir;
  dw[1 + t] = vn * s[1 + t] - bn * s[5 + t] * ir;
  dw[1 + u] = vn * s[1 + u] - bn * s[5 + u] * ir;
  dw[4] = vn * s[4] + gamma * p * s[1 + n];
  dw[5 + n] = vn * s[5 + n];
  dw[5 + t] = vn * s[5 + t] - bn * s[1 + t] + bt * s[1 + n];
  dw[5 + u] = vn * s[5 + u] - bn * s[1 + u] + bu * s[1 + n];
}

// physical flux of a rotated state q = (rho, un, ut, uu, p, bt, bu); u = conserved
template <class T> __device__ __forceinline__ void phys_flux(const T* q, T bn, T igm1, T* f, T* u) {
  const T r = q[0], un = q[1], ut = q[2], uu = q[3], p = q[4], bt = q[5], bu = q[6];
  const T b2 = bn * bn + bt * bt + bu * bu;
  const T pt = p + T(0.5) * b2;
  const T e = p * igm1 + T(0.5) * r * (un * un + ut * ut + uu * uu) + T(0.5) * b2;
  const T vb = un * bn + ut * bt + uu * bu;
  f[0] = r * un;
  f[1] = r * un * un + pt - bn * bn;
  f[2] = r * un * ut - bn * bt;
  f[3] = r * un * uu - bn * bu;
  f[4] = (e + pt) * un - bn * vb;
  f[5] = bt * un - bn * ut;
  f[6] = bu * un - bn * uu;
  u[0] = r; u[1] = r * un; u[2] = r * ut; u[3] = r * uu; u[4] = e; u[5] = bt; u[6] = bu;
}

// Quotients that share a divisor: FP64 divides each time (the written
// formula, bit for bit); FP32 multiplies by one reciprocal (the FP32 path
// compiles its divisions as a reciprocal and a product anyway).
template <class T> struct Quot {
  T d;
  __device__ __forceinline__ explicit Quot(T den) : d(den) {}
  __device__ __forceinline__ T operator()(T num) const { return num / d; }
};
template <> struct Quot<float> {
  float r;
  __device__ __forceinline__ explicit Quot(float den) : r(1.0f / den) {}
  __device__ __forceinline__ float operator()(float num) const { return num * r; }
};

// HLLD flux between rotated states ql, qr with common normal field bn
template <class T> __device__ void hlld_flux(const T* ql, const T* qr, T bn, T gamma, T* f) {
  const T eps = Eps<T>::v();
  const T gm1 = gamma - T(1);
  const T igm1 = T(1) / gm1;
  T fl[7], fr[7], ul[7], ur[7];
  phys_flux(ql, bn, igm1, fl, ul);
  phys_flux(qr, bn, igm1, fr, ur);
  // max(sqrt(a), sqrt(b)) = sqrt(max(a, b)): the square root is monotone and
  // correctly rounded, so one root serves both sides
  const T cl2 = cfast2(ql[0], ql[4], bn, ql[5], ql[6], gamma);
  const T cr2 = cfast2(qr[0], qr[4], bn, qr[5], qr[6], gamma);
  const T cmax = dsqrt(tmaxd(cl2, cr2));
  const T sl = tmind(ql[1], qr[1]) - cmax;
  const T sr = tmaxd(ql[1], qr[1]) + cmax;
  if (sl > T(0)) {
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fl[k];
    return;
  }
  if (sr < T(0)) {
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fr[k];
    return;
  }
  const T bn2 = bn * bn;
  const T rl = ql[0], rr = qr[0];
  const T uln = ql[1], urn = qr[1];
  const T ptl = ql[4] + T(0.5) * (bn2 + ql[5] * ql[5] + ql[6] * ql[6]);
  const T ptr = qr[4] + T(0.5) * (bn2 + qr[5] * qr[5] + qr[6] * qr[6]);
  const T dl = sl - uln, dr = sr - urn;
  const Quot<T> byden(dr * rr - dl * rl);
  const T sm = byden(dr * rr * urn - dl * rl * uln - ptr + ptl);
  const T pts = byden(dr * rr * ptl - dl * rl * ptr + rl * rr * dr * dl * (urn - uln));

  T rs[2], vs[2], ws[2], bts[2], bus[2], es[2], vbs[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const T* q = a == 0 ? ql : qr;
    const T sx = a == 0 ? sl : sr;
    const T da = sx - q[1];
    const T ssm = sx - sm;
    const Quot<T> byssm(ssm);
    rs[a] = byssm(q[0] * da);
    const T rds = q[0] * da * ssm;
    const T e = rds - bn2;
    if (dabs(e) <= eps * (dabs(rds) + bn2)) {
      vs[a] = q[2]; ws[a] = q[3]; bts[a] = q[5]; bus[a] = q[6];
    } else {
      const T ie = T(1) / e;
      const T tq = bn * (sm - q[1]) * ie;
      vs[a] = q[2] - q[5] * tq;
      ws[a] = q[3] - q[6] * tq;
      const T qq = (q[0] * da * da - bn2) * ie;
      bts[a] = q[5] * qq;
      bus[a] = q[6] * qq;
    }
    const T vb = q[1] * bn + q[2] * q[5] + q[3] * q[6];
    vbs[a] = sm * bn + vs[a] * bts[a] + ws[a] * bus[a];
    const T ea = a == 0 ? ul[4] : ur[4];
    es[a] = byssm(da * ea - (a == 0 ? ptl : ptr) * q[1] + pts * sm + bn * (vb - vbs[a]));
  }
  const T usl[7] = {rs[0], rs[0] * sm, rs[0] * vs[0], rs[0] * ws[0], es[0], bts[0], bus[0]};
  const T usr[7] = {rs[1], rs[1] * sm, rs[1] * vs[1], rs[1] * ws[1], es[1], bts[1], bus[1]};
  if (bn2 <= eps * pts) {
    if (sm >= T(0)) {
#pragma unroll
      for (int k = 0; k < 7; ++k) f[k] = fl[k] + sl * (usl[k] - ul[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) f[k] = fr[k] + sr * (usr[k] - ur[k]);
    }
    return;
  }
  const T sql = dsqrt(rs[0]), sqr = dsqrt(rs[1]);
  const T abn = dabs(bn);
  const T sls = sm - abn / sql;
  const T srs = sm + abn / sqr;
  if (sls >= T(0)) {
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fl[k] + sl * (usl[k] - ul[k]);
    return;
  }
  if (srs <= T(0)) {
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fr[k] + sr * (usr[k] - ur[k]);
    return;
  }
  const T sgn = bn > T(0) ? T(1) : T(-1);
  const T idn = T(1) / (sql + sqr);
  const T vss = (sql * vs[0] + sqr * vs[1] + (bts[1] - bts[0]) * sgn) * idn;
  const T wss = (sql * ws[0] + sqr * ws[1] + (bus[1] - bus[0]) * sgn) * idn;
  const T btss = (sql * bts[1] + sqr * bts[0] + sql * sqr * (vs[1] - vs[0]) * sgn) * idn;
  const T buss = (sql * bus[1] + sqr * bus[0] + sql * sqr * (ws[1] - ws[0]) * sgn) * idn;
  const T vbss = sm * bn + vss * btss + wss * buss;
  if (sm >= T(0)) {
    const T ess = es[0] - sql * (vbs[0] - vbss) * sgn;
    const T uss[7] = {rs[0], rs[0] * sm, rs[0] * vss, rs[0] * wss, ess, btss, buss};
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fl[k] + sls * uss[k] - (sls - sl) * usl[k] - sl * ul[k];
  } else {
    const T ess = es[1] + sqr * (vbs[1] - vbss) * sgn;
    const T uss[7] = {rs[1], rs[1] * sm, rs[1] * vss, rs[1] * wss, ess, btss, buss};
#pragma unroll
    for (int k = 0; k < 7; ++k) f[k] = fr[k] + srs * uss[k] - (srs - sr) * usr[k] - sr * ur[k];
  }
}

template <class T> __device__ __forceinline__ T upw(T fm, T lo, T hi) {
  if (fm > T(0)) return lo;
  if (fm < T(0)) return hi;
  return T(0.5) * (lo + hi);
}

// Gardiner-Stone edge EMF at (a-1/2, b-1/2); see the argument names of the
// cell references r[ab] (a-offset, b-offset) and face EMFs/mass fluxes.
template <class T>
__device__ __forceinline__ T gs_emf(T ea_lo, T ea_hi, T eb_lo, T eb_hi, T r00, T r10, T r01, T r11, T fa_lo, T fa_hi,
                                    T fb_lo, T fb_hi) {
  const T db_hi = upw(fa_hi, r01 - eb_lo, r11 - eb_hi);
  const T db_lo = upw(fa_lo, eb_lo - r00, eb_hi - r10);
  const T da_hi = upw(fb_hi, r10 - ea_lo, r11 - ea_hi);
  const T da_lo = upw(fb_lo, ea_lo - r00, ea_hi - r01);
  return T(0.25) * (((ea_hi + ea_lo) + eb_hi) + eb_lo) + T(0.25) * (db_lo - db_hi) + T(0.25) * (da_lo - da_hi);
}

__device__ __forceinline__ double tree2(double a, double b) { return a + b; }
__device__ __forceinline__ double tree4(double a, double b, double c, double d) { return (a + b) + (c + d); }
__device__ __forceinline__ double tree8(const double* v) {
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}

}  // namespace amrdev
