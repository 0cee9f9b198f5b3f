// Oracle physics core: the per-cell, per-face and per-edge formulas of the
// ideal-MHD level advance, written out plainly in the operation order that the
// scheme fixes. TEST INFRASTRUCTURE ONLY: nothing on the product path may
// include, link or call this file; only tests/, the smoke check and the CPU
// baseline leg of the benchmark use it.
//
// The paper (Carroll-Nellenback et al., "Efficient Parallelization for AMR MHD
// Multiphysics Calculations") names the hyperbolic advance of each grid
// (Abstract, Sec. 1) but never states the numerical scheme. The scheme below
// is the one the hot path is specified with, and every point where a choice
// had to be made is a numbered reading (R1..R16), restated where it is used:
//   R1  MUSCL-Hancock with the primitive-variable half-step predictor,
//       unsplit; the v(div B) term of the induction equation is dropped.
//   R2  minmod(a, b) = 0 unless a, b have the same strict sign, else the one
//       of smaller magnitude, a on a tie; a = backward, b = forward difference.
//       The slope of the normal B component in its own direction is the
//       unlimited difference of the two face values.
//   R3  The HLLD normal field is the mean of the normal B of the two predicted
//       face states.
//   R4  HLLD (Miyoshi & Kusano 2005): fast speed from the face state, wave
//       speeds S_L = min(uL,uR) - max(cfL,cfR), S_R = max(uL,uR) + max(cfL,cfR);
//       degenerate star state when |e| <= eps (|rho (S-u)(S-S_M)| + Bn^2),
//       double-star states skipped when Bn^2 <= eps p_T*;  eps = 1e-12 (FP64).
//   R5  CT edge EMFs: Gardiner & Stone upwinded average of the four face
//       EMFs with cell-centre reference -(v x B) at the half step, upwinded by
//       the sign of the face mass flux, the mean of both sides at exactly 0.
//   Transverse rotation: at a d-face the normal is d, t1 = (d+1) mod 3,
//   t2 = (d+2) mod 3.
#pragma once
#include <cmath>

namespace oracle {

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7, NFIELD = 8 };

using std::sqrt;
using std::fabs;

template <class T> inline T tmax(T a, T b) { return a > b ? a : b; }
template <class T> inline T tmin(T a, T b) { return a < b ? a : b; }

// R2: minmod with a = backward difference, b = forward difference.
template <class T> inline T minmod(T a, T b) {
  if (a > T(0) && b > T(0)) return (a <= b) ? a : b;
  if (a < T(0) && b < T(0)) return (a >= b) ? a : b;
  return T(0);
}

// Fast magnetosonic speed along a direction with normal field bn:
// c_f^2 = 1/2 [ (g p + |B|^2)/rho + sqrt(((g p + |B|^2)/rho)^2 - 4 g p bn^2 / rho^2) ].
template <class T> inline T fast_speed(T rho, T p, T bn, T bt, T bu, T gamma) {
  T irho = T(1) / rho;
  T gp = gamma * p;
  T b2 = bn * bn + bt * bt + bu * bu;
  T a = (gp + b2) * irho;
  T disc = a * a - T(4) * (gp * irho) * (bn * bn * irho);
  if (disc < T(0)) disc = T(0);
  return sqrt(T(0.5) * (a + sqrt(disc)));
}

// Conservative -> primitive recovery of one cell (a3).
// u: rho, mx, my, mz, E; bc: cell-centred B (mean of the two faces per
// component; in 2D Bz is itself cell-centred). Output w: rho, vx, vy, vz, p,
// bx, by, bz. p = (g-1) (E - |m|^2/(2 rho) - |B|^2/2).
template <class T> inline void cons_to_prim(const T* u, const T* bc, T gm1, T* w) {
  T r = u[RHO];
  T ir = T(1) / r;
  T vx = u[MX] * ir, vy = u[MY] * ir, vz = u[MZ] * ir;
  T ke = T(0.5) * (u[MX] * vx + u[MY] * vy + u[MZ] * vz);
  T me = T(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
  w[0] = r; w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = gm1 * ((u[EN] - ke) - me);
  w[5] = bc[0]; w[6] = bc[1]; w[7] = bc[2];
}

// R1: primitive-form quasi-linear term A_d(W) s for direction d, where s is
// the slope vector (difference per cell) of W in direction d.
template <class T> inline void prim_rhs(const T* w, const T* s, int d, T gamma, T ir, T* dw) {
  const int n = d, t = (d + 1) % 3, u = (d + 2) % 3;
  T rho = w[0], p = w[4];
  T vn = w[1 + n];
  T bn = w[5 + n], bt = w[5 + t], bu = w[5 + u];
  dw[0] = vn * s[0] + rho * s[1 + n];
  dw[1 + n] = vn * s[1 + n] + (s[4] + bt * s[5 + t] + bu * s[5 + u]) * ir;
  dw[1 + t] = vn * s[1 + t] - bn * s[5 + t] * ir;
  dw[1 + u] = vn * s[1 + u] - bn * s[5 + u] * ir;
  dw[4] = vn * s[4] + gamma * p * s[1 + n];
  dw[5 + n] = vn * s[5 + n];
  dw[5 + t] = vn * s[5 + t] - bn * s[1 + t] + bt * s[1 + n];
  dw[5 + u] = vn * s[5 + u] - bn * s[1 + u] + bu * s[1 + n];
}

// Ideal-MHD flux along the normal of a rotated state.
// q: rho, un, ut, uu, p, bt, bu (normal field bn given separately).
// f: rho, m_n, m_t, m_u, E, B_t, B_u.  e: total energy of the state.
template <class T> inline void mhd_flux(const T* q, T bn, T igm1, T* f, T* cons) {
  T r = q[0], un = q[1], ut = q[2], uu = q[3], p = q[4], bt = q[5], bu = q[6];
  T b2 = bn * bn + bt * bt + bu * bu;
  T pt = p + T(0.5) * b2;
  T e = p * igm1 + T(0.5) * r * (un * un + ut * ut + uu * uu) + T(0.5) * b2;
  T vb = un * bn + ut * bt + uu * bu;
  f[0] = r * un;
  f[1] = r * un * un + pt - bn * bn;
  f[2] = r * un * ut - bn * bt;
  f[3] = r * un * uu - bn * bu;
  f[4] = (e + pt) * un - bn * vb;
  f[5] = bt * un - bn * ut;
  f[6] = bu * un - bn * uu;
  cons[0] = r; cons[1] = r * un; cons[2] = r * ut; cons[3] = r * uu;
  cons[4] = e; cons[5] = bt; cons[6] = bu;
}

// R4: HLLD flux (Miyoshi & Kusano 2005) between rotated states ql, qr with
// common normal field bn. Output f as in mhd_flux.
template <class T> inline void hlld(const T* ql, const T* qr, T bn, T gamma, T eps, T* f) {
  const T gm1 = gamma - T(1);
  const T igm1 = T(1) / gm1;
  T fl[7], fr[7], ul[7], ur[7];
  mhd_flux(ql, bn, igm1, fl, ul);
  mhd_flux(qr, bn, igm1, fr, ur);
  T cfl = fast_speed(ql[0], ql[4], bn, ql[5], ql[6], gamma);
  T cfr = fast_speed(qr[0], qr[4], bn, qr[5], qr[6], gamma);
  T cmax = tmax(cfl, cfr);
  T sl = tmin(ql[1], qr[1]) - cmax;
  T sr = tmax(ql[1], qr[1]) + cmax;
  if (sl > T(0)) { for (int k = 0; k < 7; ++k) f[k] = fl[k]; return; }
  if (sr < T(0)) { for (int k = 0; k < 7; ++k) f[k] = fr[k]; return; }
  T bn2 = bn * bn;
  T rl = ql[0], rr = qr[0];
  T uln = ql[1], urn = qr[1];
  T ptl = ql[4] + T(0.5) * (bn2 + ql[5] * ql[5] + ql[6] * ql[6]);
  T ptr = qr[4] + T(0.5) * (bn2 + qr[5] * qr[5] + qr[6] * qr[6]);
  T dl = sl - uln, dr = sr - urn;
  T den = dr * rr - dl * rl;
  T sm = (dr * rr * urn - dl * rl * uln - ptr + ptl) / den;
  T pts = (dr * rr * ptl - dl * rl * ptr + rl * rr * dr * dl * (urn - uln)) / den;

  // star states, side by side: index 0 = left, 1 = right
  T rs[2], vs[2], ws[2], bts[2], bus[2], es[2], vbs[2];
  const T* qs[2] = {ql, qr};
  const T sx[2] = {sl, sr};
  const T* us[2] = {ul, ur};
  for (int a = 0; a < 2; ++a) {
    const T* q = qs[a];
    T da = sx[a] - q[1];
    T ssm = sx[a] - sm;
    rs[a] = q[0] * da / ssm;
    T rds = q[0] * da * ssm;
    T e = rds - bn2;
    if (fabs(e) <= eps * (fabs(rds) + bn2)) {
      vs[a] = q[2]; ws[a] = q[3]; bts[a] = q[5]; bus[a] = q[6];
    } else {
      T ie = T(1) / e;
      T tq = bn * (sm - q[1]) * ie;
      vs[a] = q[2] - q[5] * tq;
      ws[a] = q[3] - q[6] * tq;
      T qq = (q[0] * da * da - bn2) * ie;
      bts[a] = q[5] * qq;
      bus[a] = q[6] * qq;
    }
    T vb = q[1] * bn + q[2] * q[5] + q[3] * q[6];
    vbs[a] = sm * bn + vs[a] * bts[a] + ws[a] * bus[a];
    es[a] = (da * us[a][4] - (a == 0 ? ptl : ptr) * q[1] + pts * sm + bn * (vb - vbs[a])) / ssm;
  }
  T usl[7] = {rs[0], rs[0] * sm, rs[0] * vs[0], rs[0] * ws[0], es[0], bts[0], bus[0]};
  T usr[7] = {rs[1], rs[1] * sm, rs[1] * vs[1], rs[1] * ws[1], es[1], bts[1], bus[1]};

  if (bn2 <= eps * pts) {
    if (sm >= T(0)) { for (int k = 0; k < 7; ++k) f[k] = fl[k] + sl * (usl[k] - ul[k]); }
    else            { for (int k = 0; k < 7; ++k) f[k] = fr[k] + sr * (usr[k] - ur[k]); }
    return;
  }
  T sql = sqrt(rs[0]), sqr = sqrt(rs[1]);
  T abn = fabs(bn);
  T sls = sm - abn / sql;
  T srs = sm + abn / sqr;
  if (sls >= T(0)) { for (int k = 0; k < 7; ++k) f[k] = fl[k] + sl * (usl[k] - ul[k]); return; }
  if (srs <= T(0)) { for (int k = 0; k < 7; ++k) f[k] = fr[k] + sr * (usr[k] - ur[k]); return; }
  T sgn = bn > T(0) ? T(1) : T(-1);
  T idn = T(1) / (sql + sqr);
  T vss = (sql * vs[0] + sqr * vs[1] + (bts[1] - bts[0]) * sgn) * idn;
  T wss = (sql * ws[0] + sqr * ws[1] + (bus[1] - bus[0]) * sgn) * idn;
  T btss = (sql * bts[1] + sqr * bts[0] + sql * sqr * (vs[1] - vs[0]) * sgn) * idn;
  T buss = (sql * bus[1] + sqr * bus[0] + sql * sqr * (ws[1] - ws[0]) * sgn) * idn;
  T vbss = sm * bn + vss * btss + wss * buss;
  if (sm >= T(0)) {
    T ess = es[0] - sql * (vbs[0] - vbss) * sgn;
    T uss[7] = {rs[0], rs[0] * sm, rs[0] * vss, rs[0] * wss, ess, btss, buss};
    for (int k = 0; k < 7; ++k) f[k] = fl[k] + sls * uss[k] - (sls - sl) * usl[k] - sl * ul[k];
  } else {
    T ess = es[1] + sqr * (vbs[1] - vbss) * sgn;
    T uss[7] = {rs[1], rs[1] * sm, rs[1] * vss, rs[1] * wss, ess, btss, buss};
    for (int k = 0; k < 7; ++k) f[k] = fr[k] + srs * uss[k] - (srs - sr) * usr[k] - sr * ur[k];
  }
}

// R5 upwind selector: lo if the mass flux is positive, hi if negative, mean at 0.
template <class T> inline T upwind(T fmass, T lo, T hi) {
  if (fmass > T(0)) return lo;
  if (fmass < T(0)) return hi;
  return T(0.5) * (lo + hi);
}

// R5: Gardiner-Stone edge EMF E_c at edge (a-1/2, b-1/2) in the (a,b) plane,
// (a, b, c) cyclic. ea_lo/ea_hi: E_c from the a-faces at rows b-1 and b;
// eb_lo/eb_hi: E_c from the b-faces at columns a-1 and a; r00, r10, r01, r11:
// reference E_c at cells (a-1,b-1), (a,b-1), (a-1,b), (a,b); fa_lo/fa_hi: mass
// fluxes through the a-faces; fb_lo/fb_hi: through the b-faces.
template <class T> inline T gs_edge_emf(T ea_lo, T ea_hi, T eb_lo, T eb_hi,
                                        T r00, T r10, T r01, T r11,
                                        T fa_lo, T fa_hi, T fb_lo, T fb_hi) {
  T db_hi = upwind(fa_hi, r01 - eb_lo, r11 - eb_hi);
  T db_lo = upwind(fa_lo, eb_lo - r00, eb_hi - r10);
  T da_hi = upwind(fb_hi, r10 - ea_lo, r11 - ea_hi);
  T da_lo = upwind(fb_lo, ea_lo - r00, ea_hi - r01);
  return T(0.25) * (((ea_hi + ea_lo) + eb_hi) + eb_lo) + T(0.25) * (db_lo - db_hi) +
         T(0.25) * (da_lo - da_hi);
}

}  // namespace oracle
