// Hand-written reverse mode of the costliest pointwise formulas of the
// advance: the HLLD flux (hlld_flux), the half-step primitive predictor
// (prim_terms summed over directions) and the recovery. Each function returns the exact
// transposed Jacobian-vector product of the formula in the compute type R
// (double: the FP64 forward; float: the FP32 stencil of the mixed-precision
// forward, with its own degenerate-state threshold), taking the branch the
// forward takes (wave-speed selection, supersonic, degenerate and
// double-star cases); it recomputes the forward's intermediates in the same
// operation order so that every branch decision is the forward's.
// Included by adjoint.cu (compiled without FMA contraction, like the strict
// forward).
#pragma once
#include <type_traits>

#include "mhd_device.cuh"

namespace amrdev {

// physical flux and conserved state of one rotated state: intermediates kept
template <class R> struct PFlux {
  R r, un, ut, uu, p, bt, bu, b2, pt, e, vb, f[7], u[7];
};

template <class R> __device__ __forceinline__ void pflux_fwd(const R* q, R bn, R igm1, PFlux<R>& s) {
  s.r = q[0]; s.un = q[1]; s.ut = q[2]; s.uu = q[3]; s.p = q[4]; s.bt = q[5]; s.bu = q[6];
  s.b2 = bn * bn + s.bt * s.bt + s.bu * s.bu;
  s.pt = s.p + R(0.5) * s.b2;
  s.e = s.p * igm1 + R(0.5) * s.r * (s.un * s.un + s.ut * s.ut + s.uu * s.uu) + R(0.5) * s.b2;
  s.vb = s.un * bn + s.ut * s.bt + s.uu * s.bu;
  s.f[0] = s.r * s.un;
  s.f[1] = s.r * s.un * s.un + s.pt - bn * bn;
  s.f[2] = s.r * s.un * s.ut - bn * s.bt;
  s.f[3] = s.r * s.un * s.uu - bn * s.bu;
  s.f[4] = (s.e + s.pt) * s.un - bn * s.vb;
  s.f[5] = s.bt * s.un - bn * s.ut;
  s.f[6] = s.bu * s.un - bn * s.uu;
  s.u[0] = s.r; s.u[1] = s.r * s.un; s.u[2] = s.r * s.ut; s.u[3] = s.r * s.uu; s.u[4] = s.e;
  s.u[5] = s.bt; s.u[6] = s.bu;
}

// accumulates into gq[7], *gbn the transpose of (f, u)(q, bn) applied to (gf, gu)
template <class R>
__device__ __forceinline__ void pflux_bwd(const PFlux<R>& s, R bn, R igm1, const R* gf, const R* gu, R* gq, R* gbn) {
  R gr = 0, gun = 0, gut = 0, guu = 0, gp = 0, gbt = 0, gbu = 0, gb = 0;
  R ge = gu[4], gpt = 0, gvb = 0;
  // u
  gr += gu[0] + s.un * gu[1] + s.ut * gu[2] + s.uu * gu[3];
  gun += s.r * gu[1];
  gut += s.r * gu[2];
  guu += s.r * gu[3];
  gbt += gu[5];
  gbu += gu[6];
  // f
  gr += s.un * gf[0];
  gun += s.r * gf[0];
  gr += s.un * s.un * gf[1];
  gun += R(2.0) * s.r * s.un * gf[1];
  gpt += gf[1];
  gb -= R(2.0) * bn * gf[1];
  gr += s.un * s.ut * gf[2];
  gun += s.r * s.ut * gf[2];
  gut += s.r * s.un * gf[2];
  gb -= s.bt * gf[2];
  gbt -= bn * gf[2];
  gr += s.un * s.uu * gf[3];
  gun += s.r * s.uu * gf[3];
  guu += s.r * s.un * gf[3];
  gb -= s.bu * gf[3];
  gbu -= bn * gf[3];
  ge += s.un * gf[4];
  gpt += s.un * gf[4];
  gun += (s.e + s.pt) * gf[4];
  gb -= s.vb * gf[4];
  gvb -= bn * gf[4];
  gbt += s.un * gf[5];
  gun += s.bt * gf[5];
  gb -= s.ut * gf[5];
  gut -= bn * gf[5];
  gbu += s.un * gf[6];
  gun += s.bu * gf[6];
  gb -= s.uu * gf[6];
  guu -= bn * gf[6];
  // vb = un bn + ut bt + uu bu
  gun += bn * gvb;
  gb += s.un * gvb;
  gut += s.bt * gvb;
  gbt += s.ut * gvb;
  guu += s.bu * gvb;
  gbu += s.uu * gvb;
  // e = p igm1 + r K / 2 + b2 / 2;  pt = p + b2 / 2
  R gb2 = R(0.5) * ge + R(0.5) * gpt;
  gp += igm1 * ge + gpt;
  gr += R(0.5) * (s.un * s.un + s.ut * s.ut + s.uu * s.uu) * ge;
  gun += s.r * s.un * ge;
  gut += s.r * s.ut * ge;
  guu += s.r * s.uu * ge;
  // b2 = bn^2 + bt^2 + bu^2
  gb += R(2.0) * bn * gb2;
  gbt += R(2.0) * s.bt * gb2;
  gbu += R(2.0) * s.bu * gb2;
  gq[0] += gr; gq[1] += gun; gq[2] += gut; gq[3] += guu; gq[4] += gp; gq[5] += gbt; gq[6] += gbu;
  *gbn += gb;
}

// fast speed cfast(rho, p, bn, bt, bu): value and transpose
template <class R> struct CFast {
  R irho, gp, b2, a, X, Y, disc, sd, c2, cf;
  bool clamp;
};
template <class R>
__device__ __forceinline__ R cfast_fwd(R rho, R p, R bn, R bt, R bu, R gamma, CFast<R>& s) {
  s.irho = R(1.0) / rho;
  s.gp = gamma * p;
  s.b2 = bn * bn + bt * bt + bu * bu;
  s.a = (s.gp + s.b2) * s.irho;
  s.X = s.gp * s.irho;
  s.Y = bn * bn * s.irho;
  s.disc = s.a * s.a - R(4.0) * s.X * s.Y;
  s.clamp = s.disc < R(0.0);
  if (s.clamp) s.disc = R(0.0);
  s.sd = sqrt(s.disc);
  s.c2 = R(0.5) * (s.a + s.sd);
  s.cf = sqrt(s.c2);
  return s.cf;
}
// accumulates d cf / d (rho, p, bn, bt, bu) * g into g5[0..4]
template <class R>
__device__ __forceinline__ void cfast_bwd(const CFast<R>& s, R bn, R bt, R bu, R gamma, R g, R* g5) {
  const R gc2 = g * R(0.5) / s.cf;
  R ga = R(0.5) * gc2;
  const R gsd = R(0.5) * gc2;
  const R gdisc = (s.clamp || s.sd == R(0.0)) ? R(0.0) : gsd * R(0.5) / s.sd;
  ga += R(2.0) * s.a * gdisc;
  const R gX = -R(4.0) * s.Y * gdisc, gY = -R(4.0) * s.X * gdisc;
  R girho = s.gp * gX + bn * bn * gY + (s.gp + s.b2) * ga;
  const R ggp = s.irho * gX + s.irho * ga;
  const R gb2 = s.irho * ga;
  g5[0] += -s.irho * s.irho * girho;
  g5[1] += gamma * ggp;
  g5[2] += R(2.0) * bn * s.irho * gY + R(2.0) * bn * gb2;
  g5[3] += R(2.0) * bt * gb2;
  g5[4] += R(2.0) * bu * gb2;
}

// the star state of one side: intermediates kept
template <class R> struct Star {
  R S, da, ssm, rs, rds, e, ie, tq, qq, vs, ws, bts, bus, vb, vbs, es;
  bool degen;
};

// gx[15] = J^T g of hlld_flux at x = (ql[7], qr[7], bn) (written)
template <class R> __device__ void hlld_vjp(const R* x, const R* g, R gamma, R* gx) {
  const R* ql = x;
  const R* qr = x + 7;
  const R bn = x[14];
  const R eps = Eps<R>::v();
  const R gm1 = gamma - R(1.0);
  const R igm1 = R(1.0) / gm1;
  PFlux<R> FL, FR;
  pflux_fwd(ql, bn, igm1, FL);
  pflux_fwd(qr, bn, igm1, FR);
  CFast<R> cL, cR;
  const R cl = cfast_fwd(ql[0], ql[4], bn, ql[5], ql[6], gamma, cL);
  const R cr = cfast_fwd(qr[0], qr[4], bn, qr[5], qr[6], gamma, cR);
  const bool cmax_l = cl > cr;  // tmaxd(cl, cr)
  const R cmax = cmax_l ? cl : cr;
  const bool smin_l = ql[1] < qr[1];  // tmind(uln, urn)
  const bool smax_l = ql[1] > qr[1];  // tmaxd(uln, urn)
  const R sl = (smin_l ? ql[1] : qr[1]) - cmax;
  const R sr = (smax_l ? ql[1] : qr[1]) + cmax;
  R gql[7] = {0, 0, 0, 0, 0, 0, 0}, gqr[7] = {0, 0, 0, 0, 0, 0, 0}, gbn = R(0.0);
  R gfl[7] = {0, 0, 0, 0, 0, 0, 0}, gfr[7] = {0, 0, 0, 0, 0, 0, 0};
  R gul[7] = {0, 0, 0, 0, 0, 0, 0}, gur[7] = {0, 0, 0, 0, 0, 0, 0};
  R gsl = R(0.0), gsr = R(0.0);
  if (sl > R(0.0) || sr < R(0.0)) {
    R* gf = sl > R(0.0) ? gfl : gfr;
    for (int k = 0; k < 7; ++k) gf[k] = g[k];
  } else {
    const R bn2 = bn * bn;
    const R rl = ql[0], rr = qr[0], uln = ql[1], urn = qr[1];
    const R ptl = ql[4] + R(0.5) * (bn2 + ql[5] * ql[5] + ql[6] * ql[6]);
    const R ptr = qr[4] + R(0.5) * (bn2 + qr[5] * qr[5] + qr[6] * qr[6]);
    const R dl = sl - uln, dr = sr - urn;
    const R den = dr * rr - dl * rl;
    const R nsm = dr * rr * urn - dl * rl * uln - ptr + ptl;
    const R sm = nsm / den;
    const R npt = dr * rr * ptl - dl * rl * ptr + rl * rr * dr * dl * (urn - uln);
    const R pts = npt / den;
    Star<R> st[2];
    for (int a = 0; a < 2; ++a) {
      const R* q = a == 0 ? ql : qr;
      Star<R>& z = st[a];
      z.S = a == 0 ? sl : sr;
      z.da = z.S - q[1];
      z.ssm = z.S - sm;
      z.rs = q[0] * z.da / z.ssm;
      z.rds = q[0] * z.da * z.ssm;
      z.e = z.rds - bn2;
      z.degen = fabs(z.e) <= eps * (fabs(z.rds) + bn2);
      if (z.degen) {
        z.vs = q[2]; z.ws = q[3]; z.bts = q[5]; z.bus = q[6];
      } else {
        z.ie = R(1.0) / z.e;
        z.tq = bn * (sm - q[1]) * z.ie;
        z.vs = q[2] - q[5] * z.tq;
        z.ws = q[3] - q[6] * z.tq;
        z.qq = (q[0] * z.da * z.da - bn2) * z.ie;
        z.bts = q[5] * z.qq;
        z.bus = q[6] * z.qq;
      }
      z.vb = q[1] * bn + q[2] * q[5] + q[3] * q[6];
      z.vbs = sm * bn + z.vs * z.bts + z.ws * z.bus;
      const R ea = a == 0 ? FL.u[4] : FR.u[4];
      const R pta = a == 0 ? ptl : ptr;
      z.es = (z.da * ea - pta * q[1] + pts * sm + bn * (z.vb - z.vbs)) / z.ssm;
    }
    // adjoints of the star quantities
    R grs[2] = {0, 0}, gvs[2] = {0, 0}, gws[2] = {0, 0}, gbts[2] = {0, 0}, gbus[2] = {0, 0}, ges[2] = {0, 0};
    R gvbs[2] = {0, 0};
    R gsm = R(0.0), gpts = R(0.0);
    // us = (rs, rs sm, rs vs, rs ws, es, bts, bus): transpose of a side's star state
    // sides as compile-time constants (I0 / I1) keep every per-side array in registers
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    auto us_bwd = [&](auto A, const R* gus) {
      constexpr int a = decltype(A)::value;
      const Star<R>& z = st[a];
      grs[a] += gus[0] + sm * gus[1] + z.vs * gus[2] + z.ws * gus[3];
      gsm += z.rs * gus[1];
      gvs[a] += z.rs * gus[2];
      gws[a] += z.rs * gus[3];
      ges[a] += gus[4];
      gbts[a] += gus[5];
      gbus[a] += gus[6];
    };
    auto us_val = [&](auto A, int k) {
      constexpr int a = decltype(A)::value;
      const Star<R>& z = st[a];
      switch (k) {
        case 0: return z.rs;
        case 1: return z.rs * sm;
        case 2: return z.rs * z.vs;
        case 3: return z.rs * z.ws;
        case 4: return z.es;
        case 5: return z.bts;
        default: return z.bus;
      }
    };
    // f = fa + Sa (usa - ua)
    auto single_star = [&](auto A) {
      constexpr int a = decltype(A)::value;
      const R S = a == 0 ? sl : sr;
      const R* u = a == 0 ? FL.u : FR.u;
      R* gf = a == 0 ? gfl : gfr;
      R* gu = a == 0 ? gul : gur;
      R gus[7];
      R gS = R(0.0);
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        gf[k] += g[k];
        gS += (us_val(A, k) - u[k]) * g[k];
        gus[k] = S * g[k];
        gu[k] -= S * g[k];
      }
      us_bwd(A, gus);
      if (a == 0) gsl += gS;
      else gsr += gS;
    };
    if (bn2 <= eps * pts) {
      if (sm >= R(0.0)) single_star(I0{});
      else single_star(I1{});
    } else {
      const R sql = sqrt(st[0].rs), sqr = sqrt(st[1].rs);
      const R abn = fabs(bn);
      const R sls = sm - abn / sql;
      const R srs = sm + abn / sqr;
      if (sls >= R(0.0)) {
        single_star(I0{});
      } else if (srs <= R(0.0)) {
        single_star(I1{});
      } else {
        const R sgn = bn > R(0.0) ? R(1.0) : -R(1.0);
        const R isum = sql + sqr;
        const R idn = R(1.0) / isum;
        const R nv = sql * st[0].vs + sqr * st[1].vs + (st[1].bts - st[0].bts) * sgn;
        const R nw = sql * st[0].ws + sqr * st[1].ws + (st[1].bus - st[0].bus) * sgn;
        const R nbt = sql * st[1].bts + sqr * st[0].bts + sql * sqr * (st[1].vs - st[0].vs) * sgn;
        const R nbu = sql * st[1].bus + sqr * st[0].bus + sql * sqr * (st[1].ws - st[0].ws) * sgn;
        const R vss = nv * idn, wss = nw * idn, btss = nbt * idn, buss = nbu * idn;
        const R vbss = sm * bn + vss * btss + wss * buss;
        auto double_star = [&](auto A) {
        constexpr int a = decltype(A)::value;
        const Star<R>& z = st[a];
        const R sq = a == 0 ? sql : sqr;
        const R ss = a == 0 ? sls : srs;  // S*
        const R S = a == 0 ? sl : sr;
        const R* u = a == 0 ? FL.u : FR.u;
        R* gf = a == 0 ? gfl : gfr;
        R* gu = a == 0 ? gul : gur;
        // ess = es_a -/+ sq (vbs_a - vbss) sgn
        const R sgn_side = a == 0 ? -R(1.0) : R(1.0);
        const R ess = z.es + sgn_side * sq * (z.vbs - vbss) * sgn;
        const R uss[7] = {z.rs, z.rs * sm, z.rs * vss, z.rs * wss, ess, btss, buss};
        // f = fa + S* uss - (S* - S) usa - S ua
        R guss[7], gusa[7];
        R gss = R(0.0), gS = R(0.0);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const R usa = us_val(A, k);
          gf[k] += g[k];
          gss += (uss[k] - usa) * g[k];
          guss[k] = ss * g[k];
          gusa[k] = -(ss - S) * g[k];
          gS += (usa - u[k]) * g[k];
          gu[k] -= S * g[k];
        }
        if (a == 0) gsl += gS;
        else gsr += gS;
        us_bwd(A, gusa);
        // uss = (rs_a, rs_a sm, rs_a vss, rs_a wss, ess, btss, buss)
        R gvss = z.rs * guss[2], gwss = z.rs * guss[3], gbtss = guss[5], gbuss = guss[6];
        grs[a] += guss[0] + sm * guss[1] + vss * guss[2] + wss * guss[3];
        gsm += z.rs * guss[1];
        const R gess = guss[4];
        // ess
        ges[a] += gess;
        R gsq = sgn_side * (z.vbs - vbss) * sgn * gess;
        gvbs[a] += sgn_side * sq * sgn * gess;
        R gvbss = -sgn_side * sq * sgn * gess;
        // vbss = sm bn + vss btss + wss buss
        gsm += bn * gvbss;
        gbn += sm * gvbss;
        gvss += btss * gvbss;
        gbtss += vss * gvbss;
        gwss += buss * gvbss;
        gbuss += wss * gvbss;
        // vss = nv idn etc.
        R gidn = nv * gvss + nw * gwss + nbt * gbtss + nbu * gbuss;
        const R gnv = idn * gvss, gnw = idn * gwss, gnbt = idn * gbtss, gnbu = idn * gbuss;
        R gsql = R(0.0), gsqr = R(0.0);
        gsql += st[0].vs * gnv + st[0].ws * gnw + st[1].bts * gnbt + st[1].bus * gnbu +
                sqr * (st[1].vs - st[0].vs) * sgn * gnbt + sqr * (st[1].ws - st[0].ws) * sgn * gnbu;
        gsqr += st[1].vs * gnv + st[1].ws * gnw + st[0].bts * gnbt + st[0].bus * gnbu +
                sql * (st[1].vs - st[0].vs) * sgn * gnbt + sql * (st[1].ws - st[0].ws) * sgn * gnbu;
        gvs[0] += sql * gnv - sql * sqr * sgn * gnbt;
        gvs[1] += sqr * gnv + sql * sqr * sgn * gnbt;
        gws[0] += sql * gnw - sql * sqr * sgn * gnbu;
        gws[1] += sqr * gnw + sql * sqr * sgn * gnbu;
        gbts[0] += -sgn * gnv + sqr * gnbt;
        gbts[1] += sgn * gnv + sql * gnbt;
        gbus[0] += -sgn * gnw + sqr * gnbu;
        gbus[1] += sgn * gnw + sql * gnbu;
        // idn = 1 / (sql + sqr)
        const R gisum = -idn * idn * gidn;
        gsql += gisum;
        gsqr += gisum;
        // S* = sm -/+ abn / sq
        gsm += gss;
        if (a == 0) {
          gsql += abn / (sql * sql) * gss;
          gbn += -(bn > R(0.0) ? R(1.0) : (bn < R(0.0) ? -R(1.0) : R(0.0))) / sql * gss;
        } else {
          gsqr += -abn / (sqr * sqr) * gss;
          gbn += (bn > R(0.0) ? R(1.0) : (bn < R(0.0) ? -R(1.0) : R(0.0))) / sqr * gss;
        }
        if (a == 0) gsql += gsq;
        else gsqr += gsq;
        // sq = sqrt(rs)
        grs[0] += R(0.5) / sql * gsql;
        grs[1] += R(0.5) / sqr * gsqr;
        };
        if (sm >= R(0.0)) double_star(I0{});
        else double_star(I1{});
      }
    }
    // the two sides' star quantities, in reverse
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const R* q = a == 0 ? ql : qr;
      R* gq = a == 0 ? gql : gqr;
      R* gu = a == 0 ? gul : gur;
      const Star<R>& z = st[a];
      const R ea = a == 0 ? FL.u[4] : FR.u[4];
      const R pta = a == 0 ? ptl : ptr;
      // es = (da ea - pta un + pts sm + bn (vb - vbs)) / ssm
      const R nes = z.da * ea - pta * q[1] + pts * sm + bn * (z.vb - z.vbs);
      const R gnes = ges[a] / z.ssm;
      R gssm = -nes / (z.ssm * z.ssm) * ges[a];
      R gda = ea * gnes;
      gu[4] += z.da * gnes;
      R gpta = -q[1] * gnes;
      gq[1] += -pta * gnes;
      gpts += sm * gnes;
      gsm += pts * gnes;
      gbn += (z.vb - z.vbs) * gnes;
      R gvb = bn * gnes;
      gvbs[a] += -bn * gnes;
      // vbs = sm bn + vs bts + ws bus
      gsm += bn * gvbs[a];
      gbn += sm * gvbs[a];
      gvs[a] += z.bts * gvbs[a];
      gbts[a] += z.vs * gvbs[a];
      gws[a] += z.bus * gvbs[a];
      gbus[a] += z.ws * gvbs[a];
      // vb = un bn + ut bt + uu bu
      gq[1] += bn * gvb;
      gbn += q[1] * gvb;
      gq[2] += q[5] * gvb;
      gq[5] += q[2] * gvb;
      gq[3] += q[6] * gvb;
      gq[6] += q[3] * gvb;
      if (z.degen) {
        gq[2] += gvs[a];
        gq[3] += gws[a];
        gq[5] += gbts[a];
        gq[6] += gbus[a];
      } else {
        // bts = bt qq, bus = bu qq, vs = ut - bt tq, ws = uu - bu tq
        R gqq = q[5] * gbts[a] + q[6] * gbus[a];
        gq[5] += z.qq * gbts[a] - z.tq * gvs[a];
        gq[6] += z.qq * gbus[a] - z.tq * gws[a];
        gq[2] += gvs[a];
        gq[3] += gws[a];
        R gtq = -q[5] * gvs[a] - q[6] * gws[a];
        // qq = (r da^2 - bn2) ie; tq = bn (sm - un) ie
        R gie = (q[0] * z.da * z.da - bn2) * gqq + bn * (sm - q[1]) * gtq;
        gq[0] += z.da * z.da * z.ie * gqq;
        gda += R(2.0) * q[0] * z.da * z.ie * gqq;
        gbn += -R(2.0) * bn * z.ie * gqq + (sm - q[1]) * z.ie * gtq;
        gsm += bn * z.ie * gtq;
        gq[1] += -bn * z.ie * gtq;
        // ie = 1/e; e = rds - bn2; rds = r da ssm
        const R ge = -z.ie * z.ie * gie;
        const R grds = ge;
        gbn += -R(2.0) * bn * ge;
        gq[0] += z.da * z.ssm * grds;
        gda += q[0] * z.ssm * grds;
        gssm += q[0] * z.da * grds;
      }
      // rs = r da / ssm
      gq[0] += z.da / z.ssm * grs[a];
      gda += q[0] / z.ssm * grs[a];
      gssm += -z.rs / z.ssm * grs[a];
      // ssm = S - sm; da = S - un
      R gS = gssm + gda;
      gsm += -gssm;
      gq[1] += -gda;
      if (a == 0) gsl += gS;
      else gsr += gS;
      // pta = p + (bn2 + bt^2 + bu^2) / 2
      gq[4] += gpta;
      gbn += bn * gpta;
      gq[5] += q[5] * gpta;
      gq[6] += q[6] * gpta;
    }
    // sm = nsm / den; pts = npt / den
    const R gnsm = gsm / den, gnpt = gpts / den;
    const R gden = -sm / den * gsm - pts / den * gpts;
    // den = dr rr - dl rl
    R gdr = rr * gden, gdl = -rl * gden;
    R grr = dr * gden, grl = -dl * gden;
    // nsm = dr rr urn - dl rl uln - ptr + ptl
    gdr += rr * urn * gnsm;
    grr += dr * urn * gnsm;
    gqr[1] += dr * rr * gnsm;
    gdl += -rl * uln * gnsm;
    grl += -dl * uln * gnsm;
    gql[1] += -dl * rl * gnsm;
    R gptr = -gnsm, gptl = gnsm;
    // npt = dr rr ptl - dl rl ptr + rl rr dr dl (urn - uln)
    const R du = urn - uln;
    gdr += rr * ptl * gnpt + rl * rr * dl * du * gnpt;
    grr += dr * ptl * gnpt + rl * dr * dl * du * gnpt;
    gptl += dr * rr * gnpt;
    gdl += -rl * ptr * gnpt + rl * rr * dr * du * gnpt;
    grl += -dl * ptr * gnpt + rr * dr * dl * du * gnpt;
    gptr += -dl * rl * gnpt;
    gqr[1] += rl * rr * dr * dl * gnpt;
    gql[1] += -rl * rr * dr * dl * gnpt;
    // dl = sl - uln; dr = sr - urn
    gsl += gdl;
    gql[1] += -gdl;
    gsr += gdr;
    gqr[1] += -gdr;
    gql[0] += grl;
    gqr[0] += grr;
    // ptl, ptr
    gql[4] += gptl;
    gbn += bn * gptl + bn * gptr;
    gql[5] += ql[5] * gptl;
    gql[6] += ql[6] * gptl;
    gqr[4] += gptr;
    gqr[5] += qr[5] * gptr;
    gqr[6] += qr[6] * gptr;
  }
  // sl = min(uln, urn) - cmax; sr = max(uln, urn) + cmax
  if (gsl != R(0.0) || gsr != R(0.0)) {
    if (smin_l) gql[1] += gsl;
    else gqr[1] += gsl;
    if (smax_l) gql[1] += gsr;
    else gqr[1] += gsr;
    const R gcmax = gsr - gsl;
    R g5[5] = {0, 0, 0, 0, 0};
    if (cmax_l) {
      cfast_bwd(cL, bn, ql[5], ql[6], gamma, gcmax, g5);
      gql[0] += g5[0]; gql[4] += g5[1]; gbn += g5[2]; gql[5] += g5[3]; gql[6] += g5[4];
    } else {
      cfast_bwd(cR, bn, qr[5], qr[6], gamma, gcmax, g5);
      gqr[0] += g5[0]; gqr[4] += g5[1]; gbn += g5[2]; gqr[5] += g5[3]; gqr[6] += g5[4];
    }
  }
  pflux_bwd(FL, bn, igm1, gfl, gul, gql, &gbn);
  pflux_bwd(FR, bn, igm1, gfr, gur, gqr, &gbn);
  for (int k = 0; k < 7; ++k) {
    gx[k] = gql[k];
    gx[7 + k] = gqr[k];
  }
  gx[14] = gbn;
}

// transpose of dw = A_D(w) s (prim_terms) applied to G: accumulates into gw, gs
// and the adjoint of ir = 1 / rho
template <int D, class R>
__device__ __forceinline__ void prim_terms_vjp(const R* w, const R* s, R gamma, R ir, const R* G, R* gw, R* gs,
                                               R& gir) {
  constexpr int n = D, t = (D + 1) % 3, u = (D + 2) % 3;
  const R rho = w[0], p = w[4];
  const R vn = w[1 + n];
  const R bn = w[5 + n], bt = w[5 + t], bu = w[5 + u];
  // every component carries vn s_f: d/dvn = s . G, d/ds_f += vn G_f
  R sg = R(0.0);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    sg += s[f] * G[f];
    gs[f] += vn * G[f];
  }
  gw[1 + n] += sg;
  // dw0: rho s[1+n]
  gw[0] += s[1 + n] * G[0];
  gs[1 + n] += rho * G[0];
  // dw[1+n]: (s4 + bt s[5+t] + bu s[5+u]) ir
  const R pn = s[4] + bt * s[5 + t] + bu * s[5 + u];
  gir += pn * G[1 + n];
  gs[4] += ir * G[1 + n];
  gs[5 + t] += bt * ir * G[1 + n];
  gs[5 + u] += bu * ir * G[1 + n];
  gw[5 + t] += s[5 + t] * ir * G[1 + n];
  gw[5 + u] += s[5 + u] * ir * G[1 + n];
  // dw[1+t], dw[1+u]: - bn s[5+t] ir, - bn s[5+u] ir
  gw[5 + n] -= (s[5 + t] * G[1 + t] + s[5 + u] * G[1 + u]) * ir;
  gs[5 + t] -= bn * ir * G[1 + t];
  gs[5 + u] -= bn * ir * G[1 + u];
  gir -= bn * (s[5 + t] * G[1 + t] + s[5 + u] * G[1 + u]);
  // dw4: gamma p s[1+n]
  gw[4] += gamma * s[1 + n] * G[4];
  gs[1 + n] += gamma * p * G[4];
  // dw[5+t], dw[5+u]: - bn s[1+t] + bt s[1+n], - bn s[1+u] + bu s[1+n]
  gw[5 + n] -= s[1 + t] * G[5 + t] + s[1 + u] * G[5 + u];
  gs[1 + t] -= bn * G[5 + t];
  gs[1 + u] -= bn * G[5 + u];
  gw[5 + t] += s[1 + n] * G[5 + t];
  gw[5 + u] += s[1 + n] * G[5 + u];
  gs[1 + n] += bt * G[5 + t] + bu * G[5 + u];
}

// gx = J^T g of the half-step predictor wh = w - sum_d h_d A_d(w) s_d at
// x = (w[8], s_0[8], .., s_{DIM-1}[8]); gx has 8 + 8 DIM entries (written)
template <int DIM, class R>
__device__ __forceinline__ void predict_vjp(const R* x, const R* g, R gamma, const R* h, R* gx) {
  const R* w = x;
  const R ir = R(1.0) / w[0];
  R gir = R(0.0);
#pragma unroll
  for (int f = 0; f < 8; ++f) gx[f] = g[f];
#pragma unroll
  for (int q = 8; q < 8 + 8 * DIM; ++q) gx[q] = R(0.0);
  R G[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) G[f] = -h[0] * g[f];
  prim_terms_vjp<0>(w, x + 8, gamma, ir, G, gx, gx + 8, gir);
#pragma unroll
  for (int f = 0; f < 8; ++f) G[f] = -h[1] * g[f];
  prim_terms_vjp<1>(w, x + 16, gamma, ir, G, gx, gx + 16, gir);
  if (DIM == 3) {
#pragma unroll
    for (int f = 0; f < 8; ++f) G[f] = -h[2] * g[f];
    prim_terms_vjp<2>(w, x + 24, gamma, ir, G, gx, gx + 24, gir);
  }
  gx[0] -= ir * ir * gir;
}

// gx[8] = J^T g of the FP64 recovery W(U, B_c) (recover() in mhd_device.cuh): x = (rho,
// m_x, m_y, m_z, E, B_cx, B_cy, B_cz), W = (rho, v, p, B_c), p = gm1 ((E - ke) - me)
__device__ __forceinline__ void recover_vjp(const double* x, const double* g, double gm1, double* gx) {
  const double r = x[0], ir = 1.0 / r;
  const double vx = x[1] * ir, vy = x[2] * ir, vz = x[3] * ir;
  const double gp = g[4];
  const double gke = -gm1 * gp, gme = -gm1 * gp;
  // ke = (m_x vx + m_y vy + m_z vz) / 2; v = m ir
  const double gvx = g[1] + 0.5 * x[1] * gke, gvy = g[2] + 0.5 * x[2] * gke, gvz = g[3] + 0.5 * x[3] * gke;
  const double gir = x[1] * gvx + x[2] * gvy + x[3] * gvz;
  gx[0] = g[0] - ir * ir * gir;
  gx[1] = 0.5 * vx * gke + ir * gvx;
  gx[2] = 0.5 * vy * gke + ir * gvy;
  gx[3] = 0.5 * vz * gke + ir * gvz;
  gx[4] = gm1 * gp;
  // me = |B_c|^2 / 2
  gx[5] = g[5] + x[5] * gme;
  gx[6] = g[6] + x[6] * gme;
  gx[7] = g[7] + x[7] * gme;
}

}  // namespace amrdev
