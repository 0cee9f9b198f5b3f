// Staged level-advance kernels and the ghost-fill, prolongation, register,
// reflux, restriction, CFL and I/O kernels. Included by one translation unit
// per compilation mode with AMRK_NS set to a distinct namespace.
//
// Work decomposition: every launch batches all patches of a level: blockIdx.y
// selects the patch, blockIdx.x/threadIdx.x the cell (or face/edge) of that
// patch's region; patches of uneven size leave surplus blocks idle. Map-driven
// kernels run one thread per map row, each row writing one destination value
// set (no atomics, deterministic).
#include <algorithm>

#include "hierarchy.hpp"
#include "kernels.hpp"
#include "mhd_device.cuh"

#ifndef AMRK_NS
#error "AMRK_NS must name the instantiation namespace"
#endif

namespace AMRK_NS {
using namespace amrk;
using namespace amrdev;

constexpr int TPB = 256;

__host__ __device__ __forceinline__ int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

// region = interior widened by m layers; thread t -> local storage coords
template <int DIM>
__device__ __forceinline__ bool region_cell(const DPatch& P, int m, int t, int& i, int& j, int& k) {
  const int rx = P.n[0] + 2 * m, ry = P.n[1] + 2 * m, rz = DIM == 3 ? P.n[2] + 2 * m : 1;
  if (t >= rx * ry * rz) return false;
  i = 4 - m + t % rx;
  j = 4 - m + (t / rx) % ry;
  k = DIM == 3 ? 4 - m + t / (rx * ry) : 0;
  return true;
}

__device__ __forceinline__ int lidx(const DPatch& P, int i, int j, int k) { return i + P.ext[0] * (j + P.ext[1] * k); }

template <int DIM> __device__ __forceinline__ int stride_of(const DPatch& P, int d) {
  return d == 0 ? 1 : (d == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
}

// ------------------------------------------------------------------ advance stages
template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_prim(LevelArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w + 2, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const long long fs = P.fs;
  const T* U = (const T*)a.cur + P.off;
  double u[5], bc[3], w[8];
#pragma unroll
  for (int f = 0; f < 5; ++f) u[f] = (double)U[f * fs + L];
  bc[0] = 0.5 * ((double)U[5 * fs + L] + (double)U[5 * fs + L + 1]);
  bc[1] = 0.5 * ((double)U[6 * fs + L] + (double)U[6 * fs + L + P.ext[0]]);
  if (DIM == 3) bc[2] = 0.5 * ((double)U[7 * fs + L] + (double)U[7 * fs + L + P.ext[0] * P.ext[1]]);
  else bc[2] = (double)U[7 * fs + L];
  floor_density(u, a.fl.rho, a.fl.events);
  recover(u, bc, a.gamma - 1.0, w);
  floor_pressure(w, a.fl.p, a.fl.events);
  T* W = (T*)a.scr + P.soff + SC_W * fs;
#pragma unroll
  for (int f = 0; f < 8; ++f) W[f * fs + L] = (T)w[f];
}

template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_predict(LevelArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w + 1, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const long long fs = P.fs;
  const T* U = (const T*)a.cur + P.off;
  T* S = (T*)a.scr + P.soff;
  const T* W = S + SC_W * fs;
  const double dt = *a.dtp * a.dtscale;
  T w[8], s[3][8];
#pragma unroll
  for (int f = 0; f < 8; ++f) w[f] = W[f * fs + L];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = stride_of<DIM>(P, d);
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f == BX + d) s[d][f] = U[(BX + d) * fs + L + sd] - U[(BX + d) * fs + L];
      else s[d][f] = mm(w[f] - W[f * fs + L - sd], W[f * fs + L + sd] - w[f]);
      S[(SC_S + 8 * d + f) * fs + L] = s[d][f];
    }
  }
  const T ir = T(1) / w[0];
  const T gamma = (T)a.gamma;
  T wh[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) wh[f] = w[f];
  {
    T dw[8];
    const T h0 = (T)(0.5 * dt * a.idx[0]);
    prim_terms<T, 0>(w, s[0], gamma, ir, dw);
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h0 * dw[f];
    const T h1 = (T)(0.5 * dt * a.idx[1]);
    prim_terms<T, 1>(w, s[1], gamma, ir, dw);
#pragma unroll
    for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h1 * dw[f];
    if (DIM == 3) {
      const T h2 = (T)(0.5 * dt * a.idx[2]);
      prim_terms<T, 2>(w, s[2], gamma, ir, dw);
#pragma unroll
      for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h2 * dw[f];
    }
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) S[(SC_WH + f) * fs + L] = wh[f];
  S[(SC_REF + 0) * fs + L] = wh[3] * wh[6] - wh[2] * wh[7];
  S[(SC_REF + 1) * fs + L] = wh[1] * wh[7] - wh[3] * wh[5];
  S[(SC_REF + 2) * fs + L] = wh[2] * wh[5] - wh[1] * wh[6];
}

// d-faces with normal index in [4-w, n+4+w] and transverse cells in
// [4-w-1, n+4+w+1); face stored at the cell on its high side.
template <class T, int DIM, int D> __global__ void __launch_bounds__(TPB) k_flux(LevelArgs a) {
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
  T* S = (T*)a.scr + P.soff;
  T wl[8], wr[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    wl[f] = S[(SC_WH + f) * fs + Ll] + T(0.5) * S[(SC_S + 8 * D + f) * fs + Ll];
    wr[f] = S[(SC_WH + f) * fs + L] - T(0.5) * S[(SC_S + 8 * D + f) * fs + L];
  }
  constexpr int n = D, tt = (D + 1) % 3, uu = (D + 2) % 3;
  const T bn = T(0.5) * (wl[5 + n] + wr[5 + n]);
  const T ql[7] = {wl[0], wl[1 + n], wl[1 + tt], wl[1 + uu], wl[4], wl[5 + tt], wl[5 + uu]};
  const T qr[7] = {wr[0], wr[1 + n], wr[1 + tt], wr[1 + uu], wr[4], wr[5 + tt], wr[5 + uu]};
  T fr[7];
  hlld_flux<T>(ql, qr, bn, (T)a.gamma, fr);
  T* F = S + (SC_F + 8 * D) * fs;
  F[RHO * fs + L] = fr[0];
  F[(MX + n) * fs + L] = fr[1];
  F[(MX + tt) * fs + L] = fr[2];
  F[(MX + uu) * fs + L] = fr[3];
  F[EN * fs + L] = fr[4];
  F[(BX + tt) * fs + L] = fr[5];
  F[(BX + uu) * fs + L] = fr[6];
  F[(BX + n) * fs + L] = T(0);
}

// c-edges: c-coordinate cells in [4-w, n+4+w), a,b in [4-w, n+4+w]
template <class T, int DIM, int C> __global__ void __launch_bounds__(TPB) k_emf(LevelArgs a) {
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
  const int sa = stride_of<DIM>(P, A), sb = stride_of<DIM>(P, B);
  const long long fs = P.fs;
  T* S = (T*)a.scr + P.soff;
  const T* Fa = S + (SC_F + 8 * A) * fs;
  const T* Fb = S + (SC_F + 8 * B) * fs;
  const T* R = S + (SC_REF + C) * fs;
  const int q11 = L, q01 = L - sa, q10 = L - sb, q00 = L - sa - sb;
  const T ea_hi = -Fa[(BX + B) * fs + q11], ea_lo = -Fa[(BX + B) * fs + q10];
  const T eb_hi = Fb[(BX + A) * fs + q11], eb_lo = Fb[(BX + A) * fs + q01];
  S[(SC_E + C) * fs + L] = gs_emf<T>(ea_lo, ea_hi, eb_lo, eb_hi, R[q00], R[q10], R[q01], R[q11], Fa[q10], Fa[q11],
                                     Fb[q01], Fb[q11]);
}

template <class T, int DIM>
__device__ __forceinline__ T face_update(const T* S, long long fs, const DPatch& P, int d, int L, T v, const T* dtd) {
  const T* E0 = S + (SC_E + 0) * fs;
  const T* E1 = S + (SC_E + 1) * fs;
  const T* E2 = S + (SC_E + 2) * fs;
  const int sx = 1, sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  if (DIM == 2) {
    if (d == 0) v = v - dtd[1] * (E2[L + sy] - E2[L]);
    else v = v + dtd[0] * (E2[L + sx] - E2[L]);
  } else {
    if (d == 0) {
      v = v - dtd[1] * (E2[L + sy] - E2[L]);
      v = v + dtd[2] * (E1[L + sz] - E1[L]);
    } else if (d == 1) {
      v = v - dtd[2] * (E0[L + sz] - E0[L]);
      v = v + dtd[0] * (E2[L + sx] - E2[L]);
    } else {
      v = v - dtd[0] * (E1[L + sx] - E1[L]);
      v = v + dtd[1] * (E0[L + sy] - E0[L]);
    }
  }
  return v;
}

template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_update(LevelArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, a.w, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const long long fs = P.fs;
  const T* U = (const T*)a.cur + P.off;
  T* V = (T*)a.nxt + P.off;
  const T* S = (const T*)a.scr + P.soff;
  const double dt = *a.dtp * a.dtscale;
  T dtd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dtd[d] = (T)(dt * a.idx[d]);
  constexpr int NCF = DIM == 3 ? 5 : 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    T v = U[f * fs + L];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T* F = S + (SC_F + 8 * d + f) * fs;
      v = v - dtd[d] * (F[L + stride_of<DIM>(P, d)] - F[L]);
    }
    V[f * fs + L] = v;
  }
  const int hi[3] = {P.n[0] + 4 + a.w - 1, P.n[1] + 4 + a.w - 1, DIM == 3 ? P.n[2] + 4 + a.w - 1 : 0};
  const int cc[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    V[(BX + d) * fs + L] = face_update<T, DIM>(S, fs, P, d, L, U[(BX + d) * fs + L], dtd);
    if (cc[d] == hi[d]) {
      const int L2 = L + stride_of<DIM>(P, d);
      V[(BX + d) * fs + L2] = face_update<T, DIM>(S, fs, P, d, L2, U[(BX + d) * fs + L2], dtd);
    }
  }
}

// ------------------------------------------------------------------ registers
// coarse side: rows (l, qc, d, Lface, side, pf, Lfine) -> creg = dt F_c
template <class T, int DIM> __global__ void k_reg_coarse_faces(RowArgs a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[1]];
  const int d = row[2], L = row[3];
  const double dt = *a.dtp * a.dtscale;
  const T* F = (const T*)a.scr + P.soff + (SC_F + 8 * d) * P.fs;
  constexpr int NCF = DIM == 3 ? 5 : 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    a.creg[r * 6 + n] = dt * (double)F[f * P.fs + L];
  }
}

template <class T, int DIM> __global__ void k_reg_coarse_edges(RowArgs a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[1]];
  const int c = row[2], L = row[3];
  const double dt = *a.dtp * a.dtscale;
  const T* E = (const T*)a.scr + P.soff + (SC_E + c) * P.fs;
  a.ecreg[r] = dt * (double)E[L];
}

// fine side, one sub-step: freg[s] = dt 2^-(dim-1) * tree sum of the sub-faces
template <class T, int DIM> __global__ void k_reg_fine_faces(RowArgs a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[5]];
  const int d = row[2], L = row[6];
  const double dt = *a.dtp * a.dtscale;
  const double af = dt * (DIM == 3 ? 0.25 : 0.5);
  const T* F = (const T*)a.scr + P.soff + (SC_F + 8 * d) * P.fs;
  const int sx = 1, sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  int o[4];
  if (DIM == 2) {
    o[0] = 0; o[1] = d == 0 ? sy : sx;
  } else if (d == 0) {
    o[0] = 0; o[1] = sy; o[2] = sz; o[3] = sy + sz;
  } else if (d == 1) {
    o[0] = 0; o[1] = sx; o[2] = sz; o[3] = sx + sz;
  } else {
    o[0] = 0; o[1] = sx; o[2] = sy; o[3] = sx + sy;
  }
  constexpr int NCF = DIM == 3 ? 5 : 6;
  double* out = a.freg + (r * 2 + (a.substep - 1)) * 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    const T* G = F + f * P.fs + L;
    double s;
    if (DIM == 2) s = tree2((double)G[o[0]], (double)G[o[1]]);
    else s = tree4((double)G[o[0]], (double)G[o[1]], (double)G[o[2]], (double)G[o[3]]);
    out[n] = af * s;
  }
}

template <class T, int DIM> __global__ void k_reg_fine_edges(RowArgs a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[4]];
  const int c = row[2], L = row[5];
  const double dt = *a.dtp * a.dtscale;
  const T* E = (const T*)a.scr + P.soff + (SC_E + c) * P.fs;
  double v;
  if (DIM == 3) {
    const int sc = c == 0 ? 1 : (c == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
    v = (dt * 0.5) * tree2((double)E[L], (double)E[L + sc]);
  } else {
    v = dt * (double)E[L];
  }
  a.efreg[r * 2 + (a.substep - 1)] = v;
}

// ------------------------------------------------------------------ ghost fill
// Same-level copies as boxes, cells and faces in one list. A box record
// (FILL_BOX_W ints) holds everything a copy needs, so no patch record is read:
// the destination and source element offsets of its first position (64-bit;
// field 0 of a cell box, the face field of a face box), the x and y extents of
// both patches, both field strides, the box extents nx and ny, the number of
// fields nv (5 cells in 3D, 6 in 2D with B_z, 1 for faces), cx = min(nx, 64)
// and the multipliers ceil(2^31 / cx), ceil(2^31 / ny). A box is a list of
// rows q = y + ny z along x; a chunk (int4: box, x0, q0, nrows) is nrows whole
// rows of cx positions from (x0, q0), at most FILL_CHUNK positions, so a
// position's coordinates follow from its lane by two multiply-high divisions:
// floor(a / n) = hi32(2a ceil(2^31 / n)), exact while a n < 2^31.
constexpr int FILL_TPB = FILL_CHUNK;
struct FillPos {
  long long d, s;
  int dfs, sfs, nv;
};
// position t of chunk record cr, box record br (4 int4)
__device__ __forceinline__ bool fill_pos(const int4 cr, const int4* br, int t, FillPos& o) {
  const int4 b2 = br[2], b3 = br[3];  // (dfs, sfs, nx, ny), (nv, cx, mcx, mny)
  const unsigned r = __umulhi(2u * (unsigned)t, (unsigned)b3.z);
  const int x = cr.y + t - (int)r * b3.y;
  if ((int)r >= cr.w || x >= b2.z) return false;
  const unsigned q = (unsigned)cr.z + r;
  const unsigned z = __umulhi(2u * q, (unsigned)b3.w);
  const int y = (int)(q - z * (unsigned)b2.w);
  const int4 b0 = br[0], b1 = br[1];  // offsets; (dext0, dext1, sext0, sext1)
  const long long db = ((long long)(unsigned)b0.x) | ((long long)b0.y << 32);
  const long long sb = ((long long)(unsigned)b0.z) | ((long long)b0.w << 32);
  o.d = db + (x + b1.x * (y + b1.y * (int)z));
  o.s = sb + (x + b1.z * (y + b1.w * (int)z));
  o.dfs = b2.x;
  o.sfs = b2.y;
  o.nv = b3.x;
  return true;
}

// Each block copies a contiguous range of the chunk list, FILL_CHUNK threads
// per chunk, in tiles of FILL_TILE chunks whose chunk and box records are
// first staged in shared memory (a range of chunks spans at most as many
// boxes, the list being ordered by box), so that the only global loads of the
// copy loop are the copied values themselves. Each thread loads U chunks'
// positions (NV fields each) before it stores, so that the face boxes (one
// field) keep as many loads in flight as the cell boxes.
constexpr int FILL_RUN_TPB = 256, FILL_TILE = 256;
constexpr size_t FILL_SMEM = (size_t)FILL_TILE * 5 * sizeof(int4);
template <class T, int NV, int U>
__device__ __forceinline__ void fill_range(T* B, const int* boxes, const int4* ch, long long c0, long long c1,
                                           int4* sch, int4* sbox) {
  constexpr int G = FILL_RUN_TPB / FILL_CHUNK;
  const int t = threadIdx.x % FILL_CHUNK, g = threadIdx.x / FILL_CHUNK;
  for (long long t0 = c0; t0 < c1; t0 += FILL_TILE) {
    const int nt = (int)(c1 - t0 < FILL_TILE ? c1 - t0 : FILL_TILE);
    const int box0 = ch[t0].x, nbox = ch[t0 + nt - 1].x - box0 + 1;
    __syncthreads();  // the previous tile's records are no longer read
    for (int i = threadIdx.x; i < nt; i += FILL_RUN_TPB) sch[i] = ch[t0 + i];
    const int4* gb = reinterpret_cast<const int4*>(boxes) + 4LL * box0;
    for (int i = threadIdx.x; i < 4 * nbox; i += FILL_RUN_TPB) sbox[i] = gb[i];
    __syncthreads();
    for (int c = g; c < nt; c += U * G) {
      FillPos p[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int cc = c + u * G;
        ok[u] = false;
        if (cc < nt) {
          const int4 cr = sch[cc];
          ok[u] = fill_pos(cr, sbox + 4 * (cr.x - box0), t, p[u]);
        }
      }
      T v[U][NV];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int n = 0; n < NV; ++n)
          if (ok[u]) v[u][n] = B[p[u].s + (NV == 1 ? 0 : (n < 5 ? n : BZ)) * p[u].sfs];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int n = 0; n < NV; ++n)
          if (ok[u]) B[p[u].d + (NV == 1 ? 0 : (n < 5 ? n : BZ)) * p[u].dfs] = v[u][n];
    }
  }
}
// the cell boxes' chunks come first in the list (nsplit of them), then the
// face boxes'; the first split_blocks blocks share the cells' chunks in equal
// contiguous ranges, the rest the faces'
template <class T, int DIM> __global__ void __launch_bounds__(FILL_RUN_TPB) k_fill_runs(RowArgs a) {
  extern __shared__ int4 fill_smem[];
  int4* sch = fill_smem;
  int4* sbox = fill_smem + FILL_TILE;
  T* B = (T*)a.fbuf;
  const int4* ch = reinterpret_cast<const int4*>(a.chunks);
  const bool cells = (int)blockIdx.x < a.split_blocks;
  const long long lo = cells ? 0 : a.nsplit, n = cells ? a.nsplit : a.nrows - a.nsplit;
  const long long nb = cells ? a.split_blocks : (long long)gridDim.x - a.split_blocks;
  const long long b = cells ? blockIdx.x : blockIdx.x - a.split_blocks;
  const long long c0 = lo + n * b / nb, c1 = lo + n * (b + 1) / nb;
  if (c0 >= c1) return;
  if (cells) fill_range<T, DIM == 3 ? 5 : 6, 2>(B, a.rows, ch, c0, c1, sch, sbox);
  else fill_range<T, 1, 4>(B, a.rows, ch, c0, c1, sch, sbox);
}

// Prolongation and physical-boundary fills as ghost boxes of GHOST_BOX_W
// ints (dst, d, kind, src, lo[3], n[3], aux[3]), lo in dst's local ghosted
// coordinates; chunks as for the same-level boxes. gbox_pos gives the local
// coordinates x of this thread's position and its global position g (chunk
// bid: the block's index among the list's blocks).
constexpr int GBW = amrmhd::GHOST_BOX_W;
template <int DIM>
__device__ __forceinline__ bool gbox_pos(const RowArgs& a, unsigned bid, const int*& box, int* x, int* g) {
  const int bi = a.chunks[2 * bid];
  const int c = a.chunks[2 * bid + 1] + threadIdx.x;
  box = a.rows + GBW * bi;
  const int nx = box[7], ny = box[8], nz = box[9];
  if (c >= nx * ny * nz) return false;
  x[0] = box[4] + c % nx;
  x[1] = box[5] + (c / nx) % ny;
  x[2] = box[6] + c / (nx * ny);
  const DPatch& D = a.P[box[0]];
  g[0] = D.lo[0] + x[0] - 4;
  g[1] = D.lo[1] + x[1] - 4;
  g[2] = DIM == 3 ? D.lo[2] + x[2] - 4 : 0;
  return true;
}
__device__ __forceinline__ int local_of(const DPatch& P, const int* g) {
  return (g[0] - P.lo[0] + 4) + P.ext[0] * ((g[1] - P.lo[1] + 4) + P.ext[1] * (P.ext[2] > 1 ? g[2] - P.lo[2] + 4 : 0));
}

// physical boundary cells: kind 2 copies the patch's own position clamped into
// the domain (the coordinates aux[e] >= 0 replaced), kind 3 sets the inflow state
template <class T, int DIM> __global__ void __launch_bounds__(FILL_TPB) k_fill_bc_cells(RowArgs a) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, blockIdx.x, box, x, g)) return;
  const DPatch D = a.P[box[0]];
  T* dst = (T*)a.fbuf + D.off + x[0] + (long long)D.ext[0] * (x[1] + (long long)D.ext[1] * x[2]);
  constexpr int NCF = DIM == 3 ? 5 : 6;
  if (box[2] == 3) {
#pragma unroll
    for (int n = 0; n < NCF; ++n) {
      const int f = n < 5 ? n : BZ;
      dst[f * D.fs] = (T)a.inflow[f];
    }
  } else {
    int gc[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) gc[e] = box[10 + e] >= 0 ? box[10 + e] : g[e];
    const T* src = (const T*)a.fbuf + D.off + local_of(D, gc);
#pragma unroll
    for (int n = 0; n < NCF; ++n) {
      const int f = n < 5 ? n : BZ;
      dst[f * D.fs] = src[f * D.fs];
    }
  }
}

// physical boundary faces (the box's d-faces)
template <class T, int DIM> __global__ void __launch_bounds__(FILL_TPB) k_fill_bc_faces(RowArgs a) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, blockIdx.x, box, x, g)) return;
  const DPatch D = a.P[box[0]];
  const int f = BX + box[1];
  T* B = (T*)a.fbuf + D.off + f * D.fs;
  const int Ld = x[0] + D.ext[0] * (x[1] + D.ext[1] * x[2]);
  if (box[2] == 3) {
    B[Ld] = (T)a.inflow[f];
  } else {
    int gc[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) gc[e] = box[10 + e] >= 0 ? box[10 + e] : g[e];
    B[Ld] = B[local_of(D, gc)];
  }
}

// the coarse patch's local index of the parent of fine position g: the box's
// aux is the periodic wrap of g, so (g + aux) >> 1 is the parent cell (for a
// d-face, the coarse face coincident with or below the fine one)
template <int DIM> __device__ __forceinline__ int parent_local(const DPatch& C, const int* g, const int* aux) {
  int c[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) c[e] = e < DIM ? (g[e] + aux[e]) >> 1 : 0;
  return local_of(C, c);
}

// prolonged ghost cells (Sec. 2 prolongation): minmod-limited linear
// reconstruction of the parent cell at the child's centre; coarse data from
// cbuf (the parent level's state at the start of its current sub-step)
template <class T, int DIM> __device__ __forceinline__ void prolong_cells_at(const RowArgs& a, unsigned bid) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, bid, box, x, g)) return;
  const DPatch D = a.P[box[0]], C = a.P[box[3]];
  T* dst = (T*)a.fbuf + D.off + x[0] + (long long)D.ext[0] * (x[1] + (long long)D.ext[1] * x[2]);
  const T* src = (const T*)a.cbuf + C.off + parent_local<DIM>(C, g, box + 10);
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
  constexpr int NCF = DIM == 3 ? 5 : 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    const T* u = src + f * C.fs;
    const T u0 = u[0];
    T v = u0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T sl = mm(u0 - u[-st[d]], u[st[d]] - u0);
      v = v + sl * ((g[d] & 1) ? T(0.25) : T(-0.25));
    }
    dst[f * D.fs] = v;
  }
}

// B_n on the coarse n-face at b (pointer to that face), prolonged to the fine
// sub-face with transverse parities par
template <class T, int DIM>
__device__ __forceinline__ T coincident(const T* b, const int* st, int n, const int* par) {
  const T b0 = b[0];
  T v = b0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (d == n) continue;
    const T sl = mm(b0 - b[-st[d]], b[st[d]] - b0);
    v = v + sl * (par[d] ? T(0.25) : T(-0.25));
  }
  return v;
}

// prolonged ghost faces (the box's n-faces): divergence-free (Balsara) from the
// coarse faces
template <class T, int DIM> __device__ __forceinline__ void prolong_faces_at(const RowArgs& a, unsigned bid) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, bid, box, x, g)) return;
  const DPatch D = a.P[box[0]], C = a.P[box[3]];
  const int n = box[1];
  const int Lc = parent_local<DIM>(C, g, box + 10);
  const int par[3] = {g[0] & 1, g[1] & 1, DIM == 3 ? (g[2] & 1) : 0};
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
  const T* cb = (const T*)a.cbuf + C.off;
  const T* bn = cb + (BX + n) * C.fs + Lc;
  T v;
  if (!par[n]) {
    v = coincident<T, DIM>(bn, st, n, par);
  } else {
    const T lo_v = coincident<T, DIM>(bn, st, n, par);
    const T hi_v = coincident<T, DIM>(bn + st[n], st, n, par);
    T corr = T(0);
    bool first = true;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == n) continue;
      const T* bt_lo = cb + (BX + t) * C.fs + Lc;
      const T* bt_hi = bt_lo + st[t];
      const T s_hi = mm(bt_hi[0] - bt_hi[-st[n]], bt_hi[st[n]] - bt_hi[0]);
      const T s_lo = mm(bt_lo[0] - bt_lo[-st[n]], bt_lo[st[n]] - bt_lo[0]);
      const T term = (T)a.ratio[n][t] * (s_hi - s_lo);
      corr = first ? (T(0) + term) : (corr + term);
      first = false;
    }
    v = T(0.5) * (lo_v + hi_v) + T(0.125) * corr;
  }
  ((T*)a.fbuf)[D.off + (BX + n) * D.fs + x[0] + D.ext[0] * (x[1] + D.ext[1] * x[2])] = v;
}

// the prolonged ghost cells and faces of a level in one launch: blocks [0,
// c.nrows) take the cell chunks, the rest the face chunks (the two write
// disjoint positions from disjoint coarse data)
template <class T, int DIM> __global__ void __launch_bounds__(FILL_TPB) k_prolong(RowArgs c, RowArgs f) {
  if (blockIdx.x < (unsigned)c.nrows) prolong_cells_at<T, DIM>(c, blockIdx.x);
  else prolong_faces_at<T, DIM>(f, blockIdx.x - (unsigned)c.nrows);
}

// ------------------------------------------------------------------ regrid
// flagged cells of a level: max_d |rho(i+1) - rho(i-1)| / (2 rho) > theta in
// FP64 from the stored values; global indices appended (order is arbitrary)
template <class T, int DIM>
__global__ void __launch_bounds__(TPB) k_flag(LevelArgs a, double theta, int* out, unsigned long long* count,
                                              long long cap) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, 0, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const T* R = (const T*)a.cur + P.off;
  const double r = (double)R[L];
  double m = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = stride_of<DIM>(P, d);
    const double g = fabs((double)R[L + sd] - (double)R[L - sd]) / (2.0 * r);
    if (g > m) m = g;
  }
  if (!(m > theta)) return;
  const unsigned long long n = atomicAdd(count, 1ULL);
  if ((long long)n >= cap) return;
  out[3 * n] = P.lo[0] + i - 4;
  out[3 * n + 1] = P.lo[1] + j - 4;
  out[3 * n + 2] = DIM == 3 ? P.lo[2] + k - 4 : 0;
}

// the same test per cell into dense bytes: region 1 on every cell of the
// level, flags 1 where the gradient exceeds theta
template <class T, int DIM>
__global__ void __launch_bounds__(TPB) k_flag_dense(LevelArgs a, double theta, unsigned char* region,
                                                    unsigned char* flags, DenseBox box) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  if (!region_cell<DIM>(P, 0, blockIdx.x * TPB + threadIdx.x, i, j, k)) return;
  const int L = lidx(P, i, j, k);
  const T* R = (const T*)a.cur + P.off;
  const double r = (double)R[L];
  double m = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = stride_of<DIM>(P, d);
    const double g = fabs((double)R[L + sd] - (double)R[L - sd]) / (2.0 * r);
    if (g > m) m = g;
  }
  const int x = P.lo[0] + i - 4 - box.off[0], y = P.lo[1] + j - 4 - box.off[1],
            z = DIM == 3 ? P.lo[2] + k - 4 - box.off[2] : 0;
  const long long idx = ((long long)z * box.n[1] + y) * box.n[0] + x;
  region[idx] = 1;
  flags[idx] = m > theta ? 1 : 0;
}

// new fine cells, as transfer boxes (GHOST_BOX_W ints, chunks as for the ghost
// boxes): kind 0 copies the old fine patch src of the old hierarchy (P2, obuf)
// at local offset aux, kind 1 prolongs from the coarse patch src (cbuf) as for
// a ghost cell (the cells lie inside the domain: no periodic wrap)
template <class T, int DIM> __global__ void __launch_bounds__(FILL_TPB) k_transfer_cells(RowArgs a) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, blockIdx.x, box, x, g)) return;
  const DPatch D = a.P[box[0]];
  T* dst = (T*)a.fbuf + D.off + x[0] + (long long)D.ext[0] * (x[1] + (long long)D.ext[1] * x[2]);
  constexpr int NCF = DIM == 3 ? 5 : 6;
  if (box[2] == 0) {
    const DPatch O = a.P2[box[3]];
    const T* src = (const T*)a.obuf + O.off + (x[0] + box[10]) +
                   (long long)O.ext[0] * ((x[1] + box[11]) + (long long)O.ext[1] * (x[2] + box[12]));
#pragma unroll
    for (int n = 0; n < NCF; ++n) {
      const int f = n < 5 ? n : BZ;
      dst[f * D.fs] = src[f * O.fs];
    }
    return;
  }
  const DPatch C = a.P[box[3]];
  const T* src = (const T*)a.cbuf + C.off + parent_local<DIM>(C, g, box + 10);
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    const T* u = src + f * C.fs;
    const T u0 = u[0];
    T v = u0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T sl = mm(u0 - u[-st[d]], u[st[d]] - u0);
      v = v + sl * ((g[d] & 1) ? T(0.25) : T(-0.25));
    }
    dst[f * D.fs] = v;
  }
}

// new fine own faces of the box's direction: kind 0 copies the old fine face,
// kind 1 prolongs (coincident or interior, by the parity) from the coarse face
// (g + aux) >> 1 of the parent patch (aux: the periodic wrap)
template <class T, int DIM> __global__ void __launch_bounds__(FILL_TPB) k_transfer_faces(RowArgs a) {
  const int* box;
  int x[3], g[3];
  if (!gbox_pos<DIM>(a, blockIdx.x, box, x, g)) return;
  const DPatch D = a.P[box[0]];
  const int n = box[1];
  T* out = (T*)a.fbuf + D.off + (BX + n) * D.fs + x[0] + (long long)D.ext[0] * (x[1] + (long long)D.ext[1] * x[2]);
  if (box[2] == 0) {
    const DPatch O = a.P2[box[3]];
    *out = ((const T*)a.obuf)[O.off + (BX + n) * O.fs + (x[0] + box[10]) +
                              (long long)O.ext[0] * ((x[1] + box[11]) + (long long)O.ext[1] * (x[2] + box[12]))];
    return;
  }
  const DPatch C = a.P[box[3]];
  const int Lc = parent_local<DIM>(C, g, box + 10);
  const int par[3] = {g[0] & 1, g[1] & 1, DIM == 3 ? (g[2] & 1) : 0};
  const int st[3] = {1, C.ext[0], C.ext[0] * C.ext[1]};
  const T* cb = (const T*)a.cbuf + C.off;
  const T* bn = cb + (BX + n) * C.fs + Lc;
  if (!par[n]) {
    *out = coincident<T, DIM>(bn, st, n, par);
    return;
  }
  const T lo_v = coincident<T, DIM>(bn, st, n, par);
  const T hi_v = coincident<T, DIM>(bn + st[n], st, n, par);
  T corr = T(0);
  bool first = true;
#pragma unroll
  for (int t = 0; t < DIM; ++t) {
    if (t == n) continue;
    const T* bt_lo = cb + (BX + t) * C.fs + Lc;
    const T* bt_hi = bt_lo + st[t];
    const T s_hi = mm(bt_hi[0] - bt_hi[-st[n]], bt_hi[st[n]] - bt_hi[0]);
    const T s_lo = mm(bt_lo[0] - bt_lo[-st[n]], bt_lo[st[n]] - bt_lo[0]);
    const T term = (T)a.ratio[n][t] * (s_hi - s_lo);
    corr = first ? (T(0) + term) : (corr + term);
    first = false;
  }
  *out = T(0.5) * (lo_v + hi_v) + T(0.125) * corr;
}

// divergence-free closure: rows (dst, L of the first child) of a prolonged
// coarse cell; the children's divergences r, delta = K r added to the interior
// faces (faces by direction, then transverse children in z,y,x bit order);
// idx = fine 1/dx
template <class T, int DIM> __global__ void k_closure(RowArgs a) {
  const long long r = (long long)blockIdx.x * TPB + threadIdx.x;
  if (r >= a.nrows) return;
  const int* row = a.rows + 2 * r;
  const DPatch D = a.P[row[0]];
  const int L0 = row[1];
  T* B = (T*)a.fbuf + D.off;
  const int st[3] = {1, D.ext[0], D.ext[0] * D.ext[1]};
  constexpr int NC = DIM == 3 ? 8 : 4, NT = DIM == 3 ? 4 : 2;
  double res[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int x = L0 + (c & 1) * st[0] + ((c >> 1) & 1) * st[1] + (DIM == 3 ? ((c >> 2) & 1) * st[2] : 0);
    double div = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T* b = B + (BX + d) * D.fs;
      div = div + ((double)b[x + st[d]] - (double)b[x]) * a.idx[d];
    }
    res[c] = div;
  }
  int f = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int t = 0; t < NT; ++t, ++f) {
      int o[3] = {0, 0, 0}, bit = 0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        if (e == d) continue;
        o[e] = (t >> bit) & 1;
        ++bit;
      }
      o[d] = 1;
      double delta = 0.0;
#pragma unroll
      for (int c = 0; c < NC; ++c) delta += a.K[f * 8 + c] * res[c];
      T* face = B + (BX + d) * D.fs + L0 + o[0] * st[0] + o[1] * st[1] + (DIM == 3 ? o[2] * st[2] : 0);
      *face = (T)((double)*face + delta);
    }
}

// ------------------------------------------------------------------ reflux and restriction
// rows (l, qc, Lcell, f0..f5); R = (S1 + S2) - C per C/F face, applied in slot order
template <class T, int DIM>
__device__ __forceinline__ void reflux_cells_row(const RowArgs& a, const int* rows, long long r) {
  const int* row = rows + 9 * r;
  const DPatch P = a.P[row[1]];
  T* U = (T*)a.cbuf + P.off + row[2];
  constexpr int NCF = DIM == 3 ? 5 : 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    double v = (double)U[f * P.fs];
    for (int slot = 0; slot < 2 * DIM; ++slot) {
      const int e = row[3 + slot];
      if (e < 0) continue;
      const double R = (a.freg[(2 * (long long)e) * 6 + n] + a.freg[(2 * (long long)e + 1) * 6 + n]) - a.creg[(long long)e * 6 + n];
      if (slot & 1) v = v - R * a.idx[slot >> 1];
      else v = v + R * a.idx[slot >> 1];
    }
    U[f * P.fs] = (T)v;
  }
}

// rows (l, qc, d, Lface, e0..e3): B += +e0/dx_t1 - e1/dx_t1 - e2/dx_t2 + e3/dx_t2
template <class T, int DIM>
__device__ __forceinline__ void reflux_faces_row(const RowArgs& a, const int* rows, long long r) {
  const int* row = rows + 8 * r;
  const DPatch P = a.P[row[1]];
  const int d = row[2];
  T* B = (T*)a.cbuf + P.off + (BX + d) * P.fs + row[3];
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double v = (double)B[0];
#pragma unroll
  for (int slot = 0; slot < 4; ++slot) {
    const int e = row[4 + slot];
    if (e < 0) continue;
    const double RE = (a.efreg[2 * (long long)e] + a.efreg[2 * (long long)e + 1]) - a.ecreg[e];
    const double coef = slot == 0 ? a.idx[t1] : slot == 1 ? -a.idx[t1] : slot == 2 ? -a.idx[t2] : a.idx[t2];
    v = v + coef * RE;
  }
  B[0] = (T)v;
}

// rows (l, qc, Lcell, pf, Lchild0)
template <class T, int DIM>
__device__ __forceinline__ void restrict_cells_row(const RowArgs& a, const int* rows, long long r) {
  const int* row = rows + 5 * r;
  const DPatch C = a.P[row[1]], F = a.P[row[3]];
  T* dst = (T*)a.cbuf + C.off + row[2];
  const T* src = (const T*)a.fbuf + F.off + row[4];
  const int sy = F.ext[0], sz = F.ext[0] * F.ext[1];
  constexpr int NCF = DIM == 3 ? 5 : 6;
#pragma unroll
  for (int n = 0; n < NCF; ++n) {
    const int f = n < 5 ? n : BZ;
    const T* c = src + f * F.fs;
    double s;
    if (DIM == 2) {
      s = tree4((double)c[0], (double)c[1], (double)c[sy], (double)c[sy + 1]) * 0.25;
    } else {
      const double v[8] = {(double)c[0], (double)c[1], (double)c[sy], (double)c[sy + 1],
                           (double)c[sz], (double)c[sz + 1], (double)c[sz + sy], (double)c[sz + sy + 1]};
      s = tree8(v) * 0.125;
    }
    dst[f * C.fs] = (T)s;
  }
}

// rows (l, qc, d, Lface, pf, Lfine0)
template <class T, int DIM>
__device__ __forceinline__ void restrict_faces_row(const RowArgs& a, const int* rows, long long r) {
  const int* row = rows + 6 * r;
  const DPatch C = a.P[row[1]], F = a.P[row[4]];
  const int d = row[2];
  const T* c = (const T*)a.fbuf + F.off + (BX + d) * F.fs + row[5];
  const int sx = 1, sy = F.ext[0], sz = F.ext[0] * F.ext[1];
  double s;
  if (DIM == 2) {
    s = tree2((double)c[0], (double)c[d == 0 ? sy : sx]) * 0.5;
  } else {
    int o1, o2;
    if (d == 0) { o1 = sy; o2 = sz; }
    else if (d == 1) { o1 = sx; o2 = sz; }
    else { o1 = sx; o2 = sy; }
    s = tree4((double)c[0], (double)c[o1], (double)c[o2], (double)c[o1 + o2]) * 0.25;
  }
  ((T*)a.cbuf)[C.off + (BX + d) * C.fs + row[3]] = (T)s;
}

// the reflux and restriction of a fine level into its parent in one launch:
// block ranges L.b[k] .. L.b[k+1] of TPB rows take list k (reflux cells,
// reflux faces, restriction cells, restriction faces). The four write disjoint
// coarse positions (reflux only uncovered cells and faces that touch no
// covered cell, restriction the covered cells and the faces of the fine
// region's closure) and none reads what another writes.
template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_reflux_restrict(RowArgs a, RRLists L) {
  const unsigned b = blockIdx.x;
  const int k = b < L.b[1] ? 0 : (b < L.b[2] ? 1 : (b < L.b[3] ? 2 : 3));
  const long long r = (long long)(b - L.b[k]) * TPB + threadIdx.x;
  if (r >= L.n[k]) return;
  if (k == 0) reflux_cells_row<T, DIM>(a, L.rows[0], r);
  else if (k == 1) reflux_faces_row<T, DIM>(a, L.rows[1], r);
  else if (k == 2) restrict_cells_row<T, DIM>(a, L.rows[2], r);
  else restrict_faces_row<T, DIM>(a, L.rows[3], r);
}

// ------------------------------------------------------------------ CFL
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T x = __shfl_xor_sync(0xffffffffu, v, o);
    v = x > v ? x : v;
  }
  return v;
}

// per-cell rate sum_d (|v_d| + c_f,d)/dx_d; FP64 path: all FP64 (bitwise with a
// plain FP64 evaluation); mixed path: the FP64-balanced recovery of
// recover_t and FP32 fast speeds, the maximum taken in FP32 (exact) and
// carried in FP64 across blocks
// cells per thread of the CFL reduction: one atomic per block of TPB x CFL_CPT
// cells (a single address takes every block's atomic)
constexpr int CFL_CPT = 4;

template <class T, int DIM> __global__ void __launch_bounds__(TPB) k_cfl(CflArgs a) {
  const DPatch P = a.P[a.ids[blockIdx.y]];
  int i, j, k;
  T tmax = T(0);  // per-thread maximum in the working type; the reduction is FP64
  bool bad = false;
  // loop invariants in the working type (conversions and comparisons of FP64
  // values issue on the FP64 pipe): gamma, 1/dx, gamma - 1 and the floors
  const T g = (T)a.gamma;
  const T ix[3] = {(T)a.idx[0], (T)a.idx[1], (T)a.idx[2]};
  const double gm1 = a.gamma - 1.0;
  const bool floors = a.fl.rho > 0.0 || a.fl.p > 0.0;
  for (int tc = blockIdx.x * TPB + threadIdx.x;; tc += gridDim.x * TPB) {
    if (!region_cell<DIM>(P, 0, tc, i, j, k)) break;
    const int L = lidx(P, i, j, k);
    const long long fs = P.fs;
    const T* U = (const T*)a.cur + P.off;
    T u[5], bl[3], br[3], w[8];
#pragma unroll
    for (int f = 0; f < 5; ++f) u[f] = U[f * fs + L];
    bl[0] = U[5 * fs + L]; br[0] = U[5 * fs + L + 1];
    bl[1] = U[6 * fs + L]; br[1] = U[6 * fs + L + P.ext[0]];
    if (DIM == 3) { bl[2] = U[7 * fs + L]; br[2] = U[7 * fs + L + P.ext[0] * P.ext[1]]; }
    else { bl[2] = U[7 * fs + L]; br[2] = U[7 * fs + L]; }
    if (floors) floor_density(u, a.fl.rho, a.fl.events);
    recover_t(u, bl, br, gm1, w);
    if (floors) floor_pressure(w, a.fl.p, a.fl.events);
    if (!(w[0] > T(0)) || !(w[4] > T(0))) bad = true;
    else {
      T rr = T(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int t = (d + 1) % 3, uu = (d + 2) % 3;
        const T cf = cfast<T>(w[0], w[4], w[5 + d], w[5 + t], w[5 + uu], g);
        rr = rr + (dabs(w[1 + d]) + cf) * ix[d];
      }
      if (!(rr < (T)INFINITY)) bad = true;  // NaN or infinite
      else if (rr > tmax) tmax = rr;
    }
  }
  if (bad) atomicOr(a.err, 1u);
  // the maximum is exact in the working type; it is widened once per block
  const T rate = warp_max(tmax);
  __shared__ T red[TPB / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
  __syncthreads();
  if (threadIdx.x < 32) {
    T v = threadIdx.x < TPB / 32 ? red[threadIdx.x] : T(0);
    v = warp_max(v);
    if (threadIdx.x == 0) atomicMax(a.slot, (unsigned long long)__double_as_longlong((double)v));
  }
}

// ------------------------------------------------------------------ packed I/O
template <class T, int DIM>
__global__ void __launch_bounds__(TPB) k_io(const DPatch* PP, const int* ids, void* state, double* packed,
                                            const long long* poff, int field, int to_state) {
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
  T* s = (T*)state + P.off + field * P.fs + L;
  double* q = packed + poff[pid] + t;
  if (to_state) *s = (T)*q;
  else *q = (double)*s;
}

// all 8 fields of one level in one launch (blockIdx.z = field); packed + foff[f]
// is field f's packed array, poff[kind * npatch_total + pid] the patch's offset in it
struct IoAll {
  long long foff[8];
};
// Each warp takes 32 x IO_EPT consecutive packed elements of one (patch,
// field), lane l the elements l, l+32, ...: the packed side is read or written
// in whole 128-byte lines, the positions in the patch follow by stepping x
// (and wrapping into y and z) instead of dividing per element, and a thread's
// IO_EPT loads are issued before its stores (device memory, or page-locked
// host memory over the host link).
constexpr int IO_EPT = 8;
template <class T, int DIM, class Q>
__global__ void __launch_bounds__(TPB) k_io_all(const DPatch* PP, const int* ids, void* state, Q* packed,
                                                const long long* const* poff, IoAll io, int to_state) {
  const int pid = ids[blockIdx.y];
  const int field = blockIdx.z;
  const DPatch P = PP[pid];
  const int fd = (field >= BX && !(DIM == 2 && field == BZ)) ? field - BX : -1;
  int r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = e >= DIM ? 1 : P.n[e] + (e == fd ? 1 : 0);
  const int n = r[0] * r[1] * r[2];
  const int t0 = blockIdx.x * (TPB * IO_EPT) + (threadIdx.x >> 5) * (32 * IO_EPT) + (threadIdx.x & 31);
  if (t0 >= n) return;
  T* sb = (T*)state + P.off + field * P.fs;
  Q* qb = packed + io.foff[field] + poff[fd + 1][pid];
  int i = t0 % r[0], j = (t0 / r[0]) % r[1], k = t0 / (r[0] * r[1]);
  int ls[IO_EPT];
#pragma unroll
  for (int m = 0; m < IO_EPT; ++m) {
    // an element past the end reads element t0 again and is not stored
    ls[m] = t0 + 32 * m < n ? lidx(P, i + 4, j + 4, DIM == 3 ? k + 4 : 0) : ls[0];
    i += 32;
    while (i >= r[0]) {
      i -= r[0];
      if (++j == r[1]) { j = 0; ++k; }
    }
  }
  if (to_state) {
    Q v[IO_EPT];
#pragma unroll
    for (int m = 0; m < IO_EPT; ++m) v[m] = qb[t0 + 32 * m < n ? t0 + 32 * m : t0];
#pragma unroll
    for (int m = 0; m < IO_EPT; ++m)
      if (t0 + 32 * m < n) sb[ls[m]] = (T)v[m];
  } else {
    T v[IO_EPT];
#pragma unroll
    for (int m = 0; m < IO_EPT; ++m) v[m] = sb[ls[m]];
#pragma unroll
    for (int m = 0; m < IO_EPT; ++m)
      if (t0 + 32 * m < n) qb[t0 + 32 * m] = (Q)v[m];
  }
}

#include "kernels_fused.cuh"

// ------------------------------------------------------------------ launchers
template <class T, int DIM> struct Impl {
  static dim3 grid_region(const LevelArgs& a, int m, int extra) {
    long long n = 1;
    for (int d = 0; d < DIM; ++d) n *= a.maxn[d] + 2 * m + extra;
    return dim3(cdiv(n, TPB), a.npatch);
  }
  static void advance(const LevelArgs& a, cudaStream_t s, int* nl) {
    k_prim<T, DIM><<<grid_region(a, a.w + 2, 0), TPB, 0, s>>>(a);
    k_predict<T, DIM><<<grid_region(a, a.w + 1, 0), TPB, 0, s>>>(a);
    k_flux<T, DIM, 0><<<grid_region(a, a.w + 1, 0), TPB, 0, s>>>(a);
    k_flux<T, DIM, 1><<<grid_region(a, a.w + 1, 0), TPB, 0, s>>>(a);
    if (DIM == 3) k_flux<T, DIM, 2><<<grid_region(a, a.w + 1, 0), TPB, 0, s>>>(a);
    if (DIM == 3) {
      k_emf<T, DIM, 0><<<grid_region(a, a.w, 1), TPB, 0, s>>>(a);
      k_emf<T, DIM, 1><<<grid_region(a, a.w, 1), TPB, 0, s>>>(a);
    }
    k_emf<T, DIM, 2><<<grid_region(a, a.w, 1), TPB, 0, s>>>(a);
    k_update<T, DIM><<<grid_region(a, a.w, 0), TPB, 0, s>>>(a);
    if (nl) *nl += DIM == 3 ? 9 : 6;
  }
  static void reg_coarse(const RowArgs& f, const RowArgs& e, cudaStream_t s, int* nl) {
    if (f.nrows) { k_reg_coarse_faces<T, DIM><<<cdiv(f.nrows, TPB), TPB, 0, s>>>(f); if (nl) ++*nl; }
    if (e.nrows) { k_reg_coarse_edges<T, DIM><<<cdiv(e.nrows, TPB), TPB, 0, s>>>(e); if (nl) ++*nl; }
  }
  static void reg_fine(const RowArgs& f, const RowArgs& e, cudaStream_t s, int* nl) {
    if (f.nrows) { k_reg_fine_faces<T, DIM><<<cdiv(f.nrows, TPB), TPB, 0, s>>>(f); if (nl) ++*nl; }
    if (e.nrows) { k_reg_fine_edges<T, DIM><<<cdiv(e.nrows, TPB), TPB, 0, s>>>(e); if (nl) ++*nl; }
  }
#define AMRK_ROWS(NAME)                                                                 \
  static void NAME(const RowArgs& a, cudaStream_t s, int* nl) {                         \
    if (!a.nrows) return;                                                               \
    k_##NAME<T, DIM><<<cdiv(a.nrows, TPB), TPB, 0, s>>>(a);                             \
    if (nl) ++*nl;                                                                      \
  }
#define AMRK_BOXES(NAME)                                                                \
  static void NAME(const RowArgs& a, cudaStream_t s, int* nl) {                         \
    if (!a.nrows) return;                                                               \
    k_##NAME<T, DIM><<<(unsigned)a.nrows, FILL_TPB, 0, s>>>(a);                          \
    if (nl) ++*nl;                                                                      \
  }
  AMRK_BOXES(fill_bc_cells)
  AMRK_BOXES(fill_bc_faces)
#undef AMRK_BOXES
  static void fill_runs(const RowArgs& a, cudaStream_t s, int* nl) {
    if (!a.nrows) return;
    // one wave: the resident blocks of every SM
    static const long long resident = [] {
      int dev = 0, sms = 152, per = 4;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fill_runs<T, DIM>, FILL_RUN_TPB, FILL_SMEM);
      return (long long)sms * (per > 0 ? per : 1);
    }();
    // blocks shared between the cell and face chunks by their element counts,
    // at least 2 x FILL_CHUNK / 4 chunks per block
    const long long nc = a.nsplit, nf = a.nrows - a.nsplit;
    const double wc = (double)nc * (DIM == 3 ? 5 : 6), wf = (double)nf;
    const long long need_c = (nc + 31) / 32, need_f = (nf + 31) / 32;
    long long bc = std::min(need_c, (long long)(resident * wc / (wc + wf) + 0.5));
    long long bf = std::min(need_f, resident - bc);
    if (nc > 0 && bc < 1) bc = 1;
    if (nf > 0 && bf < 1) bf = 1;
    RowArgs b = a;
    b.split_blocks = (int)bc;
    k_fill_runs<T, DIM><<<(unsigned)(bc + bf), FILL_RUN_TPB, FILL_SMEM, s>>>(b);
    if (nl) ++*nl;
  }
#define AMRK_BOXES(NAME)                                                                \
  static void NAME(const RowArgs& a, cudaStream_t s, int* nl) {                         \
    if (!a.nrows) return;                                                               \
    k_##NAME<T, DIM><<<(unsigned)a.nrows, FILL_TPB, 0, s>>>(a);                          \
    if (nl) ++*nl;                                                                      \
  }
  AMRK_BOXES(transfer_cells)
  AMRK_BOXES(transfer_faces)
#undef AMRK_BOXES
  AMRK_ROWS(closure)
#undef AMRK_ROWS
  static void prolong(const RowArgs& c, const RowArgs& f, cudaStream_t s, int* nl) {
    if (!c.nrows && !f.nrows) return;
    k_prolong<T, DIM><<<(unsigned)(c.nrows + f.nrows), FILL_TPB, 0, s>>>(c, f);
    if (nl) ++*nl;
  }
  static void reflux_restrict(const RowArgs& a, const RRLists& lists, cudaStream_t s, int* nl) {
    RRLists L = lists;
    L.b[0] = 0;
    for (int k = 0; k < 4; ++k) L.b[k + 1] = L.b[k] + (unsigned)cdiv(L.n[k], TPB);
    if (!L.b[4]) return;
    k_reflux_restrict<T, DIM><<<L.b[4], TPB, 0, s>>>(a, L);
    if (nl) ++*nl;
  }
  static void cfl(const CflArgs& a, cudaStream_t s, int* nl) {
    long long n = 1;
    for (int d = 0; d < DIM; ++d) n *= a.maxn[d];
    k_cfl<T, DIM><<<dim3(cdiv(n, TPB * CFL_CPT), a.npatch), TPB, 0, s>>>(a);
    if (nl) ++*nl;
  }
  static void flag(const LevelArgs& a, double theta, int* out, unsigned long long* count, long long cap,
                   cudaStream_t s) {
    k_flag<T, DIM><<<grid_region(a, 0, 0), TPB, 0, s>>>(a, theta, out, count, cap);
  }
  static void flag_dense(const LevelArgs& a, double theta, unsigned char* region, unsigned char* flags, DenseBox box,
                         cudaStream_t s) {
    k_flag_dense<T, DIM><<<grid_region(a, 0, 0), TPB, 0, s>>>(a, theta, region, flags, box);
  }
  static void io(const DPatch* P, const int* ids, int npatch, const int* maxn, void* state, double* packed,
                 const long long* poff, int field, int to_state, cudaStream_t s, int* nl) {
    long long n = 1;
    for (int d = 0; d < DIM; ++d) n *= maxn[d] + 1;
    k_io<T, DIM><<<dim3(cdiv(n, TPB), npatch), TPB, 0, s>>>(P, ids, state, packed, poff, field, to_state);
    if (nl) ++*nl;
  }
  static void io_all(const DPatch* P, const int* ids, int npatch, const int* maxn, void* state, void* packed,
                     int packed_f32, const long long* const* poff, const long long* foff, int to_state, cudaStream_t s,
                     int* nl) {
    long long n = 1;  // elements of the largest (patch, field)
    for (int d = 0; d < DIM; ++d) n *= maxn[d] + 1;
    IoAll io;
    for (int f = 0; f < 8; ++f) io.foff[f] = foff[f];
    const dim3 g(cdiv(n, TPB * IO_EPT), npatch, 8);
    if (packed_f32) k_io_all<T, DIM, float><<<g, TPB, 0, s>>>(P, ids, state, (float*)packed, poff, io, to_state);
    else k_io_all<T, DIM, double><<<g, TPB, 0, s>>>(P, ids, state, (double*)packed, poff, io, to_state);
    if (nl) ++*nl;
  }
  // fused 3D advance (2D falls back to the staged kernels)
  template <int V> static size_t fused_smem() {
    return sizeof(FusedSmem<T, FusedCfg<V>::TX, FusedCfg<V>::TY>);
  }
  template <int V> static bool fused_fits() { return fused_smem<V>() <= 227 * 1024; }
  template <int V> static void prepare_v() {
    if (fused_fits<V>()) {
      cudaFuncSetAttribute(k_advance3d_fused<T, V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<V>());
      cudaFuncSetAttribute(k_advance3d_fused<T, V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<V>());
      cudaFuncSetAttribute(k_advance3d_fused<T, V, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<V>());
      cudaFuncSetAttribute(k_advance3d_fused<T, V, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<V>());
      cudaFuncSetAttribute(k_advance3d_fused<T, V, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<V>());
    }
  }
  static void prepare() {
    if (DIM == 3) { prepare_v<0>(); prepare_v<1>(); prepare_v<2>(); prepare_v<3>(); prepare_v<4>(); }
    if (DIM == 3) {
      if (fused_fits<2>())
        cudaFuncSetAttribute(k_advance_queue<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<2>());
      cudaFuncSetAttribute(k_advance_queue<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<3>());
    }
  }
  // the queue advance: a persistent grid of the resident CTAs
  template <int V> static void launch_queue(const QueueArgs& q, cudaStream_t s) {
    static const int resident = [] {
      int dev = 0, sms = 152, per = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_advance_queue<T, V>, FusedCfg<V>::NT, fused_smem<V>());
      return sms * (per > 0 ? per : 1);
    }();
    k_advance_queue<T, V><<<resident, FusedCfg<V>::NT, fused_smem<V>(), s>>>(q);
  }
  static void advance_queue(const QueueArgs& q, int variant, cudaStream_t s, int* nl) {
    if (DIM != 3 || q.ntasks <= 0) return;
    if (variant == 2 && fused_fits<2>()) launch_queue<2>(q, s);
    else launch_queue<3>(q, s);
    if (nl) ++*nl;
  }
  // resident CTAs of a fused instance on the whole GPU
  template <int V, int MODE, bool FL> static long long fused_slots() {
    static const long long slots = [] {
      int dev = 0, sms = 152, per = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_advance3d_fused<T, V, MODE, FL>, FusedCfg<V>::NT,
                                                    fused_smem<V>());
      return (long long)sms * (per > 0 ? per : 1);
    }();
    return slots;
  }
  template <int V> static void launch_fused(const LevelArgs& a0, cudaStream_t s) {
    constexpr int TX = FusedCfg<V>::TX, TY = FusedCfg<V>::TY;
    LevelArgs a = a0;
    const int ex = a.maxn[0] + 2 * a.w, ey = a.maxn[1] + 2 * a.w;
    const int ntx = (ex + TX - 1) / TX, nty = (ey + TY - 1) / TY;
    const bool fl = a.fl.rho > 0.0 || a.fl.p > 0.0;  // floors (the host never combines them with DH)
    dim3 g;
    a.tail = 0;
    if (a.zlen == -2) {
      // whole columns; those of the last partial wave halved when they fill
      // at most half of it (else whole columns throughout)
      a.zlen = 0;
      const long long cols = (long long)ntx * nty * a.npatch;
      const long long slots = fl ? (a.bnd ? fused_slots<V, 1, true>() : fused_slots<V, 0, true>())
                                 : (a.bnd ? fused_slots<V, 1, false>()
                                          : (a.nbr && a.w == 0 ? fused_slots<V, 2, false>() : fused_slots<V, 0, false>()));
      const long long rem = cols % slots;
      if (cols > slots && rem > 0 && 2 * rem <= slots) a.tail = (int)rem;
    }
    if (a.tail > 0) {
      g = dim3((unsigned)((long long)ntx * nty * a.npatch + a.tail));
    } else {
      const int ez = a.maxn[2] + 2 * a.w, nzc = a.zlen > 0 ? (ez + a.zlen - 1) / a.zlen : 1;
      g = dim3(ntx * nty, a.npatch, nzc);
    }
    if (fl && a.bnd) k_advance3d_fused<T, V, 1, true><<<g, FusedCfg<V>::NT, fused_smem<V>(), s>>>(a, ntx);
    else if (fl) k_advance3d_fused<T, V, 0, true><<<g, FusedCfg<V>::NT, fused_smem<V>(), s>>>(a, ntx);
    else if (a.bnd) k_advance3d_fused<T, V, 1><<<g, FusedCfg<V>::NT, fused_smem<V>(), s>>>(a, ntx);
    else if (a.nbr && a.w == 0) k_advance3d_fused<T, V, 2><<<g, FusedCfg<V>::NT, fused_smem<V>(), s>>>(a, ntx);
    else k_advance3d_fused<T, V, 0><<<g, FusedCfg<V>::NT, fused_smem<V>(), s>>>(a, ntx);
  }
  static void advance_fused(const LevelArgs& a, int variant, cudaStream_t s, int* nl) {
    if (DIM != 3) {
      advance(a, s, nl);
      return;
    }
    // variants whose shared memory does not fit fall back to the 8x8 tile
    if (variant == 0 && fused_fits<0>()) launch_fused<0>(a, s);
    else if (variant == 1 && fused_fits<1>()) launch_fused<1>(a, s);
    else if (variant == 2 && fused_fits<2>()) launch_fused<2>(a, s);
    else if (variant == 4 && fused_fits<4>()) launch_fused<4>(a, s);
    else launch_fused<3>(a, s);
    if (nl) ++*nl;
  }
  // registers recomputed from the state read by the advance (fused path, 3D)
  // one launch per register side: the face rows' blocks, then the edge rows'
  static void reg_coarse_rc(const RowArgs& f, const RowArgs& e, const double* idx, double gamma, cudaStream_t s,
                            int* nl) {
    if (DIM != 3) return;
    const unsigned nbf = (unsigned)cdiv(f.nrows, 128), nbe = (unsigned)cdiv(e.nrows, 128);
    if (!(nbf + nbe)) return;
    k_regrc_coarse<T><<<nbf + nbe, 128, 0, s>>>(f, e, nbf, gamma, idx[0], idx[1], idx[2]);
    if (nl) ++*nl;
  }
  static void reg_fine_rc(const RowArgs& f, const RowArgs& e, const double* idx, double gamma, cudaStream_t s,
                          int* nl) {
    if (DIM != 3) return;
    const unsigned nbf = (unsigned)cdiv(f.nrows, 128), nbe = (unsigned)cdiv(e.nrows, 128);
    if (!(nbf + nbe)) return;
    if (f.bnd)  // from the fine advance's boundary capture
      k_regcap_fine<T><<<nbf + nbe, 128, 0, s>>>(f, e, nbf, gamma, idx[0], idx[1], idx[2]);
    else
      k_regrc_fine<T><<<nbf + nbe, 128, 0, s>>>(f, e, nbf, gamma, idx[0], idx[1], idx[2]);
    if (nl) ++*nl;
  }
  static const Ops* ops() {
    static const Ops o = {advance, reg_coarse, reg_fine, fill_runs, prolong, fill_bc_cells, fill_bc_faces,
                          reflux_restrict, cfl, io,
                          io_all, sizeof(T), prepare, advance_fused, reg_coarse_rc, reg_fine_rc, flag, transfer_cells,
                          transfer_faces, closure, advance_queue, flag_dense};
    return &o;
  }
};

}  // namespace AMRK_NS
