// Fused 3D level advance: one CTA per (patch, x-y tile, z chunk), marching
// along z with rolling plane buffers in shared memory, so that primitives,
// slopes, predicted states, HLLD fluxes and CT EMFs never leave the SM. Only
// the state is read and written in HBM. Included by kernels_impl.cuh inside
// AMRK_NS.
//
// Pipeline per iteration t (planes in patch-local storage coordinates; the
// patch's output z range is [zlo, zhi) = [4-w, n_z+4+w), a CTA's the chunk
// [zs, ze) of it: a.zlen planes from zlo + a.zlen * chunk, or all of them when
// a.zlen is 0; a chunk restarts the march 2 planes below its first output
// plane, so a split column recomputes 4 planes of primitives, 2 of predictor
// and fluxes and 1 of EMFs per extra chunk, and every output value is the
// same bit for bit whatever the split):
//   S1  W at plane t                     (tile + 2 halo)        -> ring of 3
//       (and the normal-B differences of the tile + 1 halo; then cp.async
//       prefetch of the stored values of the plane S5 updates)
//   S2  slopes, predictor, reference EMF at plane p = t-1 (tile + 1 halo)
//   S3  HLLD fluxes: x- and y-faces of plane p, z-faces of face plane p
//   S4  edge EMFs: E_z at plane p, E_x and E_y at edge plane p
//   S5  update of cell plane q = p-1: cells, B_x and B_y of plane q, B_z of face
//       plane q (and the top face plane zhi on the patch's last plane)
// followed in the next iteration by S1 without a barrier (S5 touches no buffer
// S1 writes). Buffers that span iterations are 2- or 3-slot rings by plane.

// Tile variants (x-y output tile and threads per CTA), chosen by the
// autotuning option: 0 = 16x16 / 256, 1 = 16x16 / 512, 2 = 16x8 / 256,
// 3 = 8x8 / 256, 4 = 12x12 / 256 (an 8^3 patch with its 2 extended layers).
template <int V> struct FusedCfg;
template <> struct FusedCfg<0> { static constexpr int TX = 16, TY = 16, NT = 256; };
template <> struct FusedCfg<1> { static constexpr int TX = 16, TY = 16, NT = 512; };
template <> struct FusedCfg<2> { static constexpr int TX = 16, TY = 8, NT = 256; };
template <> struct FusedCfg<3> { static constexpr int TX = 8, TY = 8, NT = 256; };
template <> struct FusedCfg<4> { static constexpr int TX = 12, TY = 12, NT = 256; };

template <class T, int TX_, int TY_> struct FusedSmem {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int PX = TX + 4, PY = TY + 4, P = PX * PY;  // W region
  static constexpr int QX = TX + 2, QY = TY + 2, Q = QX * QY;  // predict / flux / EMF region
  T w[3][8][P];
  T wh[2][8][Q];
  T sz[2][8][Q];
  T sx[8][Q];
  T sy[8][Q];
  T ref[3][3][Q];
  T fx[2][8][Q];
  T fy[2][8][Q];
  T fz[2][8][Q];
  T ez[2][Q];
  T ex[2][Q];
  T ey[2][Q];
  T db[2][3][Q];                 // normal-B face differences of the Q region (slopes of B_d along d)
  T up[9][(TX + 1) * (TY + 1)];  // the update plane's stored values (8 fields, then B_z one plane up)
};

// asynchronous 4- or 8-byte global -> shared copy (cp.async, no registers)
template <class T> __device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <class T>
__device__ __forceinline__ void hlld_face(const T* wl, const T* wr, int D, T gamma, T* out8) {
  const int n = D, t = (D + 1) % 3, u = (D + 2) % 3;
  const T bn = T(0.5) * (wl[5 + n] + wr[5 + n]);
  const T ql[7] = {wl[0], wl[1 + n], wl[1 + t], wl[1 + u], wl[4], wl[5 + t], wl[5 + u]};
  const T qr[7] = {wr[0], wr[1 + n], wr[1 + t], wr[1 + u], wr[4], wr[5 + t], wr[5 + u]};
  T fr[7];
  hlld_flux<T>(ql, qr, bn, gamma, fr);
  out8[RHO] = fr[0];
  out8[MX + n] = fr[1];
  out8[MX + t] = fr[2];
  out8[MX + u] = fr[3];
  out8[EN] = fr[4];
  out8[BX + t] = fr[5];
  out8[BX + u] = fr[6];
  out8[BX + n] = T(0);
}

template <class T>
__device__ __forceinline__ void load_recover(const T* U, long long fs, int L, int sy, int sz, double gm1, T* w,
                                             T* dB = nullptr, const Floors* fl = nullptr) {
  T u[5], bl[3], br[3];
#pragma unroll
  for (int f = 0; f < 5; ++f) u[f] = U[f * fs + L];
  bl[0] = U[5 * fs + L]; br[0] = U[5 * fs + L + 1];
  bl[1] = U[6 * fs + L]; br[1] = U[6 * fs + L + sy];
  bl[2] = U[7 * fs + L]; br[2] = U[7 * fs + L + sz];
  if (fl) floor_density(u, fl->rho, fl->events);
  recover_t(u, bl, br, gm1, w);
  if (fl) floor_pressure(w, fl->p, fl->events);
  if (dB) {
#pragma unroll
    for (int d = 0; d < 3; ++d) dB[d] = br[d] - bl[d];
  }
}

// ---------------------------------------------------------------- boundary capture
// The fluxes and EMFs on the six boundary planes of a fine patch, written by the
// fused advance and read by the fine-side registers (levels > 0), instead of
// recomputing them there. Per patch at P.boff (elements of the state type): the
// 5 conserved-flux components (field-major) of every boundary face, planes in
// the order x-low, x-high, y-low, y-high, z-low, z-high, a plane of normal e
// holding n_t1 x n_t2 faces (t1 < t2 the other axes, t1 fastest); then the
// tangential EMFs of the boundary planes in the same plane order, per plane its
// two components c != e ascending, each over n_c x (n_o + 1) edges (c fastest,
// o the remaining axis).
// slot of the e-face at local (x, y, z) if it lies on a boundary plane, else -1
__device__ __forceinline__ long long bnd_face_slot(const DPatch& P, int e, int x, int y, int z) {
  const int pos[3] = {x, y, z};
  const int side = pos[e] == 4 ? 0 : (pos[e] == P.n[e] + 4 ? 1 : -1);
  if (side < 0) return -1;
  const int t1 = e == 0 ? 1 : 0, t2 = e == 2 ? 1 : 2;
  const int u = pos[t1] - 4, v = pos[t2] - 4;
  if (u < 0 || u >= P.n[t1] || v < 0 || v >= P.n[t2]) return -1;
  const long long S0 = (long long)P.n[1] * P.n[2], S1 = (long long)P.n[0] * P.n[2], S2 = (long long)P.n[0] * P.n[1];
  const long long Se = e == 0 ? S0 : (e == 1 ? S1 : S2);
  const long long base = (e == 0 ? 0 : (e == 1 ? 2 * S0 : 2 * (S0 + S1))) + side * Se;
  return base + u + (long long)P.n[t1] * v;
}
// slot of the c-edge at local (x, y, z) on the boundary plane of normal e, else -1
__device__ __forceinline__ long long bnd_edge_slot(const DPatch& P, int c, int e, int x, int y, int z) {
  const int pos[3] = {x, y, z};
  const int side = pos[e] == 4 ? 0 : (pos[e] == P.n[e] + 4 ? 1 : -1);
  if (side < 0) return -1;
  const int o = 3 - c - e;
  const int u = pos[c] - 4, v = pos[o] - 4;
  if (u < 0 || u >= P.n[c] || v < 0 || v > P.n[o]) return -1;
  long long base = 0;
  for (int ee = 0; ee < 3; ++ee)
    for (int s2 = 0; s2 < 2; ++s2)
      for (int cc = 0; cc < 3; ++cc) {
        if (cc == ee) continue;
        if (ee == e && s2 == side && cc == c) return base + u + (long long)P.n[c] * v;
        base += (long long)P.n[cc] * (P.n[3 - cc - ee] + 1);
      }
  return -1;
}
template <class T>
__device__ __forceinline__ void bnd_store_edge(const LevelArgs& a, const DPatch& P, int c, int x, int y, int z, T v) {
  T* b = (T*)a.bnd + P.boff + 5 * bnd_faces_total(P.n);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (e == c) continue;
    const long long sl = bnd_edge_slot(P, c, e, x, y, z);
    if (sl >= 0) b[sl] = v;
  }
}

// One x-y tile (index `tile`, ntx tiles along x) of the patch at position
// `pslot` of a.ids, marched along z by the whole CTA over the z chunk `zc`
// (a.zlen planes each; 0: the whole column); smem_raw: the CTA's
// dynamic shared memory (a FusedSmem). MODE 0: plain; 1 (CAP): the level's
// boundary fluxes and EMFs are captured for the fine registers (patches with
// P.boff >= 0); 2 (DH): direct halo reads from the neighbour patches (a.nbr; a
// level of equal patches tiling the periodic domain, w = 0). FL: the recovery
// applies the density and pressure floors of a.fl (never with DH). Every thread
// of the CTA calls it with the same arguments.
template <class T, int VAR, int MODE, bool FL = false>
__device__ __forceinline__ void fused_tile(const LevelArgs& a, int pslot, int tile, int ntx, int zc,
                                           unsigned char* smem_raw, bool halves = false) {
  constexpr bool CAP = MODE == 1, DH = MODE == 2;
  using S = FusedSmem<T, FusedCfg<VAR>::TX, FusedCfg<VAR>::TY>;
  constexpr int TX = S::TX, TY = S::TY, PX = S::PX, QX = S::QX;
  S& sm = *reinterpret_cast<S*>(smem_raw);
  __shared__ long long s_nb[DH ? 27 : 1];  // element offsets of the neighbour patches (DH)
  const DPatch P = a.P[a.ids[pslot]];
  if constexpr (DH) {
    if (threadIdx.x < 27) s_nb[threadIdx.x] = a.P[a.nbr[27 * pslot + threadIdx.x]].off;
    __syncthreads();
  }
  const int w = a.w;
  const int xlo = 4 - w, xhi = P.n[0] + 4 + w, ylo = 4 - w, yhi = P.n[1] + 4 + w;
  const int zlo = 4 - w, zhi = P.n[2] + 4 + w;
  const int x0 = xlo + (tile % ntx) * TX, y0 = ylo + (tile / ntx) * TY;
  // the chunk: a.zlen planes from zlo + a.zlen zc, the whole column (a.zlen
  // 0), or with halves its lower (zc 0) or upper (zc 1) half
  const int zl = halves ? (zhi - zlo + 1) / 2 : a.zlen;
  const int zs = zlo + zc * zl, ze = zl > 0 ? min(zs + zl, zhi) : zhi;
  if (x0 >= xhi || y0 >= yhi || zs >= zhi) return;
  // a face or edge plane shared by two chunks (ze of one, zs of the next) is
  // captured by the upper chunk only
  const bool cap_ze = ze == zhi;
  const int tx = min(TX, xhi - x0), ty = min(TY, yhi - y0);
  const bool last_x = x0 + tx == xhi, last_y = y0 + ty == yhi;
  const long long fs = P.fs;
  const int sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  const T* U = (const T*)a.cur + P.off;
  T* V = (T*)a.nxt + P.off;
  const bool capture = CAP && P.boff >= 0;
  const double gm1 = a.gamma - 1.0;
  const Floors* flp = FL ? &a.fl : nullptr;
  const T gamma = (T)a.gamma;
  const double dt = *a.dtp * a.dtscale;
  const T h0 = (T)(0.5 * dt * a.idx[0]), h1 = (T)(0.5 * dt * a.idx[1]), h2 = (T)(0.5 * dt * a.idx[2]);
  const T dtd[3] = {(T)(dt * a.idx[0]), (T)(dt * a.idx[1]), (T)(dt * a.idx[2])};
  const int nth = blockDim.x;
  // W region columns: x in [x0-2, x0+tx+2), y in [y0-2, y0+ty+2); Q region: +-1
  const int wx = tx + 4, wy = ty + 4, qx = tx + 2, qy = ty + 2;
  auto widx = [&](int x, int y) { return (x - (x0 - 2)) + PX * (y - (y0 - 2)); };
  auto qidx = [&](int x, int y) { return (x - (x0 - 1)) + QX * (y - (y0 - 1)); };

  // The stages, each over the positions of one plane, every thread taking
  // positions in steps of the CTA size:
  //   S1(t)  primitives of plane t (W ring slot t mod 3; normal-B differences)
  //   S2(p)  slopes, predictor and reference EMF of plane p
  //   S3(p)  HLLD fluxes of the x- and y-faces of plane p and the z-faces of face plane p
  //   S4(p)  edge EMFs: E_z of plane p, E_x and E_y of edge plane p
  //   S5(q)  update of cell plane q (its stored values prefetched by cp.async)
  auto stage1 = [&](int t) {
      // ---------------- S1: primitives of plane t
      {
        const int slot = (t + 3) % 3;
        const int r2t = (t + 2) % 2;
        for (int c = threadIdx.x; c < PX * S::PY; c += nth) {
          const int xi = c % PX, yi = c / PX;  // constant divisors; positions beyond a partial tile skip
          if (xi >= wx || yi >= wy) continue;
          const int x = x0 - 2 + xi, y = y0 - 2 + yi;
          T wv[8], dB[3];
          if constexpr (DH) {
            // the cell (and its faces) in the neighbour patch that owns it: every
            // patch has the interior extent n, so a coordinate outside [4, n+4)
            // moves by n into the neighbour's interior (its own high faces at n+4
            // included); the neighbours' strides are this patch's
            int lx = x, ly = y, lz = t, k = 13;
            if (x < 4) { lx += P.n[0]; k -= 1; } else if (x >= P.n[0] + 4) { lx -= P.n[0]; k += 1; }
            if (y < 4) { ly += P.n[1]; k -= 3; } else if (y >= P.n[1] + 4) { ly -= P.n[1]; k += 3; }
            if (t < 4) { lz += P.n[2]; k -= 9; } else if (t >= P.n[2] + 4) { lz -= P.n[2]; k += 9; }
            load_recover((const T*)a.cur + s_nb[k], fs, lx + sy * ly + sz * lz, sy, sz, gm1, wv, dB, flp);
          } else {
            load_recover(U, fs, x + sy * y + sz * t, sy, sz, gm1, wv, dB, flp);
          }
          const int i = widx(x, y);
#pragma unroll
          for (int f = 0; f < 8; ++f) sm.w[slot][f][i] = wv[f];
          if (x >= x0 - 1 && x < x0 + tx + 1 && y >= y0 - 1 && y < y0 + ty + 1) {
            const int q = qidx(x, y);
#pragma unroll
            for (int d = 0; d < 3; ++d) sm.db[r2t][d][q] = dB[d];
          }
        }
      }
  };
  auto prefetch = [&](int qz) {
      {
        if (qz >= zs && qz < ze) {
          // the tile's cells (all 8 stored values; B_z of the top face plane
          // too on the patch's last plane), and on the patch's high x (y) side
          // the B_x (B_y) faces of the column x0+tx (the row y0+ty)
          const int nx = tx + (last_x ? 1 : 0), ny = ty + (last_y ? 1 : 0);
          const bool top = qz == zhi - 1;
          for (int c = threadIdx.x; c < (TX + 1) * (TY + 1); c += nth) {
            const int xi = c % (TX + 1), yi = c / (TX + 1);
            if (xi >= nx || yi >= ny) continue;
            const int L = (x0 + xi) + sy * (y0 + yi) + sz * qz;
            if (xi < tx && yi < ty) {
#pragma unroll
              for (int f = 0; f < 8; ++f) cp_async_elem<T>(&sm.up[f][c], U + f * fs + L);
              if (top) cp_async_elem<T>(&sm.up[8][c], U + BZ * fs + L + sz);
            } else if (yi < ty) {
              cp_async_elem<T>(&sm.up[BX][c], U + BX * fs + L);
            } else if (xi < tx) {
              cp_async_elem<T>(&sm.up[BY][c], U + BY * fs + L);
            }
          }
        }
        cp_async_commit();
      }
  };
  auto stage2 = [&](int p) {
      // ---------------- S2: slopes and predictor of plane p
      {
        const int sm1 = (p - 1 + 3) % 3, s0 = (p + 3) % 3, sp1 = (p + 1 + 3) % 3;
        const int r2 = (p + 2) % 2, r3 = (p + 3) % 3;
        for (int c = threadIdx.x; c < QX * S::QY; c += nth) {
          const int xi = c % QX, yi = c / QX;
          if (xi >= qx || yi >= qy) continue;
          const int x = x0 - 1 + xi, y = y0 - 1 + yi;
          const int i = widx(x, y);
          T wc[8], s[3][8];
          const int qd = qidx(x, y);
#pragma unroll
          for (int f = 0; f < 8; ++f) wc[f] = sm.w[s0][f][i];
#pragma unroll
          for (int f = 0; f < 8; ++f) {
            s[0][f] = f == BX ? sm.db[r2][0][qd] : mm(wc[f] - sm.w[s0][f][i - 1], sm.w[s0][f][i + 1] - wc[f]);
            s[1][f] = f == BY ? sm.db[r2][1][qd] : mm(wc[f] - sm.w[s0][f][i - PX], sm.w[s0][f][i + PX] - wc[f]);
            s[2][f] = f == BZ ? sm.db[r2][2][qd] : mm(wc[f] - sm.w[sm1][f][i], sm.w[sp1][f][i] - wc[f]);
          }
          const T ir = T(1) / wc[0];
          T wh[8], dw[8];
#pragma unroll
          for (int f = 0; f < 8; ++f) wh[f] = wc[f];
          prim_terms<T, 0>(wc, s[0], gamma, ir, dw);
#pragma unroll
          for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h0 * dw[f];
          prim_terms<T, 1>(wc, s[1], gamma, ir, dw);
#pragma unroll
          for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h1 * dw[f];
          prim_terms<T, 2>(wc, s[2], gamma, ir, dw);
#pragma unroll
          for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h2 * dw[f];
          const int q = qidx(x, y);
#pragma unroll
          for (int f = 0; f < 8; ++f) {
            sm.wh[r2][f][q] = wh[f];
            sm.sx[f][q] = s[0][f];
            sm.sy[f][q] = s[1][f];
            sm.sz[r2][f][q] = s[2][f];
          }
          sm.ref[r3][0][q] = wh[3] * wh[6] - wh[2] * wh[7];
          sm.ref[r3][1][q] = wh[1] * wh[7] - wh[3] * wh[5];
          sm.ref[r3][2][q] = wh[2] * wh[5] - wh[1] * wh[6];
        }
      }
  };
  auto stage3 = [&](int p) {
      // ---------------- S3: fluxes (x, y faces of plane p; z faces of face plane p)
      {
        const int r2 = (p + 2) % 2, rm = (p + 1) % 2;
        constexpr int NFX = (TX + 1) * (S::QY), NFY = (QX) * (TY + 1), NFZ = QX * S::QY, Q = S::Q;
        const int nf = NFX + NFY + (p >= zs ? NFZ : 0);
        // boundary capture: x- and y-faces of the chunk's own planes, z-faces of
        // its face planes (the top one only on the column's last chunk)
        const bool cap_xy = capture && p >= zs && p < ze, cap_z = capture && (p < ze || cap_ze);
        for (int c = threadIdx.x; c < nf; c += nth) {
          // one face: direction D, its high-side cell (x, y) and the offset of its low-side cell
          int D, x, y, lo;
          const T *whl, *whr, *sl, *sr;
          T* fo;
          if (c < NFX) {  // x-face at x (cells x-1, x), y in [y0-1, y0+ty+1)
            const int xi = c % (TX + 1), yi = c / (TX + 1);
            if (xi > tx || yi >= ty + 2) continue;
            D = 0; x = x0 + xi; y = y0 - 1 + yi; lo = -1;
            whl = whr = &sm.wh[r2][0][0];
            sl = sr = &sm.sx[0][0];
            fo = &sm.fx[r2][0][0];
          } else if (c < NFX + NFY) {  // y-face at y (cells y-1, y), x in [x0-1, x0+tx+1)
            const int cc = c - NFX, xi = cc % QX, yi = cc / QX;
            if (xi >= tx + 2 || yi > ty) continue;
            D = 1; x = x0 - 1 + xi; y = y0 + yi; lo = -QX;
            whl = whr = &sm.wh[r2][0][0];
            sl = sr = &sm.sy[0][0];
            fo = &sm.fy[r2][0][0];
          } else {  // z-face at face plane p (cells p-1, p)
            const int cc = c - NFX - NFY, xi = cc % QX, yi = cc / QX;
            if (xi >= tx + 2 || yi >= ty + 2) continue;
            D = 2; x = x0 - 1 + xi; y = y0 - 1 + yi; lo = 0;
            whl = &sm.wh[rm][0][0];
            whr = &sm.wh[r2][0][0];
            sl = &sm.sz[rm][0][0];
            sr = &sm.sz[r2][0][0];
            fo = &sm.fz[r2][0][0];
          }
          const int q = qidx(x, y), ql = q + lo;
          const int n = D, t = D == 2 ? 0 : D + 1, u = D == 0 ? 2 : D - 1;
          // the predicted face states, read in the face's rotated order (rho, v_n,
          // v_t, v_u, p, B_t, B_u), and the mean normal field; fluxes stored back by field
          const int fi[7] = {RHO, MX + n, MX + t, MX + u, EN, BX + t, BX + u};
          T qlv[7], qrv[7], fr[7];
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            qlv[k] = whl[fi[k] * Q + ql] + T(0.5) * sl[fi[k] * Q + ql];
            qrv[k] = whr[fi[k] * Q + q] - T(0.5) * sr[fi[k] * Q + q];
          }
          const T bnl = whl[(BX + n) * Q + ql] + T(0.5) * sl[(BX + n) * Q + ql];
          const T bnr = whr[(BX + n) * Q + q] - T(0.5) * sr[(BX + n) * Q + q];
          hlld_flux<T>(qlv, qrv, T(0.5) * (bnl + bnr), gamma, fr);
#pragma unroll
          for (int k = 0; k < 7; ++k) fo[fi[k] * Q + q] = fr[k];
          fo[(BX + n) * Q + q] = T(0);
          if (D < 2 ? cap_xy : cap_z) {  // a boundary face of a fine patch: keep its flux for the registers
            const long long sl = bnd_face_slot(P, D, x, y, p);
            if (sl >= 0) {
              T* b = (T*)a.bnd + P.boff;
              const long long F = bnd_faces_total(P.n);
#pragma unroll
              for (int k = 0; k < 5; ++k) b[fi[k] * F + sl] = fr[k];
            }
          }
        }
      }
  };
  auto stage4 = [&](int p) {
      // ---------------- S4: edge EMFs
      {
        const int r2 = (p + 2) % 2, rm = (p + 1) % 2;
        const int r3 = (p + 3) % 3, rm3 = (p + 2) % 3;  // reference EMFs of planes p and p-1
        constexpr int NEZ = (TX + 1) * (TY + 1), NEX = TX * (TY + 1), NEY = (TX + 1) * TY;
        const int nez = p < ze ? NEZ : 0;
        const bool cap_e = capture && (p < ze || cap_ze);  // E_x, E_y of edge plane p
        for (int c = threadIdx.x; c < nez + NEX + NEY; c += nth) {
          if (c < nez) {  // E_z at corner (x-1/2, y-1/2) of plane p: a = x, b = y
            const int xi = c % (TX + 1), yi = c / (TX + 1);
            if (xi > tx || yi > ty) continue;
            const int x = x0 + xi, y = y0 + yi;
            const int q11 = qidx(x, y), q01 = q11 - 1, q10 = q11 - QX, q00 = q11 - 1 - QX;
            const T ea_hi = -sm.fx[r2][BY][q11], ea_lo = -sm.fx[r2][BY][q10];
            const T eb_hi = sm.fy[r2][BX][q11], eb_lo = sm.fy[r2][BX][q01];
            sm.ez[r2][q11] = gs_emf<T>(ea_lo, ea_hi, eb_lo, eb_hi, sm.ref[r3][2][q00], sm.ref[r3][2][q10],
                                       sm.ref[r3][2][q01], sm.ref[r3][2][q11], sm.fx[r2][RHO][q10], sm.fx[r2][RHO][q11],
                                       sm.fy[r2][RHO][q01], sm.fy[r2][RHO][q11]);
            if (capture) bnd_store_edge<T>(a, P, 2, x, y, p, sm.ez[r2][q11]);
          } else if (c < nez + NEX) {  // E_x at (x, y-1/2, p-1/2): a = y, b = z
            const int cc = c - nez, xi = cc % TX, yi = cc / TX;
            if (xi >= tx || yi > ty) continue;
            const int x = x0 + xi, y = y0 + yi;
            const int q = qidx(x, y), qm = q - QX;
            // a-faces = y-faces at rows z = p-1, p; b-faces = z-faces at columns y-1, y
            const T ea_lo = -sm.fy[rm][BZ][q], ea_hi = -sm.fy[r2][BZ][q];
            const T eb_lo = sm.fz[r2][BY][qm], eb_hi = sm.fz[r2][BY][q];
            sm.ex[r2][q] = gs_emf<T>(ea_lo, ea_hi, eb_lo, eb_hi, sm.ref[rm3][0][qm], sm.ref[rm3][0][q], sm.ref[r3][0][qm],
                                     sm.ref[r3][0][q], sm.fy[rm][RHO][q], sm.fy[r2][RHO][q], sm.fz[r2][RHO][qm],
                                     sm.fz[r2][RHO][q]);
            if (cap_e) bnd_store_edge<T>(a, P, 0, x, y, p, sm.ex[r2][q]);
          } else {  // E_y at (x-1/2, y, p-1/2): a = z, b = x
            const int cc = c - nez - NEX, xi = cc % (TX + 1), yi = cc / (TX + 1);
            if (xi > tx || yi >= ty) continue;
            const int x = x0 + xi, y = y0 + yi;
            const int q = qidx(x, y), qm = q - 1;
            // a-faces = z-faces at rows x-1, x; b-faces = x-faces at columns z = p-1, p
            const T ea_lo = -sm.fz[r2][BX][qm], ea_hi = -sm.fz[r2][BX][q];
            const T eb_lo = sm.fx[rm][BZ][q], eb_hi = sm.fx[r2][BZ][q];
            // references: r00 = (z p-1, x-1), r10 = (z p, x-1), r01 = (z p-1, x), r11 = (z p, x)
            sm.ey[r2][q] = gs_emf<T>(ea_lo, ea_hi, eb_lo, eb_hi, sm.ref[rm3][1][qm], sm.ref[r3][1][qm], sm.ref[rm3][1][q],
                                     sm.ref[r3][1][q], sm.fz[r2][RHO][qm], sm.fz[r2][RHO][q], sm.fx[rm][RHO][q],
                                     sm.fx[r2][RHO][q]);
            if (cap_e) bnd_store_edge<T>(a, P, 1, x, y, p, sm.ey[r2][q]);
          }
        }
      }
  };
  auto stage5 = [&](int qz) {
      if (qz >= zs && qz < ze) {
        const int p = qz + 1;
        const int rq = (qz + 2) % 2, rp = (p + 2) % 2;
        const int nx = tx + (last_x ? 1 : 0), ny = ty + (last_y ? 1 : 0);
        for (int c = threadIdx.x; c < (TX + 1) * (TY + 1); c += nth) {
          const int xi = c % (TX + 1), yi = c / (TX + 1);
          if (xi >= nx || yi >= ny) continue;
          const int x = x0 + xi, y = y0 + yi;
          const bool in_x = x < x0 + tx, in_y = y < y0 + ty;
          const int L = x + sy * y + sz * qz;
          const int q = qidx(x, y);
          const int u = c;
          if (in_x && in_y) {
#pragma unroll
            for (int n = 0; n < 5; ++n) {
              T v = sm.up[n][u];
              v = v - dtd[0] * (sm.fx[rq][n][q + 1] - sm.fx[rq][n][q]);
              v = v - dtd[1] * (sm.fy[rq][n][q + QX] - sm.fy[rq][n][q]);
              v = v - dtd[2] * (sm.fz[rp][n][q] - sm.fz[rq][n][q]);
              V[n * fs + L] = v;
            }
            // B_z of face plane qz (and the top face plane on the last plane)
            {
              T v = sm.up[BZ][u];
              v = v - dtd[0] * (sm.ey[rq][q + 1] - sm.ey[rq][q]);
              v = v + dtd[1] * (sm.ex[rq][q + QX] - sm.ex[rq][q]);
              V[BZ * fs + L] = v;
            }
            if (qz == zhi - 1) {
              T v = sm.up[8][u];
              v = v - dtd[0] * (sm.ey[rp][q + 1] - sm.ey[rp][q]);
              v = v + dtd[1] * (sm.ex[rp][q + QX] - sm.ex[rp][q]);
              V[BZ * fs + L + sz] = v;
            }
          }
          if (in_y) {  // B_x at (x, y, qz)
            T v = sm.up[BX][u];
            v = v - dtd[1] * (sm.ez[rq][q + QX] - sm.ez[rq][q]);
            v = v + dtd[2] * (sm.ey[rp][q] - sm.ey[rq][q]);
            V[BX * fs + L] = v;
          }
          if (in_x) {  // B_y at (x, y, qz)
            T v = sm.up[BY][u];
            v = v - dtd[2] * (sm.ex[rp][q] - sm.ex[rq][q]);
            v = v + dtd[0] * (sm.ez[rq][q + 1] - sm.ez[rq][q]);
            V[BY * fs + L] = v;
          }
        }
      }
  };

  // Schedule: three barriers per plane. Phase 1 pairs the fluxes of plane p
  // with the primitives of plane p+2 (and the prefetch of the update plane);
  // phase 2 the EMFs of plane p with the predictor of plane p+1; phase 3 the
  // update of plane p-1. Rings: W 3 planes (S1(p+2) replaces W(p-1), which only
  // S2(p) of the previous phase 2 read), reference EMFs 3 planes (S2(p+1)
  // writes while S4(p) reads planes p and p-1), the rest 2 planes.
  stage1(zs - 2);
  stage1(zs - 1);
  stage1(zs);
  __syncthreads();
  stage2(zs - 1);
  __syncthreads();
  for (int p = zs - 1; p <= ze; ++p) {
    prefetch(p - 1);
    stage3(p);
    if (p + 2 <= ze + 1) stage1(p + 2);
    __syncthreads();
    if (p >= zs) stage4(p);
    if (p + 1 <= ze) stage2(p + 1);
    cp_async_wait_all();
    __syncthreads();
    stage5(p - 1);
    __syncthreads();
  }
}

// CTAs per SM of the FP32 tiles of 256 threads: two for the larger tiles
// (shared memory), three for the 8x8 tile (80 registers a thread, no spills)
template <int VAR> constexpr int fused_ctas_fp32() { return FusedCfg<VAR>::NT != 256 ? 1 : (VAR == 3 ? 3 : 2); }
template <class T, int VAR, int MODE, bool FL = false>
__global__ void __launch_bounds__(FusedCfg<VAR>::NT, sizeof(T) == 4 ? fused_ctas_fp32<VAR>() : 1)
    k_advance3d_fused(LevelArgs a, int ntx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int pslot = blockIdx.y, tile = blockIdx.x, zc = blockIdx.z;
  bool halves = false;
  if (a.tail > 0) {
    // one-dimensional grid over the columns (patch-major): the first ones
    // whole, the last a.tail ones as two halves each, so that the launch's last
    // partial wave holds half-length marches
    constexpr int TY = FusedCfg<VAR>::TY;
    const int ntiles = ntx * ((a.maxn[1] + 2 * a.w + TY - 1) / TY);
    const int full = ntiles * a.npatch - a.tail;
    const int item = blockIdx.x;
    const int col = item < full ? item : full + (item - full) / 2;
    pslot = col / ntiles;
    tile = col % ntiles;
    zc = item < full ? 0 : (item - full) % 2;
    halves = item >= full;
  }
  fused_tile<T, VAR, MODE, FL>(a, pslot, tile, ntx, zc, smem_raw, halves);
}

// ---------------------------------------------------------------- device work queue
// The multi-level advance as persistent launches (the GPU analogue of the
// paper's threaded level advances with preference to the finer levels, Sec. 4):
// one launch per sub-step of the finest level; the resident CTAs take tasks in
// ticket order from an atomic counter over a host-ordered list. Fill tasks (a
// range of same-level copy chunks into one patch, the finest level's) come
// first, then the advance tiles, finest level first: all of the finest
// level's, then a share of every coarser level's (a coarser level's advance
// is spread over the launches of its sub-step). An advance tile waits until every fill task into its patch has
// finished (a per-patch counter against the expected count). A wait only ever
// concerns tasks of smaller tickets, which running CTAs hold and finish
// without waiting, so every wait ends; each is bounded in time all the same:
// on expiry the CTA sets ERR_QUEUE_TIMEOUT in the error word and the abort
// flag, and every CTA stops taking tasks (no wait is left in flight: the CTA
// holds no asynchronous copies while it waits).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned int load_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <class T, int VAR>
__global__ void __launch_bounds__(FusedCfg<VAR>::NT, sizeof(T) == 4 ? 2 : 1)
    k_advance_queue(const __grid_constant__ QueueArgs q) {
  static_assert(FusedCfg<VAR>::NT == FILL_RUN_TPB, "the fill tasks use the CTA's threads as k_fill_runs does");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int4 s_task;
  __shared__ int s_go;
  for (;;) {
    if (threadIdx.x == 0) {
      int4 t = make_int4(-1, 0, 0, 0);
      if (!(*(volatile unsigned int*)q.err & ERR_QUEUE_TIMEOUT) && !*(volatile int*)q.abort) {
        const unsigned int k = atomicAdd(q.head, 1u);
        if (k < (unsigned int)q.ntasks) t = reinterpret_cast<const int4*>(q.tasks)[k];
      }
      s_task = t;
    }
    __syncthreads();
    const int4 t = s_task;
    if (t.x < 0) return;
    const QueueLevel& L = q.L[t.x >> 4];
    if (t.x & 1) {
      // fill task: the chunk range [t.y, t.z) of the level's same-level boxes
      int4* sch = reinterpret_cast<int4*>(smem_raw);
      T* B = (T*)L.a.cur;
      const int4* ch = reinterpret_cast<const int4*>(L.chunks);
      if (t.x & 2) fill_range<T, 5, 2>(B, L.boxes, ch, t.y, t.z, sch, sch + FILL_TILE);
      else fill_range<T, 1, 4>(B, L.boxes, ch, t.y, t.z, sch, sch + FILL_TILE);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(q.done + t.w, 1u);
      }
    } else {
      // advance tile: first every fill into its patch
      if (threadIdx.x == 0) {
        int go = 1;
        const unsigned int need = q.need[t.w];
        if (need) {
          const unsigned long long t0 = global_ns();
          while (load_acquire(q.done + t.w) < need) {
            if (*(volatile int*)q.abort) { go = 0; break; }
            if (global_ns() - t0 > q.wait_ns) {
              atomicOr(q.err, ERR_QUEUE_TIMEOUT);
              atomicExch(q.abort, 1);
              go = 0;
              break;
            }
            __nanosleep(128);
          }
          __threadfence();
        }
        s_go = go;
      }
      __syncthreads();
      if (s_go) fused_tile<T, VAR, 1>(L.a, t.y, t.z, L.ntx, 0, smem_raw);
    }
    __syncthreads();  // the task's shared memory is free for the next one
  }
}

// ------------------------------------------------------------------ register recompute
// Registers for the fused path, recomputed from the state the advance read:
// the same formulas as the fused kernel, evaluated at the listed faces/edges.
template <class T>
__device__ void predict_at(const T* U, const DPatch& P, int L, double dt, const double* idx, double gamma, T* wh,
                           T* sd /* 3 x 8 */, const Floors* fl) {
  const long long fs = P.fs;
  const int st[3] = {1, P.ext[0], P.ext[0] * P.ext[1]};
  const double gm1 = gamma - 1.0;
  T wc[8], wm[8], wp[8];
  load_recover(U, fs, L, st[1], st[2], gm1, wc, (T*)nullptr, fl);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    load_recover(U, fs, L - st[d], st[1], st[2], gm1, wm, (T*)nullptr, fl);
    load_recover(U, fs, L + st[d], st[1], st[2], gm1, wp, (T*)nullptr, fl);
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f == BX + d) sd[8 * d + f] = U[(BX + d) * fs + L + st[d]] - U[(BX + d) * fs + L];
      else sd[8 * d + f] = mm(wc[f] - wm[f], wp[f] - wc[f]);
    }
  }
  const T ir = T(1) / wc[0];
  const T g = (T)gamma;
  T dw[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) wh[f] = wc[f];
  const T h0 = (T)(0.5 * dt * idx[0]), h1 = (T)(0.5 * dt * idx[1]), h2 = (T)(0.5 * dt * idx[2]);
  prim_terms<T, 0>(wc, sd, g, ir, dw);
#pragma unroll
  for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h0 * dw[f];
  prim_terms<T, 1>(wc, sd + 8, g, ir, dw);
#pragma unroll
  for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h1 * dw[f];
  prim_terms<T, 2>(wc, sd + 16, g, ir, dw);
#pragma unroll
  for (int f = 0; f < 8; ++f) wh[f] = wh[f] - h2 * dw[f];
}

// flux through the d-face stored at L (cells L - st[d] and L), global field order
template <class T>
__device__ void face_flux_at(const T* U, const DPatch& P, int d, int L, double dt, const double* idx, double gamma,
                             T* out8, const Floors* fl) {
  const int st[3] = {1, P.ext[0], P.ext[0] * P.ext[1]};
  T whl[8], whr[8], sl[24], sr[24], wl[8], wr[8];
  predict_at(U, P, L - st[d], dt, idx, gamma, whl, sl, fl);
  predict_at(U, P, L, dt, idx, gamma, whr, sr, fl);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    wl[f] = whl[f] + T(0.5) * sl[8 * d + f];
    wr[f] = whr[f] - T(0.5) * sr[8 * d + f];
  }
  hlld_face<T>(wl, wr, d, (T)gamma, out8);
}

// E_c at the c-edge stored at L (the low a,b corner of cell L), (a,b,c) cyclic
template <class T>
__device__ T edge_emf_at(const T* U, const DPatch& P, int c, int L, double dt, const double* idx, double gamma,
                         const Floors* fl) {
  const int st[3] = {1, P.ext[0], P.ext[0] * P.ext[1]};
  const int a = (c + 1) % 3, b = (c + 2) % 3;
  const int Lc[4] = {L - st[a] - st[b], L - st[b], L - st[a], L};  // (a-1,b-1), (a,b-1), (a-1,b), (a,b)
  T wh[4][8], sd[4][24];
  for (int k = 0; k < 4; ++k) predict_at(U, P, Lc[k], dt, idx, gamma, wh[k], sd[k], fl);
  T wl[8], wr[8], fa_lo[8], fa_hi[8], fb_lo[8], fb_hi[8];
  const T g = (T)gamma;
  // a-faces at rows b-1 (cells 0 -> 1) and b (cells 2 -> 3)
#pragma unroll
  for (int f = 0; f < 8; ++f) { wl[f] = wh[0][f] + T(0.5) * sd[0][8 * a + f]; wr[f] = wh[1][f] - T(0.5) * sd[1][8 * a + f]; }
  hlld_face<T>(wl, wr, a, g, fa_lo);
#pragma unroll
  for (int f = 0; f < 8; ++f) { wl[f] = wh[2][f] + T(0.5) * sd[2][8 * a + f]; wr[f] = wh[3][f] - T(0.5) * sd[3][8 * a + f]; }
  hlld_face<T>(wl, wr, a, g, fa_hi);
  // b-faces at columns a-1 (cells 0 -> 2) and a (cells 1 -> 3)
#pragma unroll
  for (int f = 0; f < 8; ++f) { wl[f] = wh[0][f] + T(0.5) * sd[0][8 * b + f]; wr[f] = wh[2][f] - T(0.5) * sd[2][8 * b + f]; }
  hlld_face<T>(wl, wr, b, g, fb_lo);
#pragma unroll
  for (int f = 0; f < 8; ++f) { wl[f] = wh[1][f] + T(0.5) * sd[1][8 * b + f]; wr[f] = wh[3][f] - T(0.5) * sd[3][8 * b + f]; }
  hlld_face<T>(wl, wr, b, g, fb_hi);
  T r[4];
  for (int k = 0; k < 4; ++k) {
    const T* h = wh[k];
    r[k] = c == 0 ? h[3] * h[6] - h[2] * h[7] : (c == 1 ? h[1] * h[7] - h[3] * h[5] : h[2] * h[5] - h[1] * h[6]);
  }
  return gs_emf<T>(-fa_lo[BX + b], -fa_hi[BX + b], fb_lo[BX + a], fb_hi[BX + a], r[0], r[1], r[2], r[3], fa_lo[RHO],
                   fa_hi[RHO], fb_lo[RHO], fb_hi[RHO]);
}

// the floors a register recompute repeats (those of the advance it mirrors)
__device__ __forceinline__ const Floors* rc_floors(const RowArgs& a) {
  return (a.fl.rho > 0.0 || a.fl.p > 0.0) ? &a.fl : nullptr;
}

// RowArgs.fbuf = the state the level's advance read (for the coarse side the
// coarse level, for the fine side the fine level); dt = *dtp * dtscale.
template <class T>
__device__ __forceinline__ void regrc_coarse_faces_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[1]];
  const double dt = *a.dtp * a.dtscale;
  const double idx[3] = {ix, iy, iz};
  T f8[8];
  face_flux_at<T>((const T*)a.fbuf + P.off, P, row[2], row[3], dt, idx, gamma, f8, rc_floors(a));
#pragma unroll
  for (int n = 0; n < 5; ++n) a.creg[r * 6 + n] = dt * (double)f8[n];
}

template <class T>
__device__ __forceinline__ void regrc_coarse_edges_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[1]];
  const double dt = *a.dtp * a.dtscale;
  const double idx[3] = {ix, iy, iz};
  a.ecreg[r] = dt * (double)edge_emf_at<T>((const T*)a.fbuf + P.off, P, row[2], row[3], dt, idx, gamma, rc_floors(a));
}

template <class T>
__device__ __forceinline__ void regrc_fine_faces_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[5]];
  const int d = row[2], L = row[6];
  const double dt = *a.dtp * a.dtscale;
  const double idx[3] = {ix, iy, iz};
  const double af = dt * 0.25;
  const int sx = 1, sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  int o1, o2;
  if (d == 0) { o1 = sy; o2 = sz; }
  else if (d == 1) { o1 = sx; o2 = sz; }
  else { o1 = sx; o2 = sy; }
  const int off[4] = {0, o1, o2, o1 + o2};
  T f[4][8];
  const T* U = (const T*)a.fbuf + P.off;
  for (int k = 0; k < 4; ++k) face_flux_at<T>(U, P, d, L + off[k], dt, idx, gamma, f[k], rc_floors(a));
  double* out = a.freg + (r * 2 + (a.substep - 1)) * 6;
#pragma unroll
  for (int n = 0; n < 5; ++n)
    out[n] = af * tree4((double)f[0][n], (double)f[1][n], (double)f[2][n], (double)f[3][n]);
}

template <class T>
__device__ __forceinline__ void regrc_fine_edges_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[4]];
  const int c = row[2], L = row[5];
  const double dt = *a.dtp * a.dtscale;
  const double idx[3] = {ix, iy, iz};
  const int sc = c == 0 ? 1 : (c == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
  const T* U = (const T*)a.fbuf + P.off;
  const T e0 = edge_emf_at<T>(U, P, c, L, dt, idx, gamma, rc_floors(a));
  const T e1 = edge_emf_at<T>(U, P, c, L + sc, dt, idx, gamma, rc_floors(a));
  a.efreg[r * 2 + (a.substep - 1)] = (dt * 0.5) * tree2((double)e0, (double)e1);
}

// fine-side registers from the boundary capture of the fine level's fused
// advance (the same fluxes and EMFs the recompute kernels above evaluate); a
// face or edge off the boundary planes (none by construction) is recomputed
template <class T>
__device__ __forceinline__ void regcap_fine_faces_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 7 * r;
  const DPatch P = a.P[row[5]];
  const int d = row[2], L = row[6];
  const double dt = *a.dtp * a.dtscale;
  const double af = dt * 0.25;
  const int sx = 1, sy = P.ext[0], sz = P.ext[0] * P.ext[1];
  int o1, o2;
  if (d == 0) { o1 = sy; o2 = sz; }
  else if (d == 1) { o1 = sx; o2 = sz; }
  else { o1 = sx; o2 = sy; }
  const int off[4] = {0, o1, o2, o1 + o2};
  const T* b = (const T*)a.bnd + P.boff;
  const long long F = bnd_faces_total(P.n);
  T f[4][5];
  for (int k = 0; k < 4; ++k) {
    const int Lk = L + off[k];
    const int x = Lk % P.ext[0], y = (Lk / P.ext[0]) % P.ext[1], z = Lk / (P.ext[0] * P.ext[1]);
    const long long sl = P.boff >= 0 ? bnd_face_slot(P, d, x, y, z) : -1;
    if (sl >= 0) {
#pragma unroll
      for (int n = 0; n < 5; ++n) f[k][n] = b[n * F + sl];
    } else {
      const double idx[3] = {ix, iy, iz};
      T f8[8];
      face_flux_at<T>((const T*)a.fbuf + P.off, P, d, Lk, dt, idx, gamma, f8, rc_floors(a));
#pragma unroll
      for (int n = 0; n < 5; ++n) f[k][n] = f8[n];
    }
  }
  double* out = a.freg + (r * 2 + (a.substep - 1)) * 6;
#pragma unroll
  for (int n = 0; n < 5; ++n)
    out[n] = af * tree4((double)f[0][n], (double)f[1][n], (double)f[2][n], (double)f[3][n]);
}

template <class T>
__device__ __forceinline__ void regcap_fine_edges_row(const RowArgs& a, long long r, double gamma, double ix, double iy,
                                      double iz) {
  if (r >= a.nrows) return;
  const int* row = a.rows + 6 * r;
  const DPatch P = a.P[row[4]];
  const int c = row[2], L = row[5];
  const double dt = *a.dtp * a.dtscale;
  const int sc = c == 0 ? 1 : (c == 1 ? P.ext[0] : P.ext[0] * P.ext[1]);
  const T* b = (const T*)a.bnd + P.boff + 5 * bnd_faces_total(P.n);
  T ev[2];
  for (int k = 0; k < 2; ++k) {
    const int Lk = L + k * sc;
    const int x = Lk % P.ext[0], y = (Lk / P.ext[0]) % P.ext[1], z = Lk / (P.ext[0] * P.ext[1]);
    long long sl = -1;
    for (int e = 0; e < 3 && sl < 0 && P.boff >= 0; ++e)
      if (e != c) sl = bnd_edge_slot(P, c, e, x, y, z);
    if (sl >= 0) {
      ev[k] = b[sl];
    } else {
      const double idx[3] = {ix, iy, iz};
      ev[k] = edge_emf_at<T>((const T*)a.fbuf + P.off, P, c, Lk, dt, idx, gamma, rc_floors(a));
    }
  }
  a.efreg[r * 2 + (a.substep - 1)] = (dt * 0.5) * tree2((double)ev[0], (double)ev[1]);
}

// the face and the edge rows of one register side in one launch: blocks [0,
// nbf) take the face rows, the rest the edge rows (128 rows per block)
#define AMRK_REG_PAIR(NAME)                                                                          \
  template <class T>                                                                                 \
  __global__ void __launch_bounds__(128)                                                             \
      k_##NAME(RowArgs f, RowArgs e, unsigned nbf, double gamma, double ix, double iy, double iz) {  \
    if (blockIdx.x < nbf) NAME##_faces_row<T>(f, (long long)blockIdx.x * 128 + threadIdx.x, gamma, ix, iy, iz); \
    else NAME##_edges_row<T>(e, (long long)(blockIdx.x - nbf) * 128 + threadIdx.x, gamma, ix, iy, iz);  \
  }
AMRK_REG_PAIR(regrc_coarse)
AMRK_REG_PAIR(regrc_fine)
AMRK_REG_PAIR(regcap_fine)
#undef AMRK_REG_PAIR
