// The regrid's clustering on the device (Sec. 2: the new grids of level l+1
// cover the flagged cells of level l): the flag test writes the level's cells
// and its flagged cells as bytes of the clustering frame (the region's
// bounding box, or the whole level extent), the flags are buffered by 2 cells
// (dilated along x, then y, then z, with the periodic wrap where the frame
// spans the domain), and one thread per 4^dim block marks the blocks that hold
// a buffered flag inside the region and whose 3-cell surroundings lie in the
// region (proper nesting). Only the block marks come back to the host, where
// the greedy z,y,x merge of the host clustering (regrid.cpp, merge_blocks)
// turns them into boxes: the same boxes, in the same order, as the host path
// gives for the same flags.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "ctx.hpp"
#include "regrid.hpp"

namespace amrcl {

struct Frame {
  int dim;
  int off[3], n[3], full[3], nb[3];
  int per[3];
  int N[3];  // the level's extent
};

// dst = src dilated by 2 cells along dimension d (wrapping if wrap): one
// block per row of the frame (y, z), each thread 4 consecutive x (the frame's
// x extent is a multiple of the 4-cell block)
__global__ void k_dilate(const unsigned char* src, unsigned char* dst, Frame f, int d, int wrap) {
  const int row = blockIdx.x;
  const int y = row % f.n[1], z = row / f.n[1];
  const int n0 = f.n[0];
  const unsigned char* srow = src + (long long)row * n0;
  unsigned char* drow = dst + (long long)row * n0;
  for (int x = 4 * threadIdx.x; x < n0; x += 4 * blockDim.x) {
    uchar4 v;
    if (d == 0) {
      unsigned char w[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        int q = x - 2 + o;
        if (wrap) q = q < 0 ? q + n0 : (q >= n0 ? q - n0 : q);
        w[o] = (q >= 0 && q < n0) ? srow[q] : 0;
      }
      v.x = w[0] | w[1] | w[2] | w[3] | w[4];
      v.y = w[1] | w[2] | w[3] | w[4] | w[5];
      v.z = w[2] | w[3] | w[4] | w[5] | w[6];
      v.w = w[3] | w[4] | w[5] | w[6] | w[7];
    } else {
      const int c = d == 1 ? y : z, n = f.n[d];
      const long long st = d == 1 ? (long long)n0 : (long long)n0 * f.n[1];
      unsigned int acc = 0;
      for (int o = -2; o <= 2; ++o) {
        int q = c + o;
        if (wrap) q = q < 0 ? q + n : (q >= n ? q - n : q);
        else if (q < 0 || q >= n) continue;
        acc |= *(const unsigned int*)(srow + (long long)(q - c) * st + x);
      }
      v = *(const uchar4*)&acc;
    }
    *(uchar4*)(drow + x) = v;
  }
}

// one warp per 4^dim block: the block holds a buffered flag inside the region
// (want) and every cell within 3 of it lies in the region (proper nesting)
__global__ void k_blocks(const unsigned char* buf, const unsigned char* region, unsigned char* ok, Frame f) {
  const long long nblk = (long long)f.nb[0] * f.nb[1] * f.nb[2];
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nblk) return;  // the whole warp
  const int a = (int)(w % f.nb[0]), b = (int)((w / f.nb[0]) % f.nb[1]), c = (int)(w / ((long long)f.nb[0] * f.nb[1]));
  const int kz = f.dim == 3 ? 1 : 0;
  const int lo[3] = {4 * a, 4 * b, f.dim == 3 ? 4 * c : 0};
  auto at = [&](int i, int j, int k) { return ((long long)k * f.n[1] + j) * f.n[0] + i; };
  // want: 64 cells (16 in 2D), two per lane
  bool want = false;
  const int ncell = f.dim == 3 ? 64 : 16;
  for (int p = lane; p < ncell; p += 32) {
    const long long x = at(lo[0] + (p & 3), lo[1] + ((p >> 2) & 3), lo[2] + (p >> 4));
    want = want || (buf[x] & region[x]) != 0;
  }
  if (!__any_sync(0xffffffffu, want)) {
    if (lane == 0) ok[w] = 0;
    return;
  }
  // the surroundings: per dimension the 10 coordinates (wrapped where the frame
  // spans a periodic dimension), -1 outside a bounded side (skipped), -2
  // outside the frame's box (not in the region)
  const int ext = 10;
  auto coord = [&](int e, int i) {
    int q = lo[e] - 3 + i;
    if (f.full[e]) {
      if (f.per[e]) return (q % f.N[e] + f.N[e]) % f.N[e];
      return (q < 0 || q >= f.n[e]) ? -1 : q;
    }
    const int g = q + f.off[e];
    if (!f.per[e] && (g < 0 || g >= f.N[e])) return -1;
    return (q < 0 || q >= f.n[e]) ? -2 : q;
  };
  const int nz = kz ? ext : 1, tot = ext * ext * nz;
  bool allowed = true;
  for (int p = lane; p < tot && allowed; p += 32) {
    const int i = p % ext, j = (p / ext) % ext, k = p / (ext * ext);
    const int x = coord(0, i), y = coord(1, j), z = kz ? coord(2, k) : 0;
    if (x == -1 || y == -1 || z == -1) continue;
    if (x == -2 || y == -2 || z == -2 || !region[at(x, y, z)]) allowed = false;
  }
  allowed = __all_sync(0xffffffffu, allowed);
  if (lane == 0) ok[w] = allowed ? 1 : 0;
}

}  // namespace amrcl

namespace amrapi {

// New level-(l+1) boxes from the flagged cells of level l of context c (its
// ghosts filled), clustered on the device; ctx holds the scratch and errors.
amrmhd_status cluster_level_device(amrmhd_ctx* ctx, amrmhd_ctx* c, int l, double theta,
                                   std::vector<std::array<int, 7>>& boxes) {
  using namespace amrcl;
  const auto t0 = std::chrono::steady_clock::now();
  const amrmhd::Hierarchy& H = c->H;
  const amrmhd::ClusterFrame fr = amrmhd::cluster_frame(H, l);
  Frame f;
  f.dim = H.dim;
  for (int d = 0; d < 3; ++d) {
    f.off[d] = fr.off[d];
    f.n[d] = fr.n[d];
    f.full[d] = fr.full[d];
    f.nb[d] = fr.nb[d];
    f.per[d] = H.per[d] ? 1 : 0;
    f.N[d] = H.N(l, d);
  }
  const size_t ncell = (size_t)f.n[0] * f.n[1] * f.n[2], nblk = (size_t)f.nb[0] * f.nb[1] * f.nb[2];
  const size_t need = 3 * ncell + nblk + 256;
  if (ctx->cluster_cap < need) {
    if (ctx->d_cluster) cudaFree(ctx->d_cluster);
    ctx->d_cluster = nullptr;
    ctx->cluster_cap = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->d_cluster, need);
    if (e != cudaSuccess) {
      ctx->d_cluster = nullptr;
      return fail(ctx, AMRMHD_ENOMEM, std::string("regrid: cluster scratch: ") + cudaGetErrorString(e));
    }
    ctx->cluster_cap = need;
  }
  unsigned char* region = ctx->d_cluster;
  unsigned char* buf = region + ncell;
  unsigned char* tmp = buf + ncell;
  unsigned char* ok = tmp + ncell;
  cudaStream_t st = c->stream;
  const bool tr = std::getenv("AMRMHD_REGRID_TRACE") != nullptr;
  long long wait_prior = 0;
  cudaEvent_t ev[5];
  if (tr) {  // the work queued before (fills) first, then events between the steps
    const auto w0 = std::chrono::steady_clock::now();
    cudaStreamSynchronize(st);
    wait_prior = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - w0).count();
    for (auto& x : ev) cudaEventCreate(&x);
    cudaEventRecord(ev[0], st);
  }
  cudaError_t e = cudaMemsetAsync(region, 0, 2 * ncell, st);
  if (e != cudaSuccess) return fail(ctx, AMRMHD_ECUDA, std::string("regrid: ") + cudaGetErrorString(e));
  amrk::LevelArgs a = level_args(c, l, c->d_scal, 1.0, 0);
  amrk::DenseBox box;
  for (int d = 0; d < 3; ++d) { box.off[d] = f.off[d]; box.n[d] = f.n[d]; }
  if (tr) cudaEventRecord(ev[1], st);
  c->ops->flag_dense(a, theta, region, buf, box, st);
  if (tr) cudaEventRecord(ev[2], st);
  const int T = 256;
  unsigned char *src = buf, *dst = tmp;
  for (int d = 0; d < f.dim; ++d) {
    k_dilate<<<(unsigned)(f.n[1] * f.n[2]), 128, 0, st>>>(src, dst, f, d, f.full[d] && f.per[d]);
    std::swap(src, dst);
  }
  if (tr) cudaEventRecord(ev[3], st);
  k_blocks<<<(unsigned)((32 * nblk + T - 1) / T), T, 0, st>>>(src, region, ok, f);
  if (tr) cudaEventRecord(ev[4], st);
  ctx->launches += 2 + f.dim;
  std::vector<uint8_t> h(nblk + 8, 0);
  const auto t1 = std::chrono::steady_clock::now();
  e = cudaMemcpyAsync(h.data(), ok, nblk, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, AMRMHD_ECUDA, std::string("regrid: clustering: ") + cudaGetErrorString(e));
  const auto t2 = std::chrono::steady_clock::now();
  boxes = amrmhd::merge_blocks(H, l, fr, h.data());
  if (std::getenv("AMRMHD_REGRID_TRACE")) {
    auto us = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return (long long)std::chrono::duration_cast<std::chrono::microseconds>(b - a).count();
    };
    float m[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&m[i], ev[i], ev[i + 1]);
    for (auto& x : ev) cudaEventDestroy(x);
    std::fprintf(stderr, "amrmhd cluster level %d: frame %d x %d x %d, prior work %lld us, enqueue %lld us, device and "
                 "copy %lld us (memset %.0f, flag %.0f, dilate %.0f, blocks %.0f us), merge %lld us\n", l, f.n[0],
                 f.n[1], f.n[2], wait_prior, us(t0, t1), us(t1, t2), 1e3 * m[0], 1e3 * m[1], 1e3 * m[2], 1e3 * m[3],
                 us(t2, std::chrono::steady_clock::now()));
  }
  return AMRMHD_OK;
}

}  // namespace amrapi
