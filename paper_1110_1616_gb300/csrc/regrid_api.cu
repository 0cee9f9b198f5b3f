// C-ABI of the regrid (amrmhd_regrid, amrmhd_get_patches): every level above 0
// is rebuilt coarse to fine. Each stage is a context holding the levels built
// so far plus the new level: its coarser levels are copied from the previous
// stage, the new level is transferred from the old hierarchy (copy where the
// old fine level covered the parent cell, else prolongation, then the
// divergence-free closure), its ghosts are filled and its cells flagged for
// the next stage. The last stage's hierarchy and arena replace the context's.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "ctx.hpp"
#include "regrid.hpp"

using namespace amrapi;

namespace {

// AMRMHD_REGRID_TRACE set in the environment: per-stage host timings on stderr
bool trace() {
  static const bool on = std::getenv("AMRMHD_REGRID_TRACE") != nullptr;
  return on;
}

long long now_us() {
  return std::chrono::duration_cast<std::chrono::microseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define CUR(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, AMRMHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// flagged cells of level l of context c (ghosts of l filled): host triples
amrmhd_status flag_level(amrmhd_ctx* ctx, amrmhd_ctx* c, int l, double theta, std::vector<int32_t>& out) {
  long long cap = 1 << 16;
  for (int attempt = 0; attempt < 8; ++attempt) {
    int* d_out = nullptr;
    unsigned long long* d_cnt = nullptr;
    CUR(cudaMalloc((void**)&d_out, sizeof(int) * 3 * cap));
    CUR(cudaMalloc((void**)&d_cnt, sizeof(unsigned long long)));
    CUR(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), c->stream));
    amrk::LevelArgs a = level_args(c, l, c->d_scal, 1.0, 0);
    c->ops->flag(a, theta, d_out, d_cnt, cap, c->stream);
    unsigned long long n = 0;
    CUR(cudaMemcpyAsync(&n, d_cnt, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CUR(cudaStreamSynchronize(c->stream));
    if ((long long)n <= cap) {
      out.resize(3 * n);
      if (n) CUR(cudaMemcpy(out.data(), d_out, sizeof(int) * 3 * n, cudaMemcpyDeviceToHost));
      cudaFree(d_out);
      cudaFree(d_cnt);
      return AMRMHD_OK;
    }
    cudaFree(d_out);
    cudaFree(d_cnt);
    cap = (long long)n;
  }
  return fail(ctx, AMRMHD_ENOMEM, "flag list did not fit");
}

// a stage context with the given patches, a library-owned arena and the
// option settings of ctx; a light stage (ghost_from >= 0) has the fill maps of
// the levels from ghost_from on only, no register maps and no scratch
amrmhd_status make_stage(amrmhd_ctx* ctx, const std::vector<amrmhd_patch>& ps, int ghost_from, amrmhd_ctx** out,
                         long long* maps_us) {
  amrmhd_ctx* c = nullptr;
  amrmhd_status st = amrmhd_create(&ctx->cfg, ctx->stream, &c);
  if (st) return fail(ctx, st, "regrid: create");
  c->stage_light = ghost_from >= 0;
  c->stage_ghost_from = std::max(ghost_from, 0);
  c->opt_advance = ctx->opt_advance;
  c->opt_graph = ctx->opt_graph;
  c->opt_tile = ctx->opt_tile;
  c->opt_concurrent = ctx->opt_concurrent;
  c->opt_device_maps = ctx->opt_device_maps;
  c->opt_device_cluster = ctx->opt_device_cluster;
  size_t bytes = 0;
  const long long t0 = now_us();
  st = amrmhd_set_hierarchy(c, ps.data(), (int32_t)ps.size(), &bytes);
  *maps_us += now_us() - t0;
  if (st) {
    std::string m = c->err;
    amrmhd_destroy(c);
    return fail(ctx, st, "regrid: new hierarchy rejected: " + m);
  }
  void* mem = nullptr;
  const long long t1 = now_us();
  cudaError_t e = cudaMalloc(&mem, std::max<size_t>(bytes, 256));
  if (e != cudaSuccess) {
    amrmhd_destroy(c);
    return fail(ctx, AMRMHD_ENOMEM, std::string("regrid: arena: ") + cudaGetErrorString(e));
  }
  const long long t2 = now_us();
  st = amrmhd_bind_arena(c, mem, bytes);
  c->dev_allocs.push_back(mem);
  if (trace())
    std::fprintf(stderr, "amrmhd regrid stage (%zu patches, ghosts from level %d): set_hierarchy %lld us (host %lld, "
                 "ghost boxes %lld, register maps %lld), arena %.1f MB %lld us, bind %lld us\n",
                 ps.size(), ghost_from, t1 - t0, c->maps_us[0], c->maps_us[1], c->maps_us[2], bytes / 1e6, t2 - t1,
                 now_us() - t2);
  if (st) {
    std::string m = c->err;
    amrmhd_destroy(c);
    return fail(ctx, st, "regrid: bind: " + m);
  }
  *out = c;
  return AMRMHD_OK;
}

// levels 0..l of src (same patches, same order) into buffer 0 of dst
amrmhd_status copy_levels(amrmhd_ctx* ctx, amrmhd_ctx* src, amrmhd_ctx* dst, int l) {
  const size_t elem = dst->ops->elem;
  for (int q = 0; q <= l; ++q) {
    const std::vector<int>& ids = dst->H.level_patches[q];
    const long long b = dst->off[ids.front()];
    const long long e = dst->off[ids.back()] + 8 * dst->fs[ids.back()];
    if (src->off[src->H.level_patches[q].front()] != b) return fail(ctx, AMRMHD_EINVAL, "regrid: layout mismatch");
    CUR(cudaMemcpyAsync((char*)state_buf(dst, 0) + b * elem, (char*)state_buf(src, src->cur[q]) + b * elem,
                        (size_t)(e - b) * elem, cudaMemcpyDeviceToDevice, dst->stream));
    dst->cur[q] = 0;
  }
  return AMRMHD_OK;
}

// transfer of level lf of stage S from the old context O
amrmhd_status transfer(amrmhd_ctx* ctx, amrmhd_ctx* S, amrmhd_ctx* O, int lf, long long* maps_us) {
  amrmhd::TransferMaps m;
  // cell and face boxes with their chunks (box, first position) of at most FILL_CHUNK positions
  std::vector<int32_t> cb, cc, fb, fc;
  const long long t0 = now_us();
  if (ctx->opt_device_maps != 0) {
    amrmhd_status ds = device_transfer_maps(ctx, S->H, O->H, lf, S->stream, cb, fb, m.closure);
    *maps_us += now_us() - t0;
    if (ds != AMRMHD_OK) return ds;
  } else {
    const int rc = amrmhd::transfer_maps(S->H, O->H, lf, m);
    *maps_us += now_us() - t0;
    if (rc) return fail(ctx, AMRMHD_EINVAL, "regrid: transfer map without a source");
    for (size_t r = 0; r < m.boxes.size(); r += amrmhd::GHOST_BOX_W) {
      const int32_t* b = &m.boxes[r];
      std::vector<int32_t>& boxes = b[1] < 0 ? cb : fb;
      boxes.insert(boxes.end(), b, b + amrmhd::GHOST_BOX_W);
    }
  }
  const long long t1 = now_us();
  for (int k = 0; k < 2; ++k) {
    const std::vector<int32_t>& boxes = k ? fb : cb;
    std::vector<int32_t>& ch = k ? fc : cc;
    for (size_t r = 0; r < boxes.size(); r += amrmhd::GHOST_BOX_W) {
      const int32_t* b = &boxes[r];
      const int bi = (int)(r / amrmhd::GHOST_BOX_W);
      for (int c = 0; c < b[7] * b[8] * b[9]; c += amrk::FILL_CHUNK) {
        ch.push_back(bi);
        ch.push_back(c);
      }
    }
  }
  // the five lists and the closure matrix in one device block, one copy
  double idx[3], K[96] = {0};
  level_idx(S, lf, idx);
  amrmhd::closure_matrix(S->cfg.dim, idx, K);
  std::vector<char> img;
  auto put = [&](const void* src, size_t bytes) {
    const size_t o = (img.size() + 255) / 256 * 256;
    img.resize(o + bytes);
    if (bytes) std::memcpy(img.data() + o, src, bytes);
    return o;
  };
  const size_t oK = put(K, sizeof(K)), ocb = put(cb.data(), sizeof(int32_t) * cb.size()),
               occ = put(cc.data(), sizeof(int32_t) * cc.size()), ofb = put(fb.data(), sizeof(int32_t) * fb.size()),
               ofc = put(fc.data(), sizeof(int32_t) * fc.size()),
               ok = put(m.closure.data(), sizeof(int32_t) * m.closure.size());
  char* dev = nullptr;
  amrmhd_status st = AMRMHD_OK;
  cudaError_t e0 = cudaMallocAsync((void**)&dev, img.size(), S->stream);
  if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(dev, img.data(), img.size(), cudaMemcpyHostToDevice, S->stream);
  if (e0 != cudaSuccess) {
    if (dev) cudaFreeAsync(dev, S->stream);
    return fail(ctx, AMRMHD_ECUDA, std::string("regrid: transfer lists: ") + cudaGetErrorString(e0));
  }
  int *dcb = (int*)(dev + ocb), *dcc = (int*)(dev + occ), *dfb = (int*)(dev + ofb), *dfc = (int*)(dev + ofc),
      *dk = (int*)(dev + ok);
  double* dK = (double*)(dev + oK);
  if (!st) {
    amrk::RowArgs a = row_args(S, DevList{dcb, (int64_t)cb.size() / amrmhd::GHOST_BOX_W}, lf - 1);
    a.fbuf = state_buf(S, S->cur[lf]);
    a.cbuf = state_buf(S, S->cur[lf - 1]);
    a.P2 = O->dP;
    a.obuf = O->H.nlev > lf ? state_buf(O, O->cur[lf]) : nullptr;
    int nl = 0;
    a.chunks = dcc;
    a.nrows = (int64_t)cc.size() / 2;
    S->ops->transfer_cells(a, S->stream, &nl);
    a.rows = dfb;
    a.chunks = dfc;
    a.nrows = (int64_t)fc.size() / 2;
    S->ops->transfer_faces(a, S->stream, &nl);
    a.rows = dk;
    a.chunks = nullptr;
    a.nrows = (int64_t)m.closure.size() / 2;
    for (int d = 0; d < 3; ++d) a.idx[d] = idx[d];
    a.K = dK;
    S->ops->closure(a, S->stream, &nl);
    cudaError_t e = cudaStreamSynchronize(S->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(ctx, AMRMHD_ECUDA, std::string("regrid: transfer: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(dev, S->stream);
  if (trace())
    std::fprintf(stderr, "amrmhd regrid transfer level %d: maps %lld us (%zu cell, %zu face boxes, %zu closure rows), "
                 "lists, kernels and sync %lld us\n", lf, t1 - t0, cb.size() / amrmhd::GHOST_BOX_W,
                 fb.size() / amrmhd::GHOST_BOX_W, m.closure.size() / 2, now_us() - t1);
  return st;
}

}  // namespace

extern "C" {

amrmhd_status amrmhd_regrid(amrmhd_ctx* ctx, double theta, int32_t max_levels) {
  amrmhd_status st = check_bound(ctx);
  if (st) return st;
  if (max_levels < 1 || max_levels > ctx->cfg.max_level + 1) return fail(ctx, AMRMHD_EINVAL, "bad max_levels");
  for (int d = 0; d < ctx->cfg.dim; ++d)
    if (ctx->cfg.base[d] % 4) return fail(ctx, AMRMHD_EINVAL, "regrid needs base sizes divisible by 4");
  std::vector<amrmhd_patch> ps;
  for (int q : ctx->H.level_patches[0]) {
    amrmhd_patch p;
    p.level = 0;
    for (int d = 0; d < 3; ++d) { p.lo[d] = ctx->H.p[q].lo[d]; p.hi[d] = ctx->H.p[q].hi[d]; }
    ps.push_back(p);
  }
  long long us[6] = {0, 0, 0, 0, 0, 0}, t0 = now_us();
  // the new level-(l+1) boxes from level l of context c (ghosts filled): the
  // flags on the device, clustered on the device (the block marks merged on the
  // host) or on the host (the flag list copied back)
  std::vector<std::array<int, 7>> boxes;
  auto cluster = [&](amrmhd_ctx* c, int l) -> amrmhd_status {
    long long t = now_us();
    if (ctx->opt_device_cluster) {
      amrmhd_status s = cluster_level_device(ctx, c, l, theta, boxes);
      us[1] += now_us() - t;
      if (trace())
        std::fprintf(stderr, "amrmhd regrid cluster level %d: %lld us, %zu boxes\n", l, now_us() - t, boxes.size());
      return s;
    }
    std::vector<int32_t> flags;
    amrmhd_status s = flag_level(ctx, c, l, theta, flags);
    us[0] += now_us() - t;
    if (s) return s;
    t = now_us();
    boxes = amrmhd::regrid_boxes(c->H, l, flags);
    us[1] += now_us() - t;
    return AMRMHD_OK;
  };
  // level 0 of the old context: fill and cluster
  int nl = 0;
  op_fill(ctx, 0, 1, &nl);
  us[0] += now_us() - t0;
  st = cluster(ctx, 0);
  if (st) return st;
  amrmhd_ctx* prev = ctx;
  for (int l = 0; l + 1 < max_levels; ++l) {
    if (boxes.empty()) break;
    std::vector<amrmhd_patch> next = ps;
    for (const auto& b : boxes) {
      amrmhd_patch p;
      p.level = b[0];
      for (int d = 0; d < 3; ++d) { p.lo[d] = b[1 + d]; p.hi[d] = b[4 + d]; }
      next.push_back(p);
    }
    // a light stage: levels 0..l as in prev (copied with their filled ghosts),
    // the new level l+1 transferred, filled and flagged
    amrmhd_ctx* S = nullptr;
    t0 = now_us();
    st = make_stage(ctx, next, l + 1, &S, &us[4]);
    us[2] += now_us() - t0;
    t0 = now_us();
    if (!st) st = copy_levels(ctx, prev, S, l);
    if (!st) st = transfer(ctx, S, ctx, l + 1, &us[5]);
    us[3] += now_us() - t0;
    if (!st) {
      t0 = now_us();
      op_fill(S, l + 1, 1, &nl);
      us[0] += now_us() - t0;
      boxes.clear();
      if (l + 2 < max_levels) st = cluster(S, l + 1);
    }
    if (st) {
      if (S) amrmhd_destroy(S);
      if (prev != ctx) amrmhd_destroy(prev);
      return st;
    }
    if (prev != ctx) amrmhd_destroy(prev);
    prev = S;
    ps = next;
  }
  {
    // the final context: the whole hierarchy with all its maps, every level's
    // data (with filled ghosts) from the last stage
    amrmhd_ctx* S = nullptr;
    t0 = now_us();
    st = make_stage(ctx, ps, -1, &S, &us[4]);
    us[2] += now_us() - t0;
    t0 = now_us();
    const int top = (int)S->H.nlev - 1;
    if (!st) st = copy_levels(ctx, prev, S, top);
    us[3] += now_us() - t0;
    if (st) {
      if (S) amrmhd_destroy(S);
      if (prev != ctx) amrmhd_destroy(prev);
      return st;
    }
    if (prev != ctx) amrmhd_destroy(prev);
    prev = S;
  }
  CUR(cudaStreamSynchronize(ctx->stream));
  // the context takes the last stage's hierarchy and arena; the stage object
  // then holds (and frees) the old ones
  std::swap(*ctx, *prev);
  std::swap(ctx->own_stream, prev->own_stream);
  std::swap(ctx->d_cluster, prev->d_cluster);
  std::swap(ctx->cluster_cap, prev->cluster_cap);
  ctx->launches += prev->launches;
  amrmhd_destroy(prev);
  for (int i = 0; i < 6; ++i) ctx->regrid_us[i] = us[i];
  return AMRMHD_OK;
}

amrmhd_status amrmhd_regrid_boxes(amrmhd_ctx* ctx, int32_t level, const int32_t* flags, int64_t nflags,
                                  int32_t* out, int32_t cap, int32_t* n) {
  if (!ctx || !n || nflags < 0 || (nflags && !flags)) return AMRMHD_EINVAL;
  if (!ctx->have_h) return fail(ctx, AMRMHD_ESTATE, "no hierarchy set");
  if (level < 0 || level >= ctx->H.nlev) return fail(ctx, AMRMHD_EINVAL, "bad level");
  std::vector<int32_t> f;
  f.reserve(3 * (size_t)nflags);
  const amrmhd::Hierarchy& H = ctx->H;
  for (int64_t i = 0; i < nflags; ++i) {
    const int32_t* c = flags + 3 * i;
    bool inside = true;
    for (int d = 0; d < H.dim; ++d)
      if (c[d] < 0 || c[d] >= H.N(level, d)) inside = false;
    if (!inside) continue;
    bool in_region = false;
    for (int q : H.level_patches[level]) {
      const amrmhd::HPatch& P = H.p[q];
      bool in = true;
      for (int d = 0; d < H.dim; ++d)
        if (c[d] < P.lo[d] || c[d] >= P.hi[d]) in = false;
      if (in) { in_region = true; break; }
    }
    if (in_region) f.insert(f.end(), c, c + 3);
  }
  std::vector<std::array<int, 7>> b = amrmhd::regrid_boxes(H, level, f);
  *n = (int32_t)b.size();
  if (!out) return AMRMHD_OK;
  if (cap < *n) return fail(ctx, AMRMHD_EINVAL, "box buffer too small");
  for (size_t i = 0; i < b.size(); ++i)
    for (int k = 0; k < 7; ++k) out[7 * i + k] = b[i][k];
  return AMRMHD_OK;
}

amrmhd_status amrmhd_get_patches(amrmhd_ctx* ctx, amrmhd_patch* out, int32_t cap, int32_t* n) {
  if (!ctx || !n) return AMRMHD_EINVAL;
  if (!ctx->have_h) return fail(ctx, AMRMHD_ESTATE, "no hierarchy set");
  const int np = (int)ctx->H.p.size();
  *n = np;
  if (!out) return AMRMHD_OK;
  if (cap < np) return fail(ctx, AMRMHD_EINVAL, "patch buffer too small");
  for (int q = 0; q < np; ++q) {
    out[q].level = ctx->H.p[q].level;
    for (int d = 0; d < 3; ++d) { out[q].lo[d] = ctx->H.p[q].lo[d]; out[q].hi[d] = ctx->H.p[q].hi[d]; }
  }
  return AMRMHD_OK;
}

}  // extern "C"
