// amrmhd_advance_patch_noalloc: the staged level advance of ONE patch in the
// mixed-precision path (FP32 stencil, FP64 primitive recovery), for callers
// that must not allocate device memory. Its intermediate arrays live in a
// fixed, file-scope device array instead of a caller-bound arena.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not safe,
// for example inside a framework step whose memory pool forbids new device
// allocations, a real-time loop that must not hit the allocator's
// synchronisation, or a host library that only receives pointers to the state
// it may read and write. Such a caller passes its input and output state and
// nothing else.
//
// The array below is held by every GPU that loads this library until the
// process exits. All calls on a device share it and it keeps the last call's
// contents; every entry the kernels read is written earlier in the same call,
// so nothing needs clearing. Calls that overlap on the GPU (different streams,
// or several host threads) race on the array: serialise them.
#include <mutex>

#define AMRK_NS amrk_noalloc
#include "../../include/amrmhd.h"
#include "kernels_impl.cuh"

namespace {

constexpr long long kMaxFieldElems = 16384;  // per field: (nx+9)(ny+9)(nz+9) at most
constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)amrk::SC_N * kMaxFieldElems * sizeof(float);

// Header (patch descriptor, id, dt) followed by the 70 scratch fields.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Header {
  amrk::DPatch P;
  int id;
  int pad;
  double dt;
};
static_assert(sizeof(Header) <= kHeaderBytes, "header does not fit");

__global__ void k_write_header(Header h, Header* dst) { *dst = h; }

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" amrmhd_status amrmhd_advance_patch_noalloc(const float* u_in, float* u_out, int32_t dim, const int32_t* n,
                                                      const double* dx, double gamma, double dt, int32_t w,
                                                      void* cuda_stream) {
  if (!u_in || !u_out || !n || !dx || (dim != 2 && dim != 3) || (w != 0 && w != 2)) return AMRMHD_EINVAL;
  if (!(gamma > 1.0) || !(dt >= 0.0)) return AMRMHD_EINVAL;
  long long fs = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1 || !(dx[d] > 0.0)) return AMRMHD_EINVAL;
    fs *= (long long)n[d] + 9;
  }
  if (fs > kMaxFieldElems) return AMRMHD_EINVAL;  // patch too large for the fixed array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMRMHD_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // once per device, with that device current: the device address of the array
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AMRMHD_ECUDA;
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Header h;
  for (int d = 0; d < 3; ++d) {
    h.P.lo[d] = 0;
    h.P.n[d] = d < dim ? n[d] : 1;
    h.P.ext[d] = d < dim ? n[d] + 9 : 1;
  }
  h.P.level = 0;
  h.P.off = 0;
  h.P.fs = fs;
  h.P.soff = 0;
  h.P.boff = -1;
  h.id = 0;
  h.pad = 0;
  h.dt = dt;
  Header* hd = (Header*)base;
  k_write_header<<<1, 1, 0, s>>>(h, hd);
  amrk::LevelArgs a;
  a.P = &hd->P;
  a.ids = &hd->id;
  a.npatch = 1;
  for (int d = 0; d < 3; ++d) a.maxn[d] = h.P.n[d];
  a.cur = (void*)u_in;
  a.nxt = (void*)u_out;
  a.scr = (unsigned char*)base + kHeaderBytes;
  a.dtp = &hd->dt;
  a.dtscale = 1.0;
  for (int d = 0; d < 3; ++d) a.idx[d] = d < dim ? 1.0 / dx[d] : 1.0;
  a.gamma = gamma;
  a.bnd = nullptr;
  a.nbr = nullptr;
  a.w = w;
  a.zlen = 0;
  a.tail = 0;
  if (dim == 3) amrk_noalloc::Impl<float, 3>::advance(a, s, nullptr);
  else amrk_noalloc::Impl<float, 2>::advance(a, s, nullptr);
  if (cudaGetLastError() != cudaSuccess) return AMRMHD_ECUDA;
  return AMRMHD_OK;
}
