// FP64 (FMA contraction allowed) and mixed-precision instantiations of the
// kernels, plus the small scalar kernels.
#define AMRK_NS amrk_fast
#include "kernels_impl.cuh"

namespace amrk {

const Ops* ops_fast(int variant, int dim) {
  if (variant == V_MIXED) return dim == 3 ? amrk_fast::Impl<float, 3>::ops() : amrk_fast::Impl<float, 2>::ops();
  return dim == 3 ? amrk_fast::Impl<double, 3>::ops() : amrk_fast::Impl<double, 2>::ops();
}

// the bit-level conversions of the mixed recovery next to the conversion
// instructions, compiled with this unit's flags (FP32 denormals flushed)
__global__ void k_fp_convert(long long n, const double* x, const float* y, float* xn, double* yw, float* xn_hw,
                             double* yw_hw) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  xn[i] = amrdev::narrow_bits(x[i]);
  yw[i] = amrdev::widen_bits(y[i]);
  xn_hw[i] = (float)x[i];
  yw_hw[i] = (double)y[i];
}

void launch_fp_convert(long long n, const double* x, const float* y, float* xn, double* yw, float* xn_hw,
                       double* yw_hw, cudaStream_t s) {
  k_fp_convert<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y, xn, yw, xn_hw, yw_hw);
}

// the mixed-precision recovery of one cell per thread, compiled with this
// unit's flags (the code the mixed advance runs): u (5 per cell), the low and
// high face values of B (3 + 3 per cell) -> w (8 per cell)
__global__ void k_recover_mixed(long long n, const float* u, const float* bl, const float* br, double gm1, float* w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float uu[5], l[3], r[3], wv[8];
#pragma unroll
  for (int f = 0; f < 5; ++f) uu[f] = u[5 * i + f];
#pragma unroll
  for (int c = 0; c < 3; ++c) { l[c] = bl[3 * i + c]; r[c] = br[3 * i + c]; }
  amrdev::recover_t(uu, l, r, gm1, wv);
#pragma unroll
  for (int f = 0; f < 8; ++f) w[8 * i + f] = wv[f];
}

void launch_recover_mixed(long long n, const float* u, const float* bl, const float* br, double gm1, float* w,
                          cudaStream_t s) {
  k_recover_mixed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, u, bl, br, gm1, w);
}

// ALU peak probe: every thread runs 8 independent multiply-add chains of
// `iters` steps (2 floating-point operations each); the sum of the chains is
// stored only if it takes an impossible value, so nothing is eliminated.
template <class T> __global__ void k_fma_peak(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == T(-1.2345e30)) out[blockIdx.x] = s;
}

void launch_fma_peak(int fp64, int blocks, int threads, int iters, void* out, cudaStream_t s) {
  if (fp64) k_fma_peak<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
  else k_fma_peak<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
}

// dL/dv of the initial velocity from dL/dU0 (reading 13): with rho, p and B
// held, m = rho v and E = p/(g-1) + rho |v|^2 / 2 + |B|^2 / 2, so
// dL/dv_c = rho (dL/dm_c + v_c dL/dE), v = m / rho; packed cell fields, field
// stride n (rho, mx, my, mz, E first in u and g), 3 fields out
__global__ void k_grad_velocity(long long n, const double* u, const double* g, double* gv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double rho = u[i], gE = g[4 * n + i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double v = u[(1 + c) * n + i] / rho;
    gv[c * n + i] = rho * (g[(1 + c) * n + i] + v * gE);
  }
}

void launch_grad_velocity(long long n, const double* u, const double* g, double* gv, cudaStream_t s) {
  k_grad_velocity<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, u, g, gv);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

void launch_set_scalar(double* p, double v, cudaStream_t s) { k_set_scalar<<<1, 1, 0, s>>>(p, v); }

__global__ void k_zero_u64(unsigned long long* p, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0ull;
}

void launch_zero_u64(unsigned long long* p, int n, cudaStream_t s) { k_zero_u64<<<(n + 127) / 128, 128, 0, s>>>(p, n); }

// dt0 = cfl / max_l (M_l 2^-l); the history slot is taken from a device counter
// kept after the per-level maxima (slots[nlev]).
__global__ void k_cfl_finalize(const unsigned long long* slots, int nlev, double cfl, double* dt_out, double* hist,
                               unsigned int* err) {
  double mmax = 0.0, scale = 1.0;
  for (int l = 0; l < nlev; ++l) {
    const double m = __longlong_as_double((long long)slots[l]) * scale;
    if (m > mmax) mmax = m;
    scale *= 0.5;
  }
  double dt = cfl / mmax;
  if (!(dt > 0.0) || !(dt < 1e300)) { atomicOr(err, 2u); dt = 0.0; }
  if (*err) dt = 0.0;
  *dt_out = dt;
  if (hist) {
    unsigned long long* ctr = (unsigned long long*)(slots + nlev);
    hist[*ctr] = dt;
    *ctr += 1;
  }
}

void launch_cfl_finalize(const unsigned long long* slots, int nlev, double cfl, double* dt_out, double* hist,
                         unsigned int* err, cudaStream_t s) {
  k_cfl_finalize<<<1, 1, 0, s>>>(slots, nlev, cfl, dt_out, hist, err);
}

}  // namespace amrk
