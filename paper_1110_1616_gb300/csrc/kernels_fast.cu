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
