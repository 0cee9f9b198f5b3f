// Conversions between IEEE-754 binary32 and binary64 done with integer
// operations on the bit patterns, from the two formats' definitions (sign,
// biased exponent, fraction; binary32 bias 127, binary64 bias 1023).
//
// On this part the FP64 pipe runs at a small fraction of the FP32 rate and the
// hardware conversions to and from binary64 issue on it, so the mixed path's
// FP64 energy balance spends more FP64 issue slots on converting its three
// FP32 inputs and its FP32 result than on the subtraction itself. These
// routines move the conversions to the integer pipe; the FP64 arithmetic
// (the subtraction and the scaling by gamma - 1) stays in FP64.
//
// Flush-to-zero semantics, as the mixed path is compiled with FP32 denormals
// flushed: a binary32 subnormal input converts to a signed zero, and a
// binary64 value below the smallest binary32 normal, 2^-126, converts to a
// signed zero. Otherwise both are exact IEEE
// conversions: widening is exact, narrowing rounds to nearest, ties to even,
// overflows to infinity, and keeps infinities and NaNs (NaNs made quiet).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace amrdev {

__host__ __device__ __forceinline__ uint32_t f32_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float f32_from(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ double f64_from(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double d;
  std::memcpy(&d, &b, 8);
  return d;
#endif
}
__host__ __device__ __forceinline__ void f64_split(double d, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
  hi = (uint32_t)__double2hiint(d);
  lo = (uint32_t)__double2loint(d);
#else
  uint64_t b;
  std::memcpy(&b, &d, 8);
  hi = (uint32_t)(b >> 32);
  lo = (uint32_t)b;
#endif
}

// binary32 -> binary64: the 8-bit exponent re-biased by 1023 - 127 = 896
// (255, infinity / NaN, maps to 2047), the 23 fraction bits placed at the top
// of the 52.
__host__ __device__ __forceinline__ double widen_bits(float f) {
  const uint32_t u = f32_bits(f);
  const uint32_t s = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t rebias = e == 255u ? 0x70000000u : 0x38000000u;  // 1792 or 896, at bit 20
  const uint32_t hi = e == 0u ? s : (s | (((u & 0x7fffffffu) >> 3) + rebias));
  const uint32_t lo = e == 0u ? 0u : (u << 29);
  return f64_from(hi, lo);
}

// binary64 -> binary32, round to nearest even: the 52-bit fraction cut to its
// top 23 bits, the 29 dropped bits deciding the rounding; a carry out of the
// fraction increments the exponent (and reaches infinity from the largest
// finite value), as the rounding definition requires.
__host__ __device__ __forceinline__ float narrow_bits(double d) {
  uint32_t hi, lo;
  f64_split(d, hi, lo);
  const uint32_t s = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  if (E == 0x7ff) {
    const bool nan = ((hi & 0xfffffu) | lo) != 0u;
    return f32_from(s | 0x7f800000u | (nan ? 0x400000u | ((hi & 0xfffffu) << 3) | (lo >> 29) : 0u));
  }
  const int e = E - 896;
  if (e >= 255) return f32_from(s | 0x7f800000u);
  if (e <= 0) return f32_from(s);  // below the smallest binary32 normal: flushed
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  uint32_t r = ((uint32_t)e << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) r += 1u;
  return f32_from(s | r);
}

}  // namespace amrdev
