// Exact floating-point operations done on the integer units.
//
// GB300 executes FP64 arithmetic and the conversions to and from FP64 at a
// small fraction of its FP32 / integer rate, and the defect-correction passes
// are bound by that rate.  Three of their operations are exact bit
// manipulations of IEEE 754 binary32 / binary64 encodings and need no FP64
// unit for normal values:
//   widen_f32(x)   binary32 -> binary64, exact: rebias the exponent
//                  (+ 1023 - 127) and append 29 zero bits to the fraction;
//   times4(x)      x * 4 in binary64, exact while the result stays normal:
//                  add 2 to the exponent;
//   narrow_f64(x)  binary64 -> binary32 rounded to nearest, ties to even
//                  (IEEE 754 section 4.3.1): keep the top 23 fraction bits,
//                  round on the 29 dropped bits, the carry propagating into
//                  the exponent (and to infinity past the largest finite
//                  value, as the rounding rule requires).
// Zero is handled in place; every other case outside the normal range
// (subnormal operands or results, infinities, NaN) takes the hardware
// instruction, so the results equal the hardware's bit for bit.
#pragma once
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace sorgb {

__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ float f32_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ double f64_of(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

// The hardware instructions for the rare operands, kept out of line: inlined,
// the compiler turns the branch into a predicated FP64 instruction that every
// warp issues, which would occupy the FP64 pipe this header exists to spare.
static __host__ __device__ __noinline__ double widen_hw(float x) { return (double)x; }
static __host__ __device__ __noinline__ double times4_hw(double x) { return x * 4.0; }
static __host__ __device__ __noinline__ float narrow_hw(double x) { return (float)x; }

__host__ __device__ __forceinline__ double widen_f32(float x) {
  const uint32_t b = bits_of(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  if (e != 0u && e != 0xFFu)
    return f64_of(sign | ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29));
  if ((b & 0x7FFFFFFFu) == 0u) return f64_of(sign);  // signed zero
  return widen_hw(x);                                // subnormal, infinity, NaN
}

__host__ __device__ __forceinline__ double times4(double x) {
  const uint64_t b = bits_of(x);
  const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
  if (e >= 1u && e <= 0x7FCu) return f64_of(b + (2ull << 52));  // the result is normal and finite
  if ((b << 1) == 0ull) return x;                               // signed zero
  return times4_hw(x);                                          // subnormal, overflow, infinity, NaN
}

__host__ __device__ __forceinline__ float narrow_f64(double x) {
  const uint64_t b = bits_of(x);
  const int e = (int)((b >> 52) & 0x7FFu);
  const int ef = e - 1023 + 127;  // biased binary32 exponent of the same power of two
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  if (ef >= 1 && ef <= 254) {
    const uint64_t frac = b & ((1ull << 52) - 1ull);
    const uint32_t kept = (uint32_t)(frac >> 29);
    const uint64_t dropped = frac & ((1ull << 29) - 1ull);
    const uint64_t half = 1ull << 28;
    uint32_t r = sign | ((uint32_t)ef << 23) | kept;
    if (dropped > half || (dropped == half && (kept & 1u))) r += 1u;  // ties to even; carry may reach infinity
    return f32_of(r);
  }
  if ((b << 1) == 0ull) return f32_of(sign);  // signed zero
  return narrow_hw(x);                        // subnormal results, overflow, infinity, NaN
}

}  // namespace sorgb
