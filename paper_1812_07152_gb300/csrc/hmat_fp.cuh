// FP32 <-> FP64 conversions and power-of-two scaling of doubles on the integer units.
// FP64 arithmetic and conversions run at 1/64 of the FP32 rate on this GPU, and the
// mixed mode converts every value of W on the way in and every result on the way out.
// All three follow from the IEEE 754 binary formats: a normal binary32 value (biased
// exponent 1..254) is the binary64 value with exponent rebiased by 1023 - 127 = 896
// and the 23 fraction bits at the top of the 52; narrowing keeps the top 23 fraction
// bits and rounds the 29 dropped ones to nearest, ties to even (a carry out of the
// fraction steps the exponent, up to infinity); multiplying a normal binary64 value by
// 2^e adds e to its exponent field while the sum stays in 1..2046; zero stays zero (with
// its sign) in all three. Other values (subnormals, infinities, NaN, results leaving the
// normal range) take the hardware path. kOutOfLine puts that path behind a call: inline,
// the compiler if-converts it and it runs, at the FP64 rate, for every value (measured:
// the W split's FP64 pipe 80 % busy), while a call costs registers where they are short
// (measured: the near-field epilogue is faster with the inline form).
#pragma once

#include <cstdint>

namespace hmat {

static __device__ __noinline__ double widen_f32_hw(float f) { return (double)f; }
static __device__ __noinline__ float narrow_f64_hw(double d) { return __double2float_rn(d); }
static __device__ __noinline__ double mul_f64_hw(double a, double b) { return a * b; }

template <bool kOutOfLine = false>
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7FFFFFFFu;
  if (mag - 0x00800000u >= 0x7F000000u && mag != 0) return kOutOfLine ? widen_f32_hw(f) : (double)f;
  const uint32_t hi = (b & 0x80000000u) | (mag ? (mag >> 3) + 0x38000000u : 0u);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// round-to-nearest-even binary64 -> binary32
template <bool kOutOfLine = false>
__device__ __forceinline__ float narrow_f64(double d) {
  const uint64_t b = (uint64_t)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t ex = (hi >> 20) & 0x7FFu;
  if ((hi & 0x7FFFFFFFu) == 0 && lo == 0) return __uint_as_float(hi);  // +-0
  if (ex - 897u >= 254u) return kOutOfLine ? narrow_f64_hw(d) : __double2float_rn(d);  // exponent outside 1..254
  uint32_t v = ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu;
  v += (rest > 0x10000000u || (rest == 0x10000000u && (v & 1u))) ? 1u : 0u;
  return __uint_as_float(v | (hi & 0x80000000u));
}

// d * 2^e; sc = 2^e as a double (the hardware path's factor)
template <bool kOutOfLine = false>
__device__ __forceinline__ double scale_pow2(double d, int e, double sc) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return d;  // +-0
  if (ex == 0 || ex == 0x7FF || ex + e < 1 || ex + e > 0x7FE) return kOutOfLine ? mul_f64_hw(d, sc) : d * sc;
  return __longlong_as_double(b + ((long long)e << 52));
}

}  // namespace hmat
