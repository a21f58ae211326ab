// Conversions between FP64 and FP32/BF16 done with integer bit operations.
//
// On this GPU every FP64<->FP32 conversion instruction issues on the FP64 pipe, which
// runs at 1/64 of the FP32 rate and is the bottleneck of the solver's FP64 kernels.
// These helpers rebuild the IEEE encodings on the integer pipe instead.  Values below
// the FP32 normal range (|x| < 2^-126) flush to a signed zero; Inf and NaN are kept.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace mca {

// Exact widening of a normal (or zero / Inf / NaN) float; subnormals flush to zero.
__device__ __forceinline__ double f2d_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t m = u & 0x7FFFFFu;
  uint32_t hi, lo;
  if (e == 0u) {
    hi = sign;
    lo = 0u;
  } else if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);   // 896 = 1023 - 127
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Narrowing of the FP64 encoding (hi, lo words) to float by truncating the mantissa
// (relative error < 2^-23); out-of-range magnitudes become zero or infinity.  All the
// helpers below work on 32-bit words: 64-bit integer arithmetic would also occupy the FP64
// pipe on this GPU.
__device__ __forceinline__ float d2f_trunc_words(uint32_t hi, uint32_t lo) {
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int ef = e - 896;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 0xFF) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((uint32_t)ef << 23) | m);
}

__device__ __forceinline__ float d2f_trunc(double v) {
  return d2f_trunc_words((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v));
}

// Narrowing to float with rounding to nearest (ties away from zero): half an FP32 ulp
// (bit 28 of the FP64 mantissa) is added to the magnitude before truncating; a carry into
// the exponent is the correct rounding up into the next binade.  Inf and NaN are passed to
// the truncation unchanged.
__device__ __forceinline__ float d2f_round(double v) {
  uint32_t hi = (uint32_t)__double2hiint(v);
  const uint32_t lo = (uint32_t)__double2loint(v);
  if (((hi >> 20) & 0x7FFu) == 0x7FFu) return d2f_trunc_words(hi, lo);
  const uint32_t lo2 = lo + (1u << 28);
  hi += (lo2 < lo) ? 1u : 0u;
  return d2f_trunc_words(hi, lo2);
}

// An integer 0 <= a < 2^29 as a float, rounded to nearest once, without an int-to-float
// conversion instruction: the two 15- and 14-bit halves are exact as 2^23 + h - 2^23, and
// one FMA joins them.
__device__ __forceinline__ float u29_to_float(uint32_t a) {
  const float hi = __fsub_rn(__uint_as_float(0x4B000000u | (a >> 14)), 8388608.f);
  const float lo = __fsub_rn(__uint_as_float(0x4B000000u | (a & 0x3FFFu)), 8388608.f);
  return __fmaf_rn(hi, 16384.f, lo);
}

// The low half of x as an FP32 pair: x - (double)d2f_round(x), rounded to FP32.  That
// difference is a whole number of ulps of x, at most 2^28 in size (also when the rounding
// of the high half carried into the next binade), so it is the low word of the magnitude
// minus the low word of its rounding, read as a signed 32-bit integer; u29_to_float and a
// power-of-two scale make it a float.  Returns 0 when |x| < 2^-74 (the scale would leave
// the FP32 normal range; the error is then below 2^-98) and for |x| >= 2^180, Inf, NaN.
__device__ __forceinline__ float d2f_low(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t lo = (uint32_t)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  if (ex < 949 || ex > 1202) return 0.f;
  const int32_t dl = (int32_t)(lo - ((lo + (1u << 28)) & 0xE0000000u));   // |dl| <= 2^28
  const uint32_t a = (uint32_t)(dl < 0 ? -dl : dl);
  const float mag = u29_to_float(a) * __int_as_float((ex - 948) << 23);   // * 2^(ex-1075)
  const uint32_t sign = (hi & 0x80000000u) ^ (dl < 0 ? 0x80000000u : 0u);
  return __uint_as_float(__float_as_uint(mag) ^ sign);
}

// BF16 with round-to-nearest-even on the truncated float (the discarded low 29 bits of
// the double only matter for exact BF16 ties).
__device__ __forceinline__ __nv_bfloat16 d2bf16_bits(double v) {
  const uint32_t f = __float_as_uint(d2f_trunc(v));
  uint32_t r;
  if ((f & 0x7F800000u) == 0x7F800000u)
    r = (f >> 16) | ((f & 0xFFFFu) ? 0x40u : 0u);            // Inf / NaN
  else
    r = (f + 0x7FFFu + ((f >> 16) & 1u)) >> 16;
  __nv_bfloat16_raw raw;
  raw.x = (unsigned short)r;
  return __nv_bfloat16(raw);
}

}  // namespace mca
