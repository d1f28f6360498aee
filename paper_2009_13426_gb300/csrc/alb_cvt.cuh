// Conversions to and from FP64 on the integer pipe.
//
// On GB300 the FP64 pipe (2 operations per clock and SM) bounds the FP32
// form's step, and it also executes every conversion to or from FP64. The
// conversions of the step's hot loops are therefore assembled from the IEEE
// 754 binary64 / binary32 bit fields with integer operations, which issue at
// the integer pipe's rate beside the FP64 work:
//   binary64: sign (1) | exponent (11, bias 1023) | fraction (52)
//   binary32: sign (1) | exponent (8, bias 127)   | fraction (23)
// Each result equals the rounded-to-nearest conversion bit for bit wherever
// the target's normal range holds it; the few inputs outside it behave as each
// function states. The header also compiles as plain host C++ (the bit
// casts go through memcpy there), so the same code is checked on the CPU
// against the host's own IEEE conversions.
#pragma once

#include <stdint.h>
#include <string.h>
#ifndef __CUDACC__
#define ALB_CVT_FN inline
#else
#define ALB_CVT_FN __host__ __device__ __forceinline__
#endif

namespace alb {

ALB_CVT_FN uint32_t cvt_bits_f32(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
ALB_CVT_FN float cvt_f32_of_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
ALB_CVT_FN void cvt_bits_f64(double d, uint32_t* hi, uint32_t* lo) {
#ifdef __CUDA_ARCH__
  *hi = (uint32_t)__double2hiint(d);
  *lo = (uint32_t)__double2loint(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  *hi = (uint32_t)(b >> 32);
  *lo = (uint32_t)b;
#endif
}
ALB_CVT_FN double cvt_f64_of_bits(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

// FP64 -> FP32 rounded to nearest, ties to even. Results in FP32's normal
// range (magnitude >= 2^-126) are exact roundings; a rounding carry moves into
// the exponent, so the largest values round to infinity as IEEE says.
// Magnitudes that overflow give +-inf, a NaN gives a NaN, and inputs of
// magnitude below 2^-126 (zero included) give a zero of the input's sign:
// FP32's subnormal range is not produced.
ALB_CVT_FN float cvt_f32_rn(double d) {
  uint32_t hi, lo;
  cvt_bits_f64(d, &hi, &lo);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const int e = ex - 896;                                      // FP32 biased exponent
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);      // 23 kept fraction bits
  const uint32_t r = lo & 0x1fffffffu;                         // 29 dropped bits
  const uint32_t up = (r > 0x10000000u) | ((r == 0x10000000u) & (m & 1u));
  uint32_t b = ((uint32_t)e << 23) + m + up;
  b = e >= 255 ? 0x7f800000u : b;
  b = e <= 0 ? 0u : b;
  b = (ex == 2047 && ((hi & 0xfffffu) | lo) != 0u) ? 0x7fc00000u : b;
  return cvt_f32_of_bits((hi & 0x80000000u) | b);
}

// FP32 -> FP64, exact for zeros, normal values, infinities and NaNs (the
// fraction moves up by 29 bits); a subnormal FP32 input gives a zero of its
// sign.
ALB_CVT_FN double cvt_f64(float f) {
  const uint32_t b = cvt_bits_f32(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t ed = e == 255u ? 2047u : e + 896u;
  uint32_t hi = (b & 0x80000000u) | (ed << 20) | ((b >> 3) & 0xfffffu);
  uint32_t lo = b << 29;
  hi = e == 0u ? (b & 0x80000000u) : hi;
  lo = e == 0u ? 0u : lo;
  return cvt_f64_of_bits(hi, lo);
}

// int32 -> FP64, exact for every value: the magnitude's leading one sets the
// exponent and the bits below it the fraction.
ALB_CVT_FN int cvt_clz(uint32_t a) {
#ifdef __CUDA_ARCH__
  return __clz((int)a);
#else
  int n = 0;
  while (n < 32 && !(a & (0x80000000u >> n))) ++n;
  return n;
#endif
}
ALB_CVT_FN double cvt_f64(int n) {
  const uint32_t s = n < 0 ? 0x80000000u : 0u;
  const uint32_t a = n < 0 ? 0u - (uint32_t)n : (uint32_t)n;
  const int lz = cvt_clz(a);
  const uint32_t x = (a << (lz & 31)) << 1;  // bits below the leading one, left-aligned
  uint32_t hi = s | ((uint32_t)(1054 - lz) << 20) | (x >> 12);
  uint32_t lo = x << 20;
  hi = a == 0u ? 0u : hi;
  lo = a == 0u ? 0u : lo;
  return cvt_f64_of_bits(hi, lo);
}

}  // namespace alb
