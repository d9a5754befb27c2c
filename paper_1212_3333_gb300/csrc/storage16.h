// Host conversions between FP32 and the two 16-bit cell formats the bricks can be stored
// in: IEEE binary16 (1-5-10) and bfloat16 (1-8-7), both rounded to nearest, ties to even,
// as the IEEE 754 default rounding defines it.  Used when bricks are uploaded; the kernels
// widen the cells back to FP32 before any arithmetic.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/amr.h"

namespace amr {

inline uint16_t bf16_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x0040u);  // quiet NaN
  // keep the top 16 bits, adding half an ulp minus one plus the kept lsb (ties to even)
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

inline float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

inline uint16_t f16_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  const uint32_t sign = (u >> 16) & 0x8000u;
  uint32_t a = u & 0x7fffffffu;
  if (a > 0x7f800000u) return (uint16_t)(sign | 0x7e00u);  // quiet NaN
  if (a >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u); // |x| >= 65520 rounds to infinity
  if (a >= 0x38800000u) {
    // normal binary16 (|x| >= 2^-14): rebias the exponent (127 -> 15) and keep 10 fraction
    // bits, adding half an ulp minus one plus the kept lsb (ties to even; a carry moves
    // into the exponent)
    a += 0x00000fffu + ((a >> 13) & 1u);
    return (uint16_t)(sign | ((a - 0x38000000u) >> 13));
  }
  if (a <= 0x33000000u) return (uint16_t)sign;  // |x| <= 2^-25 rounds to zero
  // subnormal binary16: |x| / 2^-24 rounded to an integer (1024 is the smallest normal)
  const uint32_t e = a >> 23;                         // 102..112
  const uint32_t mant = (a & 0x7fffffu) | 0x800000u;  // |x| = mant 2^(e - 150)
  const uint32_t shift = 126u - e;                    // |x| / 2^-24 = mant / 2^shift
  uint32_t m = mant >> shift;
  const uint32_t rem = mant & ((1u << shift) - 1u), half = 1u << (shift - 1u);
  if (rem > half || (rem == half && (m & 1u))) ++m;
  return (uint16_t)(sign | m);
}

inline float f16_value(uint16_t h) {
  const int E = (h >> 10) & 31, m = h & 1023;
  double v;
  if (E == 31) v = m ? NAN : INFINITY;
  else if (E == 0) v = std::ldexp((double)m, -24);
  else v = std::ldexp((double)(1024 + m), E - 25);
  return (float)((h & 0x8000u) ? -v : v);
}

inline uint16_t storage_bits(amr_dtype t, float x) {
  return t == AMR_F16 ? f16_bits(x) : bf16_bits(x);
}

// the FP32 value the kernels see for a cell stored as x
inline float storage_round(amr_dtype t, float x) {
  if (t == AMR_F32) return x;
  return t == AMR_F16 ? f16_value(f16_bits(x)) : bf16_value(bf16_bits(x));
}

}  // namespace amr
