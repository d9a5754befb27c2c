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
  const uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)(sign | 0x7e00u);  // quiet NaN
  const double v = std::fabs((double)x);
  if (v == 0.0) return sign;
  if (std::isinf(v)) return (uint16_t)(sign | 0x7c00u);
  int e;
  std::frexp(v, &e);               // v = f 2^e, f in [0.5, 1): leading bit at 2^(e-1)
  int E = e - 1 < -14 ? -14 : e - 1;  // binary16 exponent (subnormals share -14)
  const double s = std::ldexp(v, 10 - E);  // significand in units of the last place; exact
  double m = std::floor(s);
  const double rem = s - m;
  if (rem > 0.5 || (rem == 0.5 && std::fmod(m, 2.0) != 0.0)) m += 1.0;
  if (m >= 2048.0) {  // rounding carried into the next binade
    m = 1024.0;
    ++E;
  }
  if (E > 15) return (uint16_t)(sign | 0x7c00u);  // overflow: infinity
  const uint32_t mi = (uint32_t)m;
  if (mi < 1024u) return (uint16_t)(sign | mi);   // subnormal (E == -14)
  return (uint16_t)(sign | ((uint32_t)(E + 15) << 10) | (mi - 1024u));
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
