// Exact digit slices of float64 values for products on the bf16 tensor
// cores (Ozaki's error-free splitting; the digit extraction from the float64
// bits is this library's).  A value v with |v| < 2^e is cut into nine base-64
// digits of |v| 2^(54 - e), truncated: v = sign 2^e sum_{s=1..9} d_s 2^(-6s)
// + (below 2^(e-54)), every d_s an integer in [0, 63] and so exact in bf16.
#pragma once

#include <cstdint>

namespace dm {

constexpr int kRsSlices = 9;

// Nine signed base-64 digits of |v| * 2^(54 - e) (truncated), |v| < 2^e, from
// the float64 bits of v, as bf16 bit patterns (the high half of each word;
// the low half is ignored).  Integer and float32 operations only: GB300's
// float64 pipe, which also carries the integer-float conversions, is narrow.
// A digit d < 2^23 becomes the float d exactly as (2^23 + d) - 2^23, and a
// float with at most 8 significant bits is its own bf16 truncation.  NaN
// digits for NaN or infinity.
__device__ __forceinline__ void digits9(unsigned long long bits, int e, uint32_t (&q)[kRsSlices]) {
  const uint32_t sign = (uint32_t)(bits >> 63) << 31;
  const int ex = (int)((bits >> 52) & 0x7ff);
  const unsigned long long mant = (bits & 0xfffffffffffffull) | (ex ? (1ull << 52) : 0ull);
  const int sh = (ex ? ex : 1) - 1075 + 54 - e;  // <= 1 for |v| < 2^e
  if (ex == 0x7ff || sh > 1) {
#pragma unroll
    for (int k = 0; k < kRsSlices; ++k) q[k] = 0x7fc00000u;
    return;
  }
  const unsigned long long Y = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
  const uint32_t hi = (uint32_t)(Y >> 32), lo = (uint32_t)Y;
  // digit s occupies bits [48 - 6s, 54 - 6s) of Y
  uint32_t d[kRsSlices];
  d[0] = (hi >> 16) & 63;
  d[1] = (hi >> 10) & 63;
  d[2] = (hi >> 4) & 63;
  d[3] = ((hi & 15) << 2) | (lo >> 30);
  d[4] = (lo >> 24) & 63;
  d[5] = (lo >> 18) & 63;
  d[6] = (lo >> 12) & 63;
  d[7] = (lo >> 6) & 63;
  d[8] = lo & 63;
#pragma unroll
  for (int k = 0; k < kRsSlices; ++k)
    q[k] = __float_as_uint(__uint_as_float(0x4b000000u | d[k]) - 8388608.0f) | sign;
}

// Exponent e with |v| < 2^e for every v whose high word (sign cleared) is at
// most hmax; subnormal or zero maxima share e = -1021.
__device__ __forceinline__ int scale_exponent(uint32_t hmax) {
  const int E = (int)(hmax >> 20);
  return E == 0 ? -1021 : E - 1022;
}

}  // namespace dm
