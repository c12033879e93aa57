// float <-> double conversions by integer arithmetic on the IEEE-754
// encodings (host and device), so that the Krylov kernels keep GB300's narrow
// FP64 pipe for their FP64 arithmetic.  Widening re-biases the exponent and
// shifts the significand (exact); narrowing rounds the 52-bit significand to
// 23 bits, to nearest with ties to even (a carry into the exponent is the
// correct rounding, up to infinity).  Zeros, subnormal floats, results
// outside the normal float range, infinities and NaNs take the compiler's
// conversions.  Tested on the host against the C conversions
// (tests/test_host_fconv.py).
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FCONV_HD __host__ __device__ __forceinline__
#else
#define FCONV_HD inline
#endif

namespace thermo {

FCONV_HD uint64_t fconv_bits(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
}
FCONV_HD double fconv_double(uint64_t b) {
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
}
FCONV_HD uint32_t fconv_bits(float x) {
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  return b;
}
FCONV_HD float fconv_float(uint32_t b) {
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
}

FCONV_HD double f2d_int(float f) {
  const uint32_t u = fconv_bits(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  return fconv_double(((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                      ((uint64_t)(u & 0x7fffffu) << 29));
}

FCONV_HD float d2f_int(double x) {
  const uint64_t b = fconv_bits(x);
  const int E = (int)((b >> 52) & 0x7ffu);
  if (E < 897 || E > 1150) return (float)x;  // zero, below the normal floats, huge, inf / nan
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = b & 0xfffffffffffffull;
  uint32_t f = ((uint32_t)(E - 896) << 23) | (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1fffffffu), half = 0x10000000u;
  if (rem > half || (rem == half && (f & 1u))) ++f;
  return fconv_float(sign | f);
}

}  // namespace thermo
