// oci_cvt.cuh -- exact float <-> double conversions on the integer pipe.
//
// On this GPU the FP64 pipe runs 1/64 of the FP32 rate and the conversions
// between float and double are issued to it too.  The FP64 refinement kernels
// of the mixed forms are bound by that pipe, so the conversions they need
// (the FP32 correction into FP64, the FP64 residual into FP32) are done here
// with integer operations on the IEEE 754 binary32 / binary64 encodings:
//
//   f2d_exact: binary32 -> binary64 is exact; for a normal or zero input the
//              exponent is rebiased (+896 = 1023 - 127) and the 23 fraction bits
//              move to the top of the 52-bit fraction.
//   d2f_rn:    binary64 -> binary32 rounded to nearest, ties to even (the IEEE
//              default), for results in the normal binary32 range: the top 23 of
//              the 52 fraction bits are kept and the 29 dropped bits decide the
//              rounding; a carry out of the fraction increments the exponent,
//              which also gives infinity above the largest finite binary32.
//
// Zero goes through the integer path as well; the rare remaining inputs
// (subnormal results, infinities, NaN) take the compiler's conversion, so both
// functions return exactly what a plain C cast returns.  The header compiles
// for the host too (a CPU test compares both functions with C casts).
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OCI_CVT_FN __host__ __device__ __forceinline__
#else
#define OCI_CVT_FN static inline
#endif

namespace oci {

OCI_CVT_FN uint32_t cvt_fbits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}

OCI_CVT_FN float cvt_bitsf(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

OCI_CVT_FN double cvt_bitsd(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}

OCI_CVT_FN void cvt_dbits(double d, uint32_t &hi, uint32_t &lo) {
#if defined(__CUDA_ARCH__)
  hi = (uint32_t)__double2hiint(d);
  lo = (uint32_t)__double2loint(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  hi = (uint32_t)(u >> 32);
  lo = (uint32_t)u;
#endif
}

// binary32 -> binary64, exact.
OCI_CVT_FN double f2d_exact(float f) {
  const uint32_t u = cvt_fbits(f);
  const uint32_t s = u & 0x80000000u, a = u & 0x7fffffffu;
  if (a >= 0x7f800000u || (a != 0u && a < 0x00800000u)) return (double)f;  // inf, NaN, subnormal
  const uint32_t bias = a ? (896u << 20) : 0u;
  return cvt_bitsd(s | ((a >> 3) + bias), a << 29);
}

// binary64 -> binary32, round to nearest, ties to even.
OCI_CVT_FN float d2f_rn(double x) {
  uint32_t hi, lo;
  cvt_dbits(x, hi, lo);
  const uint32_t s = hi & 0x80000000u, ah = hi & 0x7fffffffu;
  if (ah >= (897u << 20) && ah < (1151u << 20)) {  // binary64 exponent 897..1150: binary32 normal range
    uint32_t f = ((ah - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu, half = 0x10000000u;
    f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;
    return cvt_bitsf(s | f);
  }
  if ((ah | lo) == 0u) return cvt_bitsf(s);
  return (float)x;  // subnormal or zero result, overflow, inf, NaN
}

// The same, or the compiler's conversion when hw is set (a uniform switch that
// lets a caller compare both forms).
OCI_CVT_FN double cvt_f2d(int hw, float f) { return hw ? (double)f : f2d_exact(f); }
OCI_CVT_FN float cvt_d2f(int hw, double x) { return hw ? (float)x : d2f_rn(x); }

}  // namespace oci
