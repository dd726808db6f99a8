// Double-float arithmetic on the FP32 pipe (Dekker's two-product by fused
// multiply-add, Knuth's two-sum; Dekker 1971, Bailey's double-float method)
// for the CG operator q = A_0 p: values and p held as FP32 pairs hi + lo (48
// significant bits), q assembled in FP64.  Used by the single-system and the
// batched CG operator kernels.
#pragma once

#include <cuda_runtime.h>

namespace amg {

// x = hi + lo with |lo| < ulp(hi): hi keeps the sign, the exponent and the 23
// leading fraction bits of the double (truncated), lo the remaining 29 bits
// (rounded to 24), both built with integer operations only (no FP64
// instructions).  |x| < 2^-126 gives (0, 0); |x| >= 2^128 gives (+-inf, 0).
__device__ __forceinline__ float2 split_double_float(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
  const unsigned sign = hw & 0x80000000u;
  if (e < -126) return make_float2(0.f, 0.f);
  if (e > 127) return make_float2(__uint_as_float(sign | 0x7F800000u), 0.f);
  const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | m23);
  const unsigned rem = lw & 0x1FFFFFFFu;  // x - hi = rem * 2^(e - 52)
  float lo = __uint2float_rn(rem);
  if (e >= -74)
    lo = __fmul_rn(lo, __uint_as_float((unsigned)(e - 52 + 127) << 23));
  else  // 2^(e-52) is below FP32's normal range: scale in two exact steps
    lo = __fmul_rn(__fmul_rn(lo, 0x1p-60f), __uint_as_float((unsigned)(e + 8 + 127) << 23));
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// f * 2^s as a double, exactly, built with integer operations (FP32 values
// below the normal range count as 0).
__device__ __forceinline__ double float_to_double_scaled(float f, int s) {
  const unsigned b = __float_as_uint(f);
  const int e8 = (int)((b >> 23) & 0xFFu);
  if (e8 == 0) return 0.0;
  if (e8 == 255) return (double)f;
  const unsigned hw = (b & 0x80000000u) | ((unsigned)(e8 - 127 + 1023 + s) << 20) |
                      ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hw, (int)((b & 0x7u) << 29));
}

// (sh, sl) += (ah + al) * (xh + xl)
// sh takes the rounded products through Knuth's two-sum (its rounding
// errors kept exactly), sl the errors and the cross terms, summed plainly
// (the kernel below gives each block its own sl)
__device__ __forceinline__ void df_mac(float &sh, float &sl, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float pe = __fmaf_rn(a.x, x.x, -p);                     // a.x * x.x = p + pe exactly
  const float cross = __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, pe));
  const float s = __fadd_rn(sh, p);                             // two-sum: sh + p = s + err
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, cross));
}

// (s, e) += t by Knuth's two-sum: s the rounded sum, its error added to e
__device__ __forceinline__ void two_sum_into(float &s, float &e, float t) {
  const float u = __fadd_rn(s, t);
  const float bb = __fsub_rn(u, s);
  e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(u, bb)), __fsub_rn(t, bb)));
  s = u;
}

}  // namespace amg
