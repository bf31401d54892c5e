// dfloat.cuh -- double-float arithmetic on the FP32 pipe: a double split
// into a (hi, lo) pair of floats with integer bit operations, error-free
// products by FMA, TwoSum accumulation, and the way back to a double.
// GB300 runs FP64 arithmetic and FP64<->FP32 conversions at about 2 per
// clock per SM, integer and FP32 operations at about 128, so the kernels
// keep both conversions and arithmetic off the FP64 pipe.
#pragma once

#include <cuda_runtime.h>

namespace sldg {

// ---------------------------------------------------------------------------
// double <-> (hi, lo) float pair with integer operations only
// ---------------------------------------------------------------------------
// hi = x truncated to 24 significant bits, lo = the next 23 bits rounded to
// nearest (|x - hi - lo| <= 2^-47 |x|).  |x| < 2^-126 flushes to zero; Inf and
// NaN keep their class in hi.
__device__ __forceinline__ float2 dsplit(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int ef = e - 896;  // float biased exponent of hi
  const unsigned m23 = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
  const unsigned hb = sign | ((unsigned)ef << 23) | m23;
  const unsigned cb = sign | ((unsigned)(ef - 23) << 23);
  const unsigned lb = (cb | ((lo >> 6) & 0x7FFFFFu)) + ((lo >> 5) & 1u);
  float h = __uint_as_float(hb);
  float l = __uint_as_float(lb) - __uint_as_float(cb);
  if (ef - 23 <= 0) l = 0.0f;
  if (ef <= 0) h = 0.0f;
  if (ef >= 255) {  // beyond float range, Inf or NaN
    h = __uint_as_float(sign | 0x7F800000u | ((e == 0x7FF && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u));
    l = 0.0f;
  }
  return make_float2(h, l);
}

// Exact float -> double by integer operations (zero, finite and Inf/NaN;
// float denormals, never produced here above 2^-126 scale, flush to zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned t = u & 0x7FFFFFFFu;
  unsigned hi = ((t >> 3) + (896u << 20)) | (u & 0x80000000u);
  unsigned lo = u << 29;
  if (t < 0x00800000u) {
    hi = u & 0x80000000u;
    lo = 0u;
  }
  if (t >= 0x7F800000u) hi |= 0x7FF00000u;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double djoin(float h, float l) { return f2d_bits(h) + f2d_bits(l); }

// Double-float accumulation sum += a * x with a = (ah, al), x = (xh, xl):
// error-free product of the high parts (FMA), TwoSum into the high word,
// everything smaller into the low word.
__device__ __forceinline__ void df_first(float ah, float al, float2 x, float& sh, float& sl) {
  sh = ah * x.x;
  sl = fmaf(ah, x.x, -sh);
  sl = fmaf(ah, x.y, sl);
  sl = fmaf(al, x.x, sl);
}

__device__ __forceinline__ void df_mac(float ah, float al, float2 x, float& sh, float& sl) {
  const float p = ah * x.x;
  const float e = fmaf(ah, x.x, -p);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl += err + e;
  sl = fmaf(ah, x.y, sl);
  sl = fmaf(al, x.x, sl);
}


// The 8 bytes of an FP64 element can also hold a double-float pair: hi in
// the low word, lo in the high word (the memory layout of a float2 (hi, lo)).
__device__ __forceinline__ double df_pack(float h, float l) {
  return __hiloint2double(__float_as_int(l), __float_as_int(h));
}
__device__ __forceinline__ float2 df_unpack(double x) {
  return make_float2(__int_as_float(__double2loint(x)), __int_as_float(__double2hiint(x)));
}

// Packed FP32x2 arithmetic (two independent lanes per instruction).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

}  // namespace sldg
