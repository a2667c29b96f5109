// Operand rounding shared by the field kernels: how a hidden layer's inputs
// and weights enter the contraction for each field precision.
//   f32  : unchanged
//   bf16 : round to nearest even bfloat16
//   f16  : round to nearest even binary16
//   fp8  : e4m3 code of x / s (round to nearest even, saturating at +-448),
//          times s -- s is the layer's activation or weight scale
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include "../../include/pf.h"

namespace pff {

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float round_f16(float x) { return __half2float(__float2half_rn(x)); }
__device__ __forceinline__ unsigned char e4m3_code(float x) {
  return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_value(unsigned char c) {
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
  return __half2float(__half(h));
}
__device__ __forceinline__ float round_prec(float x, int prec, float s) {
  if (prec == PF_PREC_BF16) return round_bf16(x);
  if (prec == PF_PREC_F16) return round_f16(x);
  if (prec == PF_PREC_FP8) return e4m3_value(e4m3_code(x / s)) * s;
  return x;
}

// ---- frequency encoding of the tensor-core fields (Sec. 3.4, gamma(v) =
// [sin(2^k pi v), cos(2^k pi v)], k < F), computed in float32 with every
// product and sum rounded separately (the intrinsics below are never
// contracted), so the precision-emulating oracle can take the same steps.

// sin(2 pi u), cos(2 pi u) for u in [0, 1): octant reduction in turns (exact),
// Taylor polynomials of sin (to a^9) and cos (to a^10) on [0, pi/4].
__device__ __forceinline__ void turn_sincos(float u, float* s_out, float* c_out) {
  const float v = __fmul_rn(u, 8.0f);
  const float fo = floorf(v);
  const int o = (int)fo;
  const float r = __fsub_rn(v, fo);
  const int q = (o >> 1) & 3;
  const float a = __fmul_rn((o & 1) ? __fsub_rn(1.0f, r) : r, 0.785398163f);
  const float a2 = __fmul_rn(a, a);
  float ps = 2.75573192e-06f;
  ps = __fadd_rn(__fmul_rn(ps, a2), -0.000198412698f);
  ps = __fadd_rn(__fmul_rn(ps, a2), 0.00833333333f);
  ps = __fadd_rn(__fmul_rn(ps, a2), -0.166666667f);
  const float sa = __fadd_rn(a, __fmul_rn(__fmul_rn(a, a2), ps));
  float pc = -2.75573192e-07f;
  pc = __fadd_rn(__fmul_rn(pc, a2), 2.48015873e-05f);
  pc = __fadd_rn(__fmul_rn(pc, a2), -0.00138888889f);
  pc = __fadd_rn(__fmul_rn(pc, a2), 0.0416666667f);
  pc = __fadd_rn(__fmul_rn(pc, a2), -0.5f);
  const float ca = __fadd_rn(1.0f, __fmul_rn(a2, pc));
  const float sp = (o & 1) ? ca : sa;
  const float cp = (o & 1) ? sa : ca;
  float s, c;
  if (q == 0) { s = sp; c = cp; }
  else if (q == 1) { s = cp; c = -sp; }
  else if (q == 2) { s = -sp; c = -cp; }
  else { s = -cp; c = sp; }
  *s_out = s;
  *c_out = c;
}

// One step of the encoding of input v: (s, c) = sin / cos (2^k pi v) from
// the previous step's.  At k = 0, 4, 8, ... from turn_sincos of
// frac(2^(k-1) v) (exact: a power-of-two product and its integer part); in
// between by the double-angle formulas sin 2a = 2 sin a cos a and
// cos 2a = 1 - 2 sin^2 a (three doublings at most, so the anchors' error of
// a few 1e-7 grows to a few 1e-6 at most).
__device__ __forceinline__ void freq_next(float v, int k, float& s, float& c) {
  if ((k & 3) == 0) {
    const float t = __fmul_rn(v, ldexpf(1.0f, k - 1));
    turn_sincos(__fsub_rn(t, floorf(t)), &s, &c);
  } else {
    const float s2 = __fmul_rn(__fmul_rn(s, c), 2.0f);
    c = __fsub_rn(1.0f, __fmul_rn(2.0f, __fmul_rn(s, s)));
    s = s2;
  }
}

}  // namespace pff
