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

}  // namespace pff
