// Tensor-core (tcgen05) field kernels -- placeholder until the tcgen05 path lands.
#include "pf_internal.h"

pf_status pf_tc_available(const pf_field* f) { (void)f; return PF_ERR_UNSUPPORTED; }
pf_status pf_tc_forward(pf_ctx* ctx, const pf_field*, const float*, int64_t, const uint32_t*, float*, const uint32_t*,
                        const float*, float*) {
  return pf_fail(ctx, PF_ERR_UNSUPPORTED, "tensor-core field path unavailable");
}
pf_status pf_tc_backward(pf_ctx* ctx, const pf_field*, const float*, const float*, const float*, int64_t, float*, float*) {
  return pf_fail(ctx, PF_ERR_UNSUPPORTED, "tensor-core field path unavailable");
}
#include "pf_field_common.cuh"

namespace {
struct Bounds { int64_t b[10]; float s_w[8]; int n; };

// Hidden-layer weights rounded to the field precision (fp8: per-layer scale).
__global__ void k_round_weights(const float* __restrict__ w, float* __restrict__ wr, Bounds B, int prec) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.b[B.n]) return;
  int l = 0;
  while (l + 1 < B.n && i >= B.b[l + 1]) ++l;
  wr[i] = pff::round_prec(w[i], prec, B.s_w[l]);
}
}  // namespace

pf_status pf_field_pack(pf_ctx* ctx, pf_field* f) {
  if (f->desc.prec == PF_PREC_F32) return PF_OK;
  if (!f->wr) {
    if (cudaMalloc(&f->wr, f->n_params * sizeof(float)) != cudaSuccess) return pf_fail(ctx, PF_ERR_OOM, "field pack");
    PF_CUDA(ctx, cudaMemsetAsync(f->wr, 0, f->n_params * sizeof(float), ctx->stream));
  }
  Bounds B;
  B.n = f->n_layers - 1;
  for (int l = 0; l <= B.n; ++l) B.b[l] = f->layer_off[l];
  for (int l = 0; l < 8; ++l) B.s_w[l] = f->scales_host[16 + l] > 0.f ? f->scales_host[16 + l] : 1.f;
  int64_t n = B.b[B.n];
  k_round_weights<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(f->w, f->wr, B, f->desc.prec);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}
