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
pf_status pf_field_pack(pf_ctx*, pf_field*) { return PF_OK; }
