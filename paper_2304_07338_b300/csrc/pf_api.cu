// Context, errors, scratch arena, volume checks, global majorant, device
// scan and the FP64 image error reduction.
#include "pf_internal.h"
#include <cuda_fp16.h>
#include <cstdarg>
#include <cmath>
#include <vector>
#include <algorithm>

pf_status pf_fail(pf_ctx* ctx, pf_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

pf_status pf_cuda_check(pf_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PF_OK;
  cudaGetLastError();  // clear a non-sticky error
  return pf_fail(ctx, e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

pf_status pf_scratch(pf_ctx* ctx, int slot, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  if (ctx->ws_size[slot] < bytes) {
    if (ctx->ws[slot]) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws[slot]);
      ctx->ws[slot] = nullptr;
      ctx->ws_size[slot] = 0;
    }
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&ctx->ws[slot], want);
    if (e != cudaSuccess) return pf_cuda_check(ctx, e, "scratch cudaMalloc");
    ctx->ws_size[slot] = want;
  }
  *out = ctx->ws[slot];
  return PF_OK;
}

extern "C" pf_status pf_create(pf_ctx** out, int device, void* stream) {
  if (!out) return PF_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PF_ERR_INVALID_ARG;
  }
  pf_ctx* c = new pf_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  DeviceGuard dg(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->err_dev, 256) != cudaSuccess || cudaMalloc(&c->dbl_dev, 4096) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->err_dev);
    delete c;
    return PF_ERR_OOM;
  }
  cudaMemset(c->err_dev, 0, 256);
  cudaDeviceSynchronize();
  *out = c;
  return PF_OK;
}

extern "C" pf_status pf_destroy(pf_ctx* c) {
  if (!c) return PF_OK;
  DeviceGuard dg(c->device);
  cudaStreamSynchronize(c->stream);
  for (int i = 0; i < WS_COUNT; ++i) cudaFree(c->ws[i]);
  for (auto& m : c->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    for (auto e : c->aux_ev) if (e) cudaEventDestroy(e);
    cudaStreamDestroy(c->aux);
  }
  cudaFree(c->err_dev);
  cudaFree(c->dbl_dev);
  delete c;
  return PF_OK;
}

extern "C" pf_status pf_set_stream(pf_ctx* c, void* stream) {
  if (!c) return PF_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return PF_OK;
}

extern "C" pf_status pf_set_counters(pf_ctx* c, uint64_t* counters_dev) {
  if (!c) return PF_ERR_INVALID_ARG;
  c->counters = (unsigned long long*)counters_dev;
  return PF_OK;
}

pf_status pf_aux_stream(pf_ctx* ctx) {
  if (ctx->aux) return PF_OK;
  PF_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
  for (auto& e : ctx->aux_ev) PF_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return PF_OK;
}

static cudaEvent_t take_event(pf_ctx* c) {
  if (!c->event_pool.empty()) { cudaEvent_t e = c->event_pool.back(); c->event_pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

StageTimer::StageTimer(pf_ctx* c, int st) : ctx(c), stage(st) {
  if (!ctx->timing) return;
  a = take_event(ctx);
  b = take_event(ctx);
  cudaEventRecord(a, ctx->stream);
}
StageTimer::~StageTimer() {
  if (!ctx->timing || !a) return;
  cudaEventRecord(b, ctx->stream);
  ctx->marks.push_back({stage, a, b});
}

extern "C" pf_status pf_stage_timing(pf_ctx* c, int enable) {
  if (!c) return PF_ERR_INVALID_ARG;
  c->timing = enable ? 1 : 0;
  return PF_OK;
}

extern "C" pf_status pf_stage_times(pf_ctx* c, double* ms_host, int* launches_host, int n) {
  if (!c || !ms_host || n <= 0) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(c->device);
  PF_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < n; ++i) { ms_host[i] = 0.0; if (launches_host) launches_host[i] = 0; }
  for (auto& m : c->marks) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m.a, m.b);
    if (m.stage >= 0 && m.stage < n) { ms_host[m.stage] += ms; if (launches_host) launches_host[m.stage] += 1; }
    c->event_pool.push_back(m.a);
    c->event_pool.push_back(m.b);
  }
  c->marks.clear();
  return PF_OK;
}

extern "C" const char* pf_last_error(const pf_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

pf_status pf_check_error_word(pf_ctx* c) {
  uint32_t w = 0;
  PF_CUDA(c, cudaMemcpyAsync(&w, c->err_dev, 4, cudaMemcpyDeviceToHost, c->stream));
  PF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (w == 0) return PF_OK;
  PF_CUDA(c, cudaMemsetAsync(c->err_dev, 0, 4, c->stream));
  if (w & PFE_ITER_CAP) return pf_fail(c, PF_ERR_TIMEOUT, "a device loop hit its iteration limit (error word 0x%x)", w);
  return pf_fail(c, PF_ERR_NUMERIC, "device reported a non-finite or out-of-range value (error word 0x%x)", w);
}

extern "C" pf_status pf_sync(pf_ctx* c) {
  if (!c) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(c->device);
  PF_CUDA(c, cudaStreamSynchronize(c->stream));
  return pf_check_error_word(c);
}

// Argument checks that need no context: on a problem they write a message
// into buf (len bytes) and return true.  Both the context entry points and
// the allocation-free path tracer use them, so they accept the same inputs.
bool pf_volume_problem(const pf_volume* v, char* buf, size_t len) {
  auto bad = [&](const char* fmt, auto... a) {
    if (buf && len) snprintf(buf, len, fmt, a...);
    return true;
  };
  if (!v) return bad("%s", "volume is NULL");
  if (v->nx < 1 || v->ny < 1 || v->nz < 1 || v->nx > 8192 || v->ny > 8192 || v->nz > 8192)
    return bad("%s", "volume extents must be in [1, 8192]");
  if (v->dtype < 0 || v->dtype > 2) return bad("unknown volume dtype %d", (int)v->dtype);
  if (!v->data_dev || !v->tf_lut_dev) return bad("%s", "volume data or transfer function is NULL");
  if (v->tf_n < 2 || v->tf_n > 65536) return bad("%s", "tf_n must be in [2, 65536]");
  if ((uintptr_t)v->tf_lut_dev % 16) return bad("%s", "transfer function must be 16-byte aligned");
  if (!(v->sigma_scale >= 0.f) || !std::isfinite(v->sigma_scale) || !(v->albedo >= 0.f) || !std::isfinite(v->albedo))
    return bad("%s", "sigma_scale and albedo must be finite and non-negative");
  if (!(v->majorant >= 0.f) || !std::isfinite(v->majorant)) return bad("%s", "majorant must be finite and >= 0");
  if (v->brick != 0 && (v->brick < 2 || v->brick > 256 || (v->brick & (v->brick - 1))))
    return bad("%s", "brick must be 0 (= 8) or a power of two in [2, 256]");
  const int Bb = v->brick ? v->brick : 8;
  if (v->brick_primary != 0 &&
      (v->brick_primary < Bb || v->brick_primary > 1024 || (v->brick_primary & (v->brick_primary - 1))))
    return bad("%s", "brick_primary must be 0 or a power-of-two multiple of brick, <= 1024");
  if (v->brick_shadow != 0 &&
      (v->brick_shadow < Bb || v->brick_shadow > 1024 || (v->brick_shadow & (v->brick_shadow - 1))))
    return bad("%s", "brick_shadow must be 0 or a power-of-two multiple of brick, <= 1024");
  const int64_t B = Bb;
  if (((v->nx + B - 1) / B) * ((v->ny + B - 1) / B) * ((v->nz + B - 1) / B) >= ((int64_t)1 << 31))
    return bad("%s", "too many majorant bricks (>= 2^31): use a larger brick");
  return false;
}

bool pf_lights_problem(const pf_light* l, int n, char* buf, size_t len) {
  auto bad = [&](const char* fmt, auto... a) {
    if (buf && len) snprintf(buf, len, fmt, a...);
    return true;
  };
  if (n < 1 || n > PF_MAX_LIGHTS || !l) return bad("need 1..%d lights (host array)", PF_MAX_LIGHTS);
  for (int i = 0; i < n; ++i) {
    if (l[i].kind != 0 && l[i].kind != 1) return bad("light %d: unknown kind", i);
    const float n2 = l[i].v[0] * l[i].v[0] + l[i].v[1] * l[i].v[1] + l[i].v[2] * l[i].v[2];
    if (l[i].kind == 0 && !(n2 > 0.f && std::isfinite(n2))) return bad("light %d: zero or non-finite direction", i);
    if (l[i].kind == 1 && l[i].v[0] >= 0.f && l[i].v[0] <= 1.f && l[i].v[1] >= 0.f && l[i].v[1] <= 1.f &&
        l[i].v[2] >= 0.f && l[i].v[2] <= 1.f)
      return bad("light %d: point lights must lie outside the unit box", i);
  }
  return false;
}

pf_status pf_check_volume(pf_ctx* ctx, const pf_volume* v) {
  char msg[256];
  if (pf_volume_problem(v, msg, sizeof(msg))) return pf_fail(ctx, PF_ERR_INVALID_ARG, "%s", msg);
  return PF_OK;
}

pf_status pf_check_lights(pf_ctx* ctx, const pf_light* l, int n) {
  char msg[256];
  if (pf_lights_problem(l, n, msg, sizeof(msg))) return pf_fail(ctx, PF_ERR_INVALID_ARG, "%s", msg);
  return PF_OK;
}

// ------------------------------------------------------------------ majorant
namespace {
template <typename T>
__global__ void k_max_density(const T* __restrict__ data, int64_t n, unsigned int* out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v;
    if constexpr (sizeof(T) == 4) v = (float)data[i];
    else if constexpr (sizeof(T) == 2) v = __half2float(*(const __half*)&data[i]);
    else v = (float)data[i] / 255.0f;
    m = fmaxf(m, v);
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // m >= 0: bit order = value order
}
}  // namespace


pf_status pf_majorant_impl(pf_ctx* ctx, const pf_volume* v, float* out) {
  if (v->majorant > 0.f) { *out = v->majorant; return PF_OK; }
  int64_t n = (int64_t)v->nx * v->ny * v->nz;
  unsigned int* m;
  PF_TRY(pf_scratch(ctx, WS_REDUCE, 64, (void**)&m));
  PF_CUDA(ctx, cudaMemsetAsync(m, 0, 4, ctx->stream));
  int grid = std::max(1, std::min<int>((int)((n + 255) / 256), ctx->num_sms * 8));
  if (v->dtype == PF_F32) k_max_density<float><<<grid, 256, 0, ctx->stream>>>((const float*)v->data_dev, n, m);
  else if (v->dtype == PF_F16) k_max_density<uint16_t><<<grid, 256, 0, ctx->stream>>>((const uint16_t*)v->data_dev, n, m);
  else k_max_density<uint8_t><<<grid, 256, 0, ctx->stream>>>((const uint8_t*)v->data_dev, n, m);
  PF_CUDA(ctx, cudaGetLastError());
  unsigned int bits = 0;
  std::vector<float> lut((size_t)v->tf_n * 4);
  PF_CUDA(ctx, cudaMemcpyAsync(&bits, m, 4, cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaMemcpyAsync(lut.data(), v->tf_lut_dev, lut.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  float dmax;
  memcpy(&dmax, &bits, 4);
  if (dmax > 1.0f) dmax = 1.0f;
  // alpha at dmax (same lerp as the kernels), then the table's nodes below it
  float s = dmax * (float)(v->tf_n - 1);
  int i = (int)std::floor(s);
  if (i > v->tf_n - 2) i = v->tf_n - 2;
  float f = s - (float)i;
  float a = lut[4 * i + 3], b = lut[4 * (i + 1) + 3];
  float amax = a + f * (b - a);
  for (int k = 0; k < v->tf_n; ++k) {
    float node_d = (float)k / (float)(v->tf_n - 1);
    if (node_d <= dmax && lut[4 * k + 3] > amax) amax = lut[4 * k + 3];
  }
  *out = v->sigma_scale * amax * 1.0009765625f;
  return PF_OK;
}

extern "C" pf_status pf_volume_majorant(pf_ctx* ctx, const pf_volume* v, float* out_host) {
  if (!ctx || !out_host) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, v));
  pf_volume w = *v;
  w.majorant = 0.f;
  return pf_majorant_impl(ctx, &w, out_host);
}

// ------------------------------------------------------------------ scan
namespace {
constexpr int kScanBlock = 1024, kScanItems = 4, kScanTile = kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(const uint32_t* __restrict__ in, uint64_t* __restrict__ out,
                                                           int64_t n, uint64_t* __restrict__ tile_sums) {
  __shared__ uint64_t warp_sums[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems], run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    run += v[i];
  }
  // inclusive scan of the per-thread totals across the block
  uint64_t x = run;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t w = warp_sums[lane];
    for (int off = 1; off < 32; off <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  uint64_t excl = x - run + (wid > 0 ? warp_sums[wid - 1] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == kScanBlock - 1) tile_sums[blockIdx.x] = excl;
}

// Single block: exclusive scan of the tile sums in place, total to *total.
__global__ void __launch_bounds__(1024) k_scan_sums(uint64_t* sums, int64_t m, uint64_t* total) {
  __shared__ uint64_t carry_s;
  __shared__ uint64_t warp_sums[32];
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t b = 0; b < m; b += 1024) {
    int64_t i = b + threadIdx.x;
    uint64_t v = i < m ? sums[i] : 0, x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = warp_sums[lane];
      for (int off = 1; off < 32; off <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    uint64_t incl = x + (wid > 0 ? warp_sums[wid - 1] : 0);
    uint64_t c = carry_s;
    if (i < m) sums[i] = c + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = c + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry_s;
}

__global__ void k_scan_add(uint64_t* __restrict__ out, int64_t n, const uint64_t* __restrict__ tile_sums) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_sums[i / kScanTile];
}
}  // namespace

pf_status pf_scan_u32(pf_ctx* ctx, const uint32_t* in, uint64_t* out, int64_t n) {
  int64_t tiles = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
  uint64_t* sums;
  PF_TRY(pf_scratch(ctx, WS_SCAN, (size_t)tiles * sizeof(uint64_t), (void**)&sums));
  k_scan_tiles<<<(unsigned)tiles, kScanBlock, 0, ctx->stream>>>(in, out, n, sums);
  k_scan_sums<<<1, 1024, 0, ctx->stream>>>(sums, tiles, out + n);
  if (n > 0) k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(out, n, sums);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

// ------------------------------------------------------------------ RMSE
namespace {
__global__ void k_sq_err(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* acc) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = (double)a[i] - (double)b[i];
    s += d * d;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) acc[blockIdx.x] = s;
  }
}
}  // namespace

extern "C" pf_status pf_image_rmse(pf_ctx* ctx, const float* a, const float* b, int64_t n, double* out_host) {
  if (!ctx || !a || !b || !out_host || n <= 0) return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad rmse arguments");
  DeviceGuard dg(ctx->device);
  int grid = std::max(1, std::min<int>((int)((n + 255) / 256), 512));
  k_sq_err<<<grid, 256, 0, ctx->stream>>>(a, b, n, ctx->dbl_dev);
  PF_CUDA(ctx, cudaGetLastError());
  std::vector<double> parts(grid);
  PF_CUDA(ctx, cudaMemcpyAsync(parts.data(), ctx->dbl_dev, grid * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double s = 0.0;
  for (double p : parts) s += p;  // fixed order: deterministic
  *out_host = std::sqrt(s / (double)n);
  return PF_OK;
}
