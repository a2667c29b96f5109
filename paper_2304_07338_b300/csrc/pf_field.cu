// Photon field network (Sec. 3.4), its training samples (Sec. 3.3) and its
// training loop (Sec. 3.5).
//
// This file holds the parts that are not tensor-core contractions:
//   * seeded Kaiming-uniform initialisation;
//   * the frequency encoding of the 6-D query, and the multiresolution
//     hash-grid encoding (forward, and its tables' gradient);
//   * a SIMT forward / backward (one thread per query, activations staged in
//     shared memory column-per-thread) that serves float32 fields and rounds
//     operands exactly as the tensor-core path specifies for the others;
//   * the training-sample generator and grid-cell radiance estimate;
//   * Adam and the training loop.
// The bf16 / fp16 / fp8 contractions run on tcgen05 (pf_mlp_tc.cu).
#include "pf_internal.h"
#include "pf_field_common.cuh"
#include <cmath>
#include <vector>
#include <algorithm>

using namespace pff;

// ------------------------------------------------------------------ init
namespace {
__device__ __forceinline__ void philox_block(uint64_t seed, uint32_t tag, uint64_t item, uint32_t sub, uint32_t block,
                                             uint32_t o[4]) {
  uint32_t x0 = (uint32_t)item, x1 = (uint32_t)(item >> 32), x2 = (tag << 24) | (sub & 0xFFFFFFu), x3 = block;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { a += 0x9E3779B9u; b += 0xBB67AE85u; }
    uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    uint32_t n0 = hi1 ^ x1 ^ a, n2 = hi0 ^ x3 ^ b;
    x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
  }
  o[0] = x0; o[1] = x1; o[2] = x2; o[3] = x3;
}

// w = (2u - 1) sqrt(6 / fan_in) in FP64, rounded once (Kaiming-uniform).
__global__ void k_init(float* w, int64_t off, int64_t n, int layer, int fan_in, uint64_t seed) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint32_t o[4];
  philox_block(seed, 4, (uint64_t)layer, 0, (uint32_t)(e / 4), o);
  double u = (double)(o[e % 4] >> 8) * (1.0 / 16777216.0);
  double bound = sqrt(6.0 / (double)fan_in);
  w[off + e] = (float)((2.0 * u - 1.0) * bound);
}

// Hash-grid tables: w = (2u - 1) 1e-4 (Philox tag 4, item 64 + 16 grid + level).
__global__ void k_init_table(float* w, int64_t off, int64_t n, int item, uint64_t seed) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint32_t o[4];
  philox_block(seed, 4, (uint64_t)item, 0, (uint32_t)(e / 4), o);
  double u = (double)(o[e % 4] >> 8) * (1.0 / 16777216.0);
  w[off + e] = (float)((2.0 * u - 1.0) * 1e-4);
}
}  // namespace

extern "C" pf_status pf_field_create(pf_ctx* ctx, const pf_field_desc* d, pf_field** out) {
  if (!ctx || !d || !out) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  *out = nullptr;
  if (d->in_freqs < 1 || d->in_freqs > 16) return pf_fail(ctx, PF_ERR_INVALID_ARG, "in_freqs must be in [1, 16]");
  if (d->hidden != 32 && d->hidden != 64 && d->hidden != 128)
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "hidden must be 32, 64 or 128");
  if (d->n_hidden < 1 || d->n_hidden > 8) return pf_fail(ctx, PF_ERR_INVALID_ARG, "n_hidden must be in [1, 8]");
  if (d->prec < 0 || d->prec > 3) return pf_fail(ctx, PF_ERR_INVALID_ARG, "unknown precision %d", d->prec);
  if (!(d->psi > 0.f)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "psi must be > 0");
  const bool hash = d->encoding == PF_ENC_HASHGRID;
  if (d->encoding != PF_ENC_FREQUENCY && !hash) return pf_fail(ctx, PF_ERR_INVALID_ARG, "unknown encoding");
  int hres[2][16] = {};
  if (hash) {
    const int F = d->hash_features;
    if (d->hash_levels < 1 || d->hash_levels > 16 || (F != 1 && F != 2 && F != 4 && F != 8) ||
        d->hash_log2_size < 4 || d->hash_log2_size > 24 || d->hash_base_res < 1 || d->hash_base_res > 65536 ||
        !(d->hash_scale >= 1.f && d->hash_scale <= 4.f))
      return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad hash-grid parameters");
    if (d->prec == PF_PREC_FP8) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "hash-grid fields are f32, bf16 or f16");
    double s = 1.0;
    for (int l = 0; l < d->hash_levels; ++l) {
      const double n = std::floor((double)d->hash_base_res * s);
      if (n > (double)(1 << 22)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "hash-grid level finer than 2^22 cells");
      hres[0][l] = hres[1][l] = (int)n;
      s *= (double)d->hash_scale;
    }
  }
  pf_field* f = new pf_field();
  f->ctx = ctx;
  f->device = ctx->device;
  f->desc = *d;
  f->n_in = hash ? 2 * d->hash_levels * d->hash_features + 1 : 12 * d->in_freqs;
  f->n_layers = d->n_hidden + 1;
  int64_t off = 0;
  for (int l = 0; l < f->n_layers; ++l) {
    f->fan_in[l] = l == 0 ? f->n_in : d->hidden;
    f->fan_out[l] = l == f->n_layers - 1 ? 3 : d->hidden;
    f->layer_off[l] = off;
    off += (int64_t)f->fan_in[l] * f->fan_out[l];
  }
  f->layer_off[f->n_layers] = off;
  if (hash) {
    off = (off + 7) / 8 * 8;
    const double T = std::ldexp(1.0, d->hash_log2_size);
    for (int gi = 0; gi < 2; ++gi) {
      const int D = gi == 0 ? 3 : 2;
      for (int l = 0; l < d->hash_levels; ++l) {
        const int N = hres[gi][l];
        const double verts = std::pow((double)N + 1.0, D);
        const bool dense = verts <= T;
        f->hash_res[gi][l] = N;
        f->hash_entries[gi][l] = (uint32_t)(dense ? verts : T);
        if (dense) f->hash_dense[gi] |= 1u << l;
        f->hash_off[gi][l] = off;
        off += ((int64_t)f->hash_entries[gi][l] * d->hash_features + 7) / 8 * 8;
      }
    }
  }
  f->n_params = off;
  size_t bytes = (size_t)off * sizeof(float);
  if (cudaMalloc(&f->w, bytes) != cudaSuccess || cudaMalloc(&f->m, bytes) != cudaSuccess ||
      cudaMalloc(&f->v, bytes) != cudaSuccess || cudaMalloc(&f->scales, 64 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(f->w); cudaFree(f->m); cudaFree(f->v); cudaFree(f->scales);
    delete f;
    return pf_fail(ctx, PF_ERR_OOM, "field allocation failed");
  }
  cudaMemsetAsync(f->w, 0, bytes, ctx->stream);
  cudaMemsetAsync(f->m, 0, bytes, ctx->stream);
  cudaMemsetAsync(f->v, 0, bytes, ctx->stream);
  cudaMemsetAsync(f->scales, 0, 64 * sizeof(float), ctx->stream);
  for (int l = 0; l < f->n_layers; ++l) {
    int64_t n = (int64_t)f->fan_in[l] * f->fan_out[l];
    k_init<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(f->w, f->layer_off[l], n, l, f->fan_in[l], d->seed);
  }
  if (hash)
    for (int gi = 0; gi < 2; ++gi)
      for (int l = 0; l < d->hash_levels; ++l) {
        const int64_t n = (int64_t)f->hash_entries[gi][l] * d->hash_features;
        k_init_table<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(f->w, f->hash_off[gi][l], n,
                                                                           64 + 16 * gi + l, d->seed);
      }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { pf_field_free(f); return pf_cuda_check(ctx, e, "field init"); }
  pf_status st = pf_field_pack(ctx, f);
  if (st != PF_OK) { pf_field_free(f); return st; }
  *out = f;
  return PF_OK;
}

extern "C" pf_status pf_field_free(pf_field* f) {
  if (!f) return PF_OK;
  DeviceGuard dg(f->device);
  cudaDeviceSynchronize();
  cudaFree(f->w); cudaFree(f->m); cudaFree(f->v); cudaFree(f->wq); cudaFree(f->wr); cudaFree(f->scales);
  delete f;
  return PF_OK;
}

extern "C" int64_t pf_field_num_params(const pf_field* f) { return f ? f->n_params : -1; }

extern "C" pf_status pf_field_get_weights(pf_ctx* ctx, const pf_field* f, float* dst) {
  if (!ctx || !f || !dst) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_CUDA(ctx, cudaMemcpyAsync(dst, f->w, f->n_params * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  return PF_OK;
}

extern "C" pf_status pf_field_set_weights(pf_ctx* ctx, pf_field* f, const float* src) {
  if (!ctx || !f || !src) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_CUDA(ctx, cudaMemcpyAsync(f->w, src, f->n_params * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  f->fp8_ready = 0;
  return pf_field_pack(ctx, f);
}

// ------------------------------------------------------------------ SIMT forward / backward
namespace {

struct FieldView {
  const float* w;     // master weights (output layer read from here)
  const float* wr;    // hidden layers rounded to the field precision
  int64_t off[10];
  int fan_in[10], fan_out[10];
  int n_layers, n_in, hidden, in_freqs, prec;
  float psi;
  float s_a[8], s_w[8];
  // hash-grid encoding (enc == PF_ENC_HASHGRID); vec: the gradient buffer is
  // 16-byte aligned, so entries of 4 or 8 features take vector atomics
  int enc, hl, hf, vec;
  int hres[2][16];
  uint32_t hent[2][16];
  uint32_t hdense[2];
  int64_t hoff[2][16];
};

FieldView view_of(const pf_field* f) {
  FieldView v;
  v.w = f->w;
  v.wr = f->wr ? f->wr : f->w;
  for (int l = 0; l <= f->n_layers && l < 10; ++l) v.off[l] = f->layer_off[l];
  for (int l = 0; l < f->n_layers; ++l) { v.fan_in[l] = f->fan_in[l]; v.fan_out[l] = f->fan_out[l]; }
  v.n_layers = f->n_layers; v.n_in = f->n_in; v.hidden = f->desc.hidden; v.in_freqs = f->desc.in_freqs;
  v.prec = f->desc.prec; v.psi = f->desc.psi;
  for (int l = 0; l < 8; ++l) { v.s_a[l] = f->scales_host[l]; v.s_w[l] = f->scales_host[16 + l]; }
  v.enc = f->desc.encoding;
  v.vec = 0;
  v.hl = f->desc.hash_levels;
  v.hf = f->desc.hash_features;
  for (int gi = 0; gi < 2; ++gi) {
    v.hdense[gi] = f->hash_dense[gi];
    for (int l = 0; l < 16; ++l) {
      v.hres[gi][l] = f->hash_res[gi][l];
      v.hent[gi][l] = f->hash_entries[gi][l];
      v.hoff[gi][l] = f->hash_off[gi][l];
    }
  }
  return v;
}

// ---- multiresolution hash grids (Sec. 3.4): grid gi (0: x, y, z; 1: theta',
// phi'), level l.  The cell holding x: p = clamp(x, 0, 1) * N_l in float32,
// i = min(floor(p), N_l - 1), fraction p - i (exact).
template <int D>
__device__ __forceinline__ void hash_cell(const FieldView& F, int gi, int l, const float* x, uint32_t i0[D],
                                          float fr[D]) {
  const int N = F.hres[gi][l];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float p = __fmul_rn(fminf(fmaxf(x[k], 0.f), 1.f), (float)N);
    const int i = min((int)floorf(p), N - 1);
    i0[k] = (uint32_t)i;
    fr[k] = __fsub_rn(p, (float)i);
  }
}

// Table entry of corner c (bit k: +1 along axis k): dense x-fastest index, or
// the spatial hash xor_k v_k pi_k (pi = 1, 2654435761, 805459861) modulo the
// table size (a power of two).
template <int D>
__device__ __forceinline__ uint32_t hash_index(const FieldView& F, int gi, int l, const uint32_t i0[D], int c) {
  uint32_t v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = i0[k] + ((c >> k) & 1);
  if ((F.hdense[gi] >> l) & 1u) {
    const uint32_t n1 = (uint32_t)F.hres[gi][l] + 1u;
    uint32_t idx = v[D - 1];
#pragma unroll
    for (int k = D - 2; k >= 0; --k) idx = idx * n1 + v[k];
    return idx;
  }
  uint32_t h = v[0] ^ (v[1] * 2654435761u);
  if (D == 3) h ^= v[D - 1] * 805459861u;
  return h & (F.hent[gi][l] - 1u);
}

// Multilinear weight of corner c: prod_k (bit k ? f_k : 1 - f_k).
template <int D>
__device__ __forceinline__ float corner_weight(const float fr[D], int c) {
  float w = 1.f;
#pragma unroll
  for (int k = 0; k < D; ++k) w *= ((c >> k) & 1) ? fr[k] : 1.f - fr[k];
  return w;
}

// The F features of level l of grid gi at x.
template <int D>
__device__ __forceinline__ void hash_features(const FieldView& F, int gi, int l, const float* x, float acc[8]) {
  uint32_t i0[D];
  float fr[D];
  hash_cell<D>(F, gi, l, x, i0, fr);
  const float* tab = F.w + F.hoff[gi][l];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = 0.f;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    const float* e = tab + (size_t)hash_index<D>(F, gi, l, i0, c) * F.hf;
    const float w = corner_weight<D>(fr, c);
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F.hf) acc[f] = fmaf(w, __ldg(e + f), acc[f]);
  }
}

// Spreads the gradient dx of level l's features over its corners' entries.
template <int D>
__device__ __forceinline__ void hash_scatter(const FieldView& F, int gi, int l, const float* x, const float dx[8],
                                             float* dw) {
  uint32_t i0[D];
  float fr[D];
  hash_cell<D>(F, gi, l, x, i0, fr);
  float* tab = dw + F.hoff[gi][l];
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    float* e = tab + (size_t)hash_index<D>(F, gi, l, i0, c) * F.hf;
    const float w = corner_weight<D>(fr, c);
    if (F.vec && F.hf >= 4) {
      // entries of 4 or 8 features start on 16-byte boundaries (level tables
      // on 8-float boundaries): vector atomics
      atomicAdd((float4*)e, make_float4(w * dx[0], w * dx[1], w * dx[2], w * dx[3]));
      if (F.hf == 8) atomicAdd((float4*)e + 1, make_float4(w * dx[4], w * dx[5], w * dx[6], w * dx[7]));
    } else {
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (f < F.hf) atomicAdd(e + f, w * dx[f]);
    }
  }
}

// MLP input of a hash-grid field: [position levels, direction levels, g],
// F features per level; column k of the thread's query goes to buf[k * T + tid].
template <int T>
__device__ __forceinline__ void hash_encode(const FieldView& F, const float* q, int tid, float* buf) {
  const int LF = F.hl * F.hf;
  for (int gi = 0; gi < 2; ++gi)
    for (int l = 0; l < F.hl; ++l) {
      float acc[8];
      if (gi == 0) hash_features<3>(F, 0, l, q, acc);
      else hash_features<2>(F, 1, l, q + 3, acc);
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (f < F.hf) buf[(gi * LF + l * F.hf + f) * T + tid] = acc[f];
    }
  buf[(2 * LF) * T + tid] = q[5];
}

constexpr int kSimtThreads = 64;   // forward: queries per block
constexpr int kBwdThreads = 32;    // backward: queries per block (one warp)
constexpr int kMaxK = 272;         // MLP inputs: 12 * 16 frequencies, or 2 * 16 * 8 + 1 hash-grid features

// Operand rounding of the hidden layers (see pf_field_common.cuh).
__device__ __forceinline__ float rin(float x, int prec, float s) { return round_prec(x, prec, s); }

// Forward for one block of T queries; activations column-per-thread in
// shared memory: buf[k * T + tid].  Returns the 3 outputs in y.  If keep is
// given, the (rounded) input of layer l is kept at keep[(koff[l] + k) * T + tid].
template <int T>
__device__ void simt_forward(const FieldView& F, const float* q, int tid, float* bufA, float* bufB, float* keep,
                             const int* koff, float y[3]) {
  // encoding -> bufA (rounded to the first layer's input precision)
  if (F.enc == PF_ENC_HASHGRID) hash_encode<T>(F, q, tid, bufA);
  else for (int d = 0; d < 6; ++d) {
    float v = q[d];
    for (int k = 0; k < F.in_freqs; ++k) {
      float s, c;
      sincospif(ldexpf(v, k), &s, &c);
      int idx = d * 2 * F.in_freqs + 2 * k;
      bufA[idx * T + tid] = s;
      bufA[(idx + 1) * T + tid] = c;
    }
  }
  float* in = bufA;
  float* outb = bufB;
  for (int l = 0; l < F.n_layers; ++l) {
    const bool last = (l == F.n_layers - 1);
    const int K = F.fan_in[l], N = F.fan_out[l];
    const float* W = (last ? F.w : F.wr) + F.off[l];
    if (!last) {
      for (int k = 0; k < K; ++k) {
        float r = rin(in[k * T + tid], F.prec, F.s_a[l]);
        in[k * T + tid] = r;
        if (keep) keep[((size_t)koff[l] + k) * T + tid] = r;
      }
    } else if (keep) {
      for (int k = 0; k < K; ++k) keep[((size_t)koff[l] + k) * T + tid] = in[k * T + tid];
    }
    for (int n = 0; n < N; ++n) {
      float acc = 0.f;
      const float* wr = W + (size_t)n * K;
      for (int k = 0; k < K; ++k) acc = fmaf(in[k * T + tid], __ldg(wr + k), acc);
      if (last) y[n] = acc;
      else outb[n * T + tid] = fmaxf(acc, 0.f);
    }
    float* t = in; in = outb; outb = t;
  }
}

__global__ void __launch_bounds__(kSimtThreads) k_simt_forward(FieldView F, const float* __restrict__ q, int64_t B_max,
                                                             const uint32_t* __restrict__ B_dev, float* __restrict__ out,
                                                             const uint32_t* __restrict__ slot_idx,
                                                             const float* __restrict__ slot_alb, float* __restrict__ slot_li) {
  extern __shared__ float sm[];
  float* bufA = sm;
  float* bufB = sm + kMaxK * kSimtThreads;
  int64_t B = B_dev ? (int64_t)*B_dev : B_max;
  int64_t b = (int64_t)blockIdx.x * kSimtThreads + threadIdx.x;
  if ((int64_t)blockIdx.x * kSimtThreads >= B) return;
  float qq[6];
  bool act = b < B;
  for (int d = 0; d < 6; ++d) qq[d] = act ? q[6 * b + d] : 0.5f;
  float y[3];
  simt_forward<kSimtThreads>(F, qq, threadIdx.x, bufA, bufB, nullptr, nullptr, y);
  if (!act) return;
  if (slot_idx) {
    uint32_t s = slot_idx[b];
    for (int c = 0; c < 3; ++c) slot_li[3 * (size_t)s + c] = slot_alb[3 * b + c] * exp10f(-F.psi * y[c]);
  } else {
    for (int c = 0; c < 3; ++c) out[3 * b + c] = y[c];
  }
}

// Backward: each thread recomputes its forward, keeps every layer's input,
// back-propagates dy and accumulates its dW contribution into shared memory
// partials that are added to global dW once per block.
// loss mode (targets != nullptr): the mean relative MSE's gradient with loss
// scaling -- the pass runs on dy = 2 (yhat - y) / (y^2 + 0.01), 3B times the
// gradient of the mean, so that its rounded intermediate gradients stay in
// the normal range of a 16-bit field precision, and the block's float32 dW
// contributions are multiplied by inv_n = 1/(3B); the block's loss sum goes
// to *loss.
__global__ void __launch_bounds__(kBwdThreads) k_simt_backward(FieldView F, const float* __restrict__ q,
                                                            const float* __restrict__ dy_in,
                                                            const float* __restrict__ targets, float inv_n,
                                                            int64_t B, float* __restrict__ dw, float* loss) {
  constexpr int T = kBwdThreads;
  extern __shared__ float sm[];
  int koff[10];
  int rows = 0;
  for (int l = 0; l < F.n_layers; ++l) { koff[l] = rows; rows += F.fan_in[l]; }
  int kmax = F.n_in > F.hidden ? F.n_in : F.hidden;
  float* bufA = sm;
  float* bufB = bufA + (size_t)kmax * T;
  float* keep = bufB + (size_t)kmax * T;
  float* dcur = keep + (size_t)rows * T;
  float* dnext = dcur + (size_t)kmax * T;
  int tid = threadIdx.x;
  int64_t b = (int64_t)blockIdx.x * T + tid;
  bool act = b < B;
  float qq[6];
  for (int d = 0; d < 6; ++d) qq[d] = act ? q[6 * b + d] : 0.5f;
  float y[3];
  simt_forward<T>(F, qq, tid, bufA, bufB, keep, koff, y);
  float g[3] = {0.f, 0.f, 0.f};
  float lsum = 0.f;
  if (act) {
    if (targets) {
      for (int c = 0; c < 3; ++c) {
        float t = targets[3 * b + c];
        float den = t * t + 0.01f;
        float diff = y[c] - t;
        lsum += diff * diff / den;
        g[c] = 2.f * diff / den;
      }
    } else {
      for (int c = 0; c < 3; ++c) g[c] = dy_in[3 * b + c];
    }
  }
  const float gscale = targets ? inv_n : 1.f;     // undoes the loss scaling in float32
  if (loss) {
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if (tid == 0) atomicAdd(loss, lsum * inv_n);
  }
  for (int c = 0; c < 3; ++c) dcur[c * T + tid] = g[c];
  for (int l = F.n_layers - 1; l >= 0; --l) {
    const bool last = (l == F.n_layers - 1);
    const int K = F.fan_in[l], N = F.fan_out[l];
    const float* W = (last ? F.w : F.wr) + F.off[l];
    const float* xin = keep + (size_t)koff[l] * T;
    __syncwarp();
    // dW[n][k] += sum over the block's queries of dcur[n] * xin[k]
    for (int e = tid; e < N * K; e += T) {
      int n = e / K, k = e % K;
      float s = 0.f;
      for (int t = 0; t < T; ++t) s = fmaf(dcur[n * T + t], xin[k * T + t], s);
      atomicAdd(&dw[F.off[l] + e], s * gscale);
    }
    if (l == 0) {
      if (F.enc == PF_ENC_HASHGRID && act) {
        // input gradient W_0^T dcur, level by level, spread over the corners
        const float* W0 = F.wr + F.off[0];
        const int LF = F.hl * F.hf;
        for (int gi = 0; gi < 2; ++gi)
          for (int lv = 0; lv < F.hl; ++lv) {
            const int col = gi * LF + lv * F.hf;
            float dx[8];
#pragma unroll
            for (int f = 0; f < 8; ++f) {
              float a = 0.f;
              if (f < F.hf)
                for (int n = 0; n < N; ++n) a = fmaf(dcur[n * T + tid], __ldg(W0 + (size_t)n * K + col + f), a);
              dx[f] = a * gscale;
            }
            if (gi == 0) hash_scatter<3>(F, 0, lv, qq, dx, dw);
            else hash_scatter<2>(F, 1, lv, qq + 3, dx, dw);
          }
      }
      break;
    }
    // gradient w.r.t. the input of layer l: W^T dcur, masked by the ReLU of
    // layer l-1 (taken from the rounded activation) and rounded
    for (int k = 0; k < K; ++k) {
      float acc = 0.f;
      for (int n = 0; n < N; ++n) {
        acc = fmaf(dcur[n * T + tid], __ldg(W + (size_t)n * K + k), acc);
      }
      float a = xin[k * T + tid];
      float m = rin(a, F.prec, 1.f) > 0.f ? 1.f : 0.f;
      dnext[k * T + tid] = rin(acc * m, F.prec, 1.f);
    }
    __syncwarp();
    float* t = dcur; dcur = dnext; dnext = t;
  }
}

size_t simt_fwd_smem() { return 2 * kMaxK * kSimtThreads * sizeof(float); }
size_t simt_bwd_smem(const pf_field* f) {
  int kmax = std::max(f->n_in, f->desc.hidden);
  int64_t rows = 4 * (int64_t)kmax + (f->layer_off[f->n_layers] > 0 ? 0 : 0);
  for (int l = 0; l < f->n_layers; ++l) rows += f->fan_in[l];
  return (size_t)rows * kBwdThreads * sizeof(float);
}

}  // namespace

pf_status pf_simt_forward(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B_max, const uint32_t* B_dev,
                          float* out, const uint32_t* slot_idx, const float* slot_alb, float* slot_li) {
  if (B_max <= 0) return PF_OK;
  FieldView F = view_of(f);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_simt_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)simt_fwd_smem());
    attr = true;
  }
  unsigned grid = (unsigned)((B_max + kSimtThreads - 1) / kSimtThreads);
  k_simt_forward<<<grid, kSimtThreads, simt_fwd_smem(), ctx->stream>>>(F, q, B_max, B_dev, out, slot_idx, slot_alb, slot_li);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

pf_status pf_simt_backward(pf_ctx* ctx, const pf_field* f, const float* q, const float* dy, const float* targets,
                           int64_t B, float* dw, float* loss) {
  FieldView F = view_of(f);
  F.vec = ((uintptr_t)dw & 15) == 0;
  size_t sm = simt_bwd_smem(f);
  if (sm > 227 * 1024) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "SIMT backward: network too deep for shared memory");
  cudaFuncSetAttribute(k_simt_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  unsigned grid = (unsigned)((B + kBwdThreads - 1) / kBwdThreads);
  float inv_n = targets ? 1.0f / (float)(3 * B) : 0.f;
  k_simt_backward<<<grid, kBwdThreads, sm, ctx->stream>>>(F, q, dy, targets, inv_n, B, dw, loss);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

// ------------------------------------------------------------------ fp8 calibration
namespace {
// amax of every hidden layer's input over the calibration queries, from the
// unquantised float forward pass (one thread per query).
__global__ void __launch_bounds__(kSimtThreads) k_calib(FieldView F, const float* __restrict__ q, int64_t B,
                                                      unsigned int* amax) {
  extern __shared__ float sm[];
  float* bufA = sm;
  float* bufB = sm + kMaxK * kSimtThreads;
  int tid = threadIdx.x;
  int64_t b = (int64_t)blockIdx.x * kSimtThreads + tid;
  bool act = b < B;
  for (int d = 0; d < 6; ++d) {
    float v = act ? q[6 * b + d] : 0.f;
    for (int k = 0; k < F.in_freqs; ++k) {
      float s, c;
      sincospif(ldexpf(v, k), &s, &c);
      int idx = d * 2 * F.in_freqs + 2 * k;
      bufA[idx * kSimtThreads + tid] = act ? s : 0.f;
      bufA[(idx + 1) * kSimtThreads + tid] = act ? c : 0.f;
    }
  }
  float* in = bufA;
  float* outb = bufB;
  for (int l = 0; l < F.n_layers - 1; ++l) {
    const int K = F.fan_in[l], N = F.fan_out[l];
    float m = 0.f;
    for (int k = 0; k < K; ++k) m = fmaxf(m, fabsf(in[k * kSimtThreads + tid]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((tid & 31) == 0) atomicMax(&amax[l], __float_as_uint(m));
    const float* W = F.w + F.off[l];
    for (int n = 0; n < N; ++n) {
      float acc = 0.f;
      for (int k = 0; k < K; ++k) acc = fmaf(in[k * kSimtThreads + tid], __ldg(W + (size_t)n * K + k), acc);
      outb[n * kSimtThreads + tid] = fmaxf(acc, 0.f);
    }
    float* t = in; in = outb; outb = t;
  }
}

__global__ void k_wamax(const float* __restrict__ w, int64_t off, int64_t n, unsigned int* amax) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(w[off + i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}
}  // namespace

extern "C" pf_status pf_field_calibrate_fp8(pf_ctx* ctx, pf_field* f, const float* q, int64_t B) {
  if (!ctx || !f || !q || B <= 0) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  unsigned int* amax;
  PF_TRY(pf_scratch(ctx, WS_REDUCE, 64 * sizeof(unsigned int), (void**)&amax));
  PF_CUDA(ctx, cudaMemsetAsync(amax, 0, 64 * sizeof(unsigned int), ctx->stream));
  FieldView F = view_of(f);
  cudaFuncSetAttribute(k_calib, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)simt_fwd_smem());
  k_calib<<<(unsigned)((B + kSimtThreads - 1) / kSimtThreads), kSimtThreads, simt_fwd_smem(), ctx->stream>>>(F, q, B, amax);
  for (int l = 0; l < f->n_layers - 1; ++l) {
    int64_t n = (int64_t)f->fan_in[l] * f->fan_out[l];
    k_wamax<<<64, 256, 0, ctx->stream>>>(f->w, f->layer_off[l], n, amax + 16 + l);
  }
  PF_CUDA(ctx, cudaGetLastError());
  unsigned int h[64];
  PF_CUDA(ctx, cudaMemcpyAsync(h, amax, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // power-of-two scales 2^ceil(log2(amax / 448)): dividing by them is exact
  auto pow2_scale = [](float amax) {
    int e;
    float m = std::frexp(std::max(amax, 1e-30f) / 448.0f, &e);
    return std::ldexp(1.0f, m == 0.5f ? e - 1 : e);
  };
  for (int l = 0; l < f->n_layers - 1; ++l) {
    float a, w;
    memcpy(&a, &h[l], 4);
    memcpy(&w, &h[16 + l], 4);
    f->scales_host[l] = pow2_scale(a);
    f->scales_host[16 + l] = pow2_scale(w);
  }
  PF_CUDA(ctx, cudaMemcpyAsync(f->scales, f->scales_host, 32 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  f->fp8_ready = 1;
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return pf_field_pack(ctx, f);
}

// ------------------------------------------------------------------ public forward / backward
pf_status pf_tc_available(const pf_field* f);
pf_status pf_tc_backward_available(const pf_field* f);
pf_status pf_tc_forward(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B_max, const uint32_t* B_dev, float* out,
                        const uint32_t* slot_idx, const float* slot_alb, float* slot_li);
pf_status pf_tc_backward(pf_ctx* ctx, const pf_field* f, const float* q, const float* dy, const float* targets,
                         int64_t B, float* dw, float* loss, const uint16_t* x_in, float* dx_out);

namespace {
// Hash-grid features of the tensor-core training step: one thread per
// (query, grid, level); the level's F features rounded to the field
// precision at x[b][(grid * L + level) * F ...] (x: [B][2 L F] 16-bit).
template <int PREC>
__global__ void k_hash_features(FieldView F, const float* __restrict__ q, int64_t B, uint16_t* __restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = 2 * F.hl;
  if (t >= B * per) return;
  const int64_t b = t / per;
  const int j = (int)(t % per), gi = j / F.hl, l = j % F.hl;
  float v[3];
  for (int k = 0; k < 3; ++k) v[k] = q[6 * b + (gi == 0 ? k : 3 + (k < 2 ? k : 1))];
  float acc[8];
  if (gi == 0) hash_features<3>(F, 0, l, v, acc);
  else hash_features<2>(F, 1, l, v, acc);
  uint16_t* dst = x + (size_t)b * (2 * F.hl * F.hf) + (size_t)j * F.hf;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f >= F.hf) break;
    dst[f] = PREC == PF_PREC_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(acc[f]))
                                  : __half_as_ushort(__float2half_rn(acc[f]));
  }
}

// Spreads the features' gradient dx [B][2 L F] over the level tables' corners
// (one thread per (query, grid, level)).
__global__ void k_hash_scatter(FieldView F, const float* __restrict__ q, const float* __restrict__ dx, int64_t B,
                               float scale, float* __restrict__ dw) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = 2 * F.hl;
  if (t >= B * per) return;
  const int64_t b = t / per;
  const int j = (int)(t % per), gi = j / F.hl, l = j % F.hl;
  float v[3];
  for (int k = 0; k < 3; ++k) v[k] = q[6 * b + (gi == 0 ? k : 3 + (k < 2 ? k : 1))];
  const float* src = dx + (size_t)b * (2 * F.hl * F.hf) + (size_t)j * F.hf;
  float d[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) d[f] = f < F.hf ? src[f] * scale : 0.f;
  if (gi == 0) hash_scatter<3>(F, 0, l, v, d, dw);
  else hash_scatter<2>(F, 1, l, v, d, dw);
}
}  // namespace

pf_status pf_field_forward_impl(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B_max, const uint32_t* B_dev,
                                float* out, const uint32_t* slot_idx, const float* slot_alb, float* slot_li) {
  if (f->desc.prec == PF_PREC_FP8 && !f->fp8_ready)
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "fp8 field: call pf_field_calibrate_fp8 first");
  if (pf_tc_available(f) == PF_OK) return pf_tc_forward(ctx, f, q, B_max, B_dev, out, slot_idx, slot_alb, slot_li);
  return pf_simt_forward(ctx, f, q, B_max, B_dev, out, slot_idx, slot_alb, slot_li);
}

// gamma of one (query, input) pair per thread; a warp's 32 pairs own one
// contiguous range of 64 F floats, so each lane stages its 2F features in
// shared memory (rows padded to 2F + 1 floats: no bank conflicts) and the
// warp then writes the range with consecutive lanes on consecutive floats.
__global__ void k_field_encode(const float* __restrict__ q, int64_t n_pairs, int F, float* __restrict__ out) {
  extern __shared__ float pf_enc_stage[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = 2 * F, Wp = W + 1;
  float* st = pf_enc_stage + warp * 32 * Wp;
  const float inv_w = 1.0f / (float)W;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < n_pairs;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;          // pair i = (query i / 6, input i % 6)
    if (i < n_pairs) {
      const float v = __ldg(q + i);
      float s = 0.f, c = 1.f;
      for (int k = 0; k < F; ++k) {
        pff::freq_next(v, k, s, c);
        st[lane * Wp + 2 * k] = s;
        st[lane * Wp + 2 * k + 1] = c;
      }
    }
    __syncwarp();
    const int n_out = (int)(n_pairs - base < 32 ? n_pairs - base : 32) * W;
    float* o = out + base * W;
    for (int e = lane; e < n_out; e += 32) {
      const int r = (int)(((float)e + 0.5f) * inv_w);   // e / W (e < 1024: the float quotient cannot cross an integer)
      o[e] = st[r * Wp + (e - r * W)];
    }
    __syncwarp();
  }
}

extern "C" pf_status pf_field_encode(pf_ctx* ctx, const float* q, int64_t B, int F, float* out) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  if (B < 0 || F < 1 || F > 16) return pf_fail(ctx, PF_ERR_INVALID_ARG, "need B >= 0 and 1 <= in_freqs <= 16");
  if (B == 0) return PF_OK;
  if (!q || !out) return pf_fail(ctx, PF_ERR_INVALID_ARG, "q_dev and out_dev must not be NULL");
  DeviceGuard dg(ctx->device);
  const int64_t n = B * 6;
  const size_t smem = (size_t)8 * 32 * (2 * F + 1) * sizeof(float);   // 8 warps per block
  k_field_encode<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8), 256, smem, ctx->stream>>>(
      q, n, F, out);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

extern "C" pf_status pf_field_forward(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B, float* out) {
  if (!ctx || !f || B < 0) return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad field forward arguments");
  if (B == 0) return PF_OK;
  if (!q || !out) return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad field forward arguments");
  if (f->ctx != ctx) return pf_fail(ctx, PF_ERR_INVALID_ARG, "field belongs to another context");
  DeviceGuard dg(ctx->device);
  return pf_field_forward_impl(ctx, f, q, B, nullptr, out, nullptr, nullptr, nullptr);
}

pf_status pf_field_backward_impl(pf_ctx* ctx, const pf_field* f, const float* q, const float* dy, const float* targets,
                                 int64_t B, float* dw, float* loss) {
  if (f->desc.prec == PF_PREC_FP8) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "fp8 fields are inference-only");
  if (B > 0 && pf_tc_backward_available(f) == PF_OK) {
    if (f->desc.encoding != PF_ENC_HASHGRID)   // the tensor-core backward writes every element of dw
      return pf_tc_backward(ctx, f, q, dy, targets, B, dw, loss, nullptr, nullptr);
    // hash grids: table features (gather), the MLP on tcgen05 (which writes
    // the MLP's dW and the features' gradient), then the table scatter
    FieldView F = view_of(f);
    F.vec = ((uintptr_t)dw & 15) == 0;
    const int nf = 2 * F.hl * F.hf;
    uint16_t* x;
    float* dx;
    PF_TRY(pf_scratch(ctx, WS_HASH_X, (size_t)B * nf * sizeof(uint16_t), (void**)&x));
    PF_TRY(pf_scratch(ctx, WS_HASH_DX, (size_t)B * nf * sizeof(float), (void**)&dx));
    const int64_t n_thr = B * 2 * F.hl;
    const unsigned grid = (unsigned)((n_thr + 255) / 256);
    if (f->desc.prec == PF_PREC_BF16) k_hash_features<PF_PREC_BF16><<<grid, 256, 0, ctx->stream>>>(F, q, B, x);
    else k_hash_features<PF_PREC_F16><<<grid, 256, 0, ctx->stream>>>(F, q, B, x);
    PF_CUDA(ctx, cudaGetLastError());
    const int64_t n_mlp = f->layer_off[f->n_layers];
    PF_CUDA(ctx, cudaMemsetAsync(dw + n_mlp, 0, (size_t)(f->n_params - n_mlp) * sizeof(float), ctx->stream));
    PF_TRY(pf_tc_backward(ctx, f, q, dy, targets, B, dw, loss, x, dx));
    // loss mode: the features' gradient is loss-scaled like dW (see below)
    k_hash_scatter<<<grid, 256, 0, ctx->stream>>>(F, q, dx, B, targets ? 1.0f / (float)(3 * B) : 1.0f, dw);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  }
  PF_CUDA(ctx, cudaMemsetAsync(dw, 0, f->n_params * sizeof(float), ctx->stream));
  if (B == 0) return PF_OK;
  return pf_simt_backward(ctx, f, q, dy, targets, B, dw, loss);
}

extern "C" pf_status pf_field_backward(pf_ctx* ctx, const pf_field* f, const float* q, const float* dy, int64_t B,
                                       float* dw) {
  if (!ctx || !f || !dw || B < 0 || (B > 0 && (!q || !dy)))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad field backward arguments");
  if (f->ctx != ctx) return pf_fail(ctx, PF_ERR_INVALID_ARG, "field belongs to another context");
  DeviceGuard dg(ctx->device);
  return pf_field_backward_impl(ctx, f, q, dy, nullptr, B, dw, nullptr);
}

extern "C" pf_status pf_field_loss_gradient(pf_ctx* ctx, const pf_field* f, const float* q, const float* targets,
                                            int64_t B, float* dw, float* loss_host) {
  if (!ctx || !f || !dw || B <= 0 || !q || !targets)
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad field loss-gradient arguments");
  if (f->ctx != ctx) return pf_fail(ctx, PF_ERR_INVALID_ARG, "field belongs to another context");
  DeviceGuard dg(ctx->device);
  float* loss;
  PF_TRY(pf_scratch(ctx, WS_LOSS, sizeof(float), (void**)&loss));
  PF_CUDA(ctx, cudaMemsetAsync(loss, 0, sizeof(float), ctx->stream));
  PF_TRY(pf_field_backward_impl(ctx, f, q, nullptr, targets, B, dw, loss));
  if (loss_host) {
    PF_CUDA(ctx, cudaMemcpyAsync(loss_host, loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    PF_TRY(pf_check_error_word(ctx));
  }
  return PF_OK;
}

// ------------------------------------------------------------------ Adam
namespace {
__device__ __forceinline__ void adam1(float& w, float& m, float& v, float g, float lr, float b1, float b2, float eps,
                                      float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  const float mh = m / c1, vh = v / c2;
  w = w - lr * mh / (sqrtf(vh) + eps);
}

// One Adam update per parameter; four per thread (16-byte accesses) when the
// arrays allow it (hash-grid fields carry ~10^8 parameters).
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  if (!isfinite(gi)) { atomicOr(err, 2u); return; }
  adam1(w[i], m[i], v[i], gi, lr, b1, b2, eps, c1, c2);
}

__global__ void k_adam4(float4* __restrict__ w, float4* __restrict__ m, float4* __restrict__ v,
                        const float4* __restrict__ g, int64_t n4, float lr, float b1, float b2, float eps, float c1,
                        float c2, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 gi = g[i];
  if (!isfinite(gi.x) || !isfinite(gi.y) || !isfinite(gi.z) || !isfinite(gi.w)) { atomicOr(err, 2u); return; }
  float4 wi = w[i], mi = m[i], vi = v[i];
  adam1(wi.x, mi.x, vi.x, gi.x, lr, b1, b2, eps, c1, c2);
  adam1(wi.y, mi.y, vi.y, gi.y, lr, b1, b2, eps, c1, c2);
  adam1(wi.z, mi.z, vi.z, gi.z, lr, b1, b2, eps, c1, c2);
  adam1(wi.w, mi.w, vi.w, gi.w, lr, b1, b2, eps, c1, c2);
  w[i] = wi; m[i] = mi; v[i] = vi;
}
}  // namespace

pf_status pf_adam_impl(pf_ctx* ctx, pf_field* f, const float* g, float lr, float b1, float b2, float eps) {
  f->step += 1;
  float c1 = (float)(1.0 - std::pow((double)b1, f->step));
  float c2 = (float)(1.0 - std::pow((double)b2, f->step));
  const bool vec = f->n_params % 4 == 0 && ((uintptr_t)g & 15) == 0;
  if (vec)
    k_adam4<<<(unsigned)((f->n_params / 4 + 255) / 256), 256, 0, ctx->stream>>>(
        (float4*)f->w, (float4*)f->m, (float4*)f->v, (const float4*)g, f->n_params / 4, lr, b1, b2, eps, c1, c2,
        ctx->err_dev);
  else
    k_adam<<<(unsigned)((f->n_params + 255) / 256), 256, 0, ctx->stream>>>(f->w, f->m, f->v, g, f->n_params, lr, b1,
                                                                           b2, eps, c1, c2, ctx->err_dev);
  PF_CUDA(ctx, cudaGetLastError());
  return pf_field_pack(ctx, f);
}

extern "C" pf_status pf_field_adam(pf_ctx* ctx, pf_field* f, const float* g, float lr, float b1, float b2, float eps) {
  if (!ctx || !f || !g) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  return pf_adam_impl(ctx, f, g, lr, b1, b2, eps);
}

// ------------------------------------------------------------------ training samples
namespace {
struct CacheView {
  const uint64_t* offsets;
  const float4* recs;
  const uint32_t* occupied;
  const float* cell_sigma;
  int64_t n_occupied;
  int res, n_lights, n_g;
  float g_set[16];
};

CacheView cview(const pf_cache* c) {
  CacheView v;
  v.offsets = c->offsets; v.recs = c->recs; v.occupied = c->occupied; v.cell_sigma = c->cell_sigma;
  v.n_occupied = c->n_occupied; v.res = c->res; v.n_lights = c->n_lights; v.n_g = c->n_g;
  for (int i = 0; i < 16; ++i) v.g_set[i] = c->g_set[i];
  return v;
}

// Query i of step s (Philox tag 3, item i, sub s): block 0 -> cell (integer
// scaling of the top 24 bits), position in the cell; block 1 -> direction
// (z = 1 - 2u, azimuth u turns) and phase index.
__device__ __forceinline__ void sample_query(const CacheView& C, int64_t i, int step, uint64_t seed, float q[6]) {
  uint32_t a[4], b[4];
  philox_block(seed, 3, (uint64_t)i, (uint32_t)step, 0, a);
  philox_block(seed, 3, (uint64_t)i, (uint32_t)step, 1, b);
  uint64_t ci = ((uint64_t)(a[0] >> 8) * (uint64_t)C.n_occupied) >> 24;
  uint32_t cell = C.occupied[ci];
  int R = C.res;
  int cx = (int)(cell % R), cy = (int)((cell / R) % R), cz = (int)(cell / ((uint32_t)R * R));
  const float k24 = 5.9604644775390625e-08f;
  q[0] = ((float)cx + (float)(a[1] >> 8) * k24) / (float)R;
  q[1] = ((float)cy + (float)(a[2] >> 8) * k24) / (float)R;
  q[2] = ((float)cz + (float)(a[3] >> 8) * k24) / (float)R;
  float wz = 1.0f - 2.0f * ((float)(b[0] >> 8) * k24);
  q[3] = acosf(fminf(fmaxf(wz, -1.f), 1.f)) * 0.318309886183790672f;
  q[4] = (float)(b[1] >> 8) * k24;
  int gi = (int)(((uint64_t)(b[2] >> 8) * (uint64_t)C.n_g) >> 24);
  q[5] = C.g_set[gi];
}

// Grid-cell radiance estimate of query q (see pf_estimate_targets).
__device__ __forceinline__ void estimate(const CacheView& C, const float q[6], float Ls[3]) {
  int gi = 0;
  for (int i = 0; i < C.n_g; ++i) if (C.g_set[i] == q[5]) gi = i;
  float g = C.g_set[gi];
  float st, ct, sp, cp;
  sincospif(q[3], &st, &ct);
  sincospif(2.0f * q[4], &sp, &cp);
  float wx = st * cp, wy = st * sp, wz = ct;
  int R = C.res;
  int bx = min(max((int)floorf(q[0] * (float)R), 0), R - 1);
  int by = min(max((int)floorf(q[1] * (float)R), 0), R - 1);
  int bz = min(max((int)floorf(q[2] * (float)R), 0), R - 1);
  int64_t nc = (int64_t)R * R * R;
  int64_t cell = bx + (int64_t)R * (by + (int64_t)R * bz);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  float gg = g * g, c0 = 0.0795774715459476678f * (1.f - gg), c1 = 1.f + gg, c2 = 2.f * g;
  for (int l = 0; l < C.n_lights; ++l) {
    int64_t key = (int64_t)(l * C.n_g + gi) * nc + cell;
    uint64_t e = C.offsets[key + 1];
    for (uint64_t n = C.offsets[key]; n < e; ++n) {
      float4 r0 = __ldg(&C.recs[2 * n]), r1 = __ldg(&C.recs[2 * n + 1]);
      float mu = r0.z * wx + r0.w * wy + r1.x * wz;
      float den = c1 - c2 * mu;
      float p = c0 / (den * sqrtf(den));
      a0 = fmaf(p, r1.y, a0); a1 = fmaf(p, r1.z, a1); a2 = fmaf(p, r1.w, a2);
    }
  }
  float s = C.cell_sigma[cell];
  float norm = s > 0.f ? 1.0f / ((1.0f / (float)nc) * s) : 0.f;
  Ls[0] = a0 * norm; Ls[1] = a1 * norm; Ls[2] = a2 * norm;
}

__device__ __forceinline__ float log_encode(float L, float psi) {
  return L > exp10f(-psi) ? -log10f(L) / psi : 1.0f;
}

__global__ void k_sample_queries(CacheView C, int64_t B, int step, uint64_t seed, float* __restrict__ q) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  float v[6];
  sample_query(C, i, step, seed, v);
  for (int d = 0; d < 6; ++d) q[6 * i + d] = v[d];
}

__global__ void k_estimate(CacheView C, const float* __restrict__ q, int64_t B, float psi, float* __restrict__ ls,
                           float* __restrict__ lp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  float v[6], L[3];
  for (int d = 0; d < 6; ++d) v[d] = q[6 * i + d];
  estimate(C, v, L);
  for (int c = 0; c < 3; ++c) {
    if (ls) ls[3 * i + c] = L[c];
    if (lp) lp[3 * i + c] = log_encode(L[c], psi);
  }
}

// Fused training-batch generator: queries and their log-encoded targets.
__global__ void k_batch(CacheView C, int64_t B, int step, uint64_t seed, float psi, float* __restrict__ q,
                        float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  float v[6], L[3];
  sample_query(C, i, step, seed, v);
  estimate(C, v, L);
  for (int d = 0; d < 6; ++d) q[6 * i + d] = v[d];
  for (int c = 0; c < 3; ++c) y[3 * i + c] = log_encode(L[c], psi);
}
}  // namespace

extern "C" pf_status pf_sample_queries(pf_ctx* ctx, const pf_cache* c, int64_t B, int step, uint64_t seed, float* q) {
  if (!ctx || !c || !q || B < 0 || step < 0 || step >= (1 << 24)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad query arguments");
  if (c->n_occupied == 0) return pf_fail(ctx, PF_ERR_INVALID_ARG, "cache has no occupied cells");
  DeviceGuard dg(ctx->device);
  if (B == 0) return PF_OK;
  k_sample_queries<<<(unsigned)((B + 255) / 256), 256, 0, ctx->stream>>>(cview(c), B, step, seed, q);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

extern "C" pf_status pf_estimate_targets(pf_ctx* ctx, const pf_cache* c, const float* q, int64_t B, float psi, float* ls,
                                         float* lp) {
  if (!ctx || !c || !q || B < 0 || !(psi > 0.f)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad estimate arguments");
  DeviceGuard dg(ctx->device);
  if (B == 0) return PF_OK;
  k_estimate<<<(unsigned)((B + 255) / 256), 256, 0, ctx->stream>>>(cview(c), q, B, psi, ls, lp);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

// ------------------------------------------------------------------ training loop
extern "C" pf_status pf_train_field(pf_ctx* ctx, const pf_cache* c, const pf_train_desc* d, pf_field* f, float* loss_host) {
  if (!ctx || !c || !d || !f) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (d->steps < 0 || d->batch <= 0 || !(d->lr > 0.f) || d->decay_every <= 0)
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad training description");
  if (c->n_occupied == 0) return pf_fail(ctx, PF_ERR_INVALID_ARG, "cache has no occupied cells");
  if (f->desc.prec == PF_PREC_FP8) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "fp8 fields are inference-only; train bf16/fp16");
  const bool knn = d->target == PF_TARGET_KNN;
  if (d->target != PF_TARGET_CELL && !knn) return pf_fail(ctx, PF_ERR_INVALID_ARG, "unknown target estimate");
  if (knn) {
    if (d->knn_k < 1 || d->knn_k > (1 << 20)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "knn_k must be in [1, 2^20]");
    if (d->knn_stages < 1 || d->knn_stages > PF_MAX_KNN_STAGES || d->knn_stage_begin[0] != 0.f)
      return pf_fail(ctx, PF_ERR_INVALID_ARG, "the KNN schedule needs 1..8 stages, the first starting at 0");
    for (int i = 0; i < d->knn_stages; ++i) {
      if (!(d->knn_radius[i] > 0.f && d->knn_radius[i] <= 2.f))
        return pf_fail(ctx, PF_ERR_INVALID_ARG, "KNN radii must lie in (0, 2]");
      if (!(d->knn_stage_begin[i] >= 0.f && d->knn_stage_begin[i] <= 1.f) ||
          (i > 0 && d->knn_stage_begin[i] < d->knn_stage_begin[i - 1]))
        return pf_fail(ctx, PF_ERR_INVALID_ARG, "KNN stage starts must not decrease and lie in [0, 1]");
    }
  }
  int64_t B = d->batch;
  float *q, *y, *g, *loss;
  // two batch buffers: the batch of step s + 1 (queries and targets, which do
  // not depend on the weights) is drawn on a second stream while step s
  // trains on the context's stream
  PF_TRY(pf_scratch(ctx, WS_QUERY, 2 * B * 6 * sizeof(float), (void**)&q));
  PF_TRY(pf_scratch(ctx, WS_TARGET, 2 * B * 3 * sizeof(float), (void**)&y));
  PF_TRY(pf_scratch(ctx, WS_GRAD, f->n_params * sizeof(float), (void**)&g));
  PF_TRY(pf_scratch(ctx, WS_LOSS, (size_t)std::max(d->steps, 1) * sizeof(float), (void**)&loss));
  PF_CUDA(ctx, cudaMemsetAsync(loss, 0, (size_t)std::max(d->steps, 1) * sizeof(float), ctx->stream));
  PF_TRY(pf_aux_stream(ctx));
  cudaEvent_t* ready = ctx->aux_ev;          // [b]: batch buffer b written
  cudaEvent_t* consumed = ctx->aux_ev + 2;   // [b]: last training step reading buffer b done
  cudaEvent_t fork = ctx->aux_ev[4];
  float* qb[2] = {q, q + 6 * B};
  float* yb[2] = {y, y + 3 * B};
  CacheView C = cview(c);
  int s0 = (int)std::ceil((double)d->decay_start_frac * d->steps);
  StageTimer tm(ctx, PF_STAGE_TRAIN);
  auto radius = [&](int s) {                 // the staggered schedule's cap at step s
    float r = d->knn_radius[0];
    for (int i = 1; i < d->knn_stages; ++i)
      if ((double)s >= std::ceil((double)d->knn_stage_begin[i] * d->steps)) r = d->knn_radius[i];
    return r;
  };
  auto draw = [&](int s) -> pf_status {      // batch of step s on the second stream
    if (knn) {
      k_sample_queries<<<(unsigned)((B + 255) / 256), 256, 0, ctx->aux>>>(C, B, s, d->seed, qb[s & 1]);
      PF_CUDA(ctx, cudaGetLastError());
      PF_TRY(pf_knn_targets_impl(ctx, c, qb[s & 1], B, d->knn_k, radius(s), f->desc.psi, nullptr, yb[s & 1], nullptr,
                                 nullptr, ctx->aux));
    } else {
      k_batch<<<(unsigned)((B + 255) / 256), 256, 0, ctx->aux>>>(C, B, s, d->seed, f->desc.psi, qb[s & 1], yb[s & 1]);
    }
    PF_CUDA(ctx, cudaGetLastError());
    PF_CUDA(ctx, cudaEventRecord(ready[s & 1], ctx->aux));
    return PF_OK;
  };
  PF_CUDA(ctx, cudaEventRecord(fork, ctx->stream));     // the caches were built on the context's stream
  PF_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, fork, 0));
  if (d->steps > 0) PF_TRY(draw(0));
  for (int s = 0; s < d->steps; ++s) {
    if (s + 1 < d->steps) {
      if (s >= 1) PF_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, consumed[(s + 1) & 1], 0));  // step s - 1's buffer
      PF_TRY(draw(s + 1));
    }
    PF_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ready[s & 1], 0));
    PF_TRY(pf_field_backward_impl(ctx, f, qb[s & 1], nullptr, yb[s & 1], B, g, loss + s));
    PF_CUDA(ctx, cudaEventRecord(consumed[s & 1], ctx->stream));
    int k = s < s0 ? 0 : (s - s0) / d->decay_every + 1;
    float lr = (float)((double)d->lr * std::pow((double)d->decay, k));
    PF_TRY(pf_adam_impl(ctx, f, g, lr, d->beta1, d->beta2, d->eps));
  }
  PF_CUDA(ctx, cudaEventRecord(fork, ctx->aux));        // join: nothing of the second stream outlives the call
  PF_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, fork, 0));
  if (loss_host && d->steps > 0)
    PF_CUDA(ctx, cudaMemcpyAsync(loss_host, loss, d->steps * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return pf_check_error_word(ctx);
}
