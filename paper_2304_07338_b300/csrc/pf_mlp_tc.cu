// Photon field MLP on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Forward pass (Sec. 3.4; hidden layers bf16 / fp16 / fp8 e4m3, FP32
// accumulation in tensor memory):
//   * one CTA per SM, persistent over 128-query tiles, with up to four
//     warpgroups that each carry their own tile through the layers (own A
//     tile, TMEM columns, MMA barrier and named barrier), so that one
//     group's MMAs overlap the others' CUDA-core work;
//   * the packed hidden-layer weights of the whole network are copied once
//     per CTA into shared memory, shared by the groups, with a bulk
//     asynchronous copy (cp.async.bulk, completion on an mbarrier);
//   * each thread owns one query row: it computes the frequency encoding and
//     writes it into the A tile in shared memory (K-major core-matrix layout:
//     8 rows x 16 bytes per core matrix, no swizzle);
//   * one elected thread issues tcgen05.mma over the K steps of the layer
//     (M = 128 rows, N = hidden width) into a TMEM accumulator and commits
//     to an mbarrier;
//   * every warp reads its 32 TMEM lanes back (tcgen05.ld), applies the fp8
//     dequantisation, ReLU and the next layer's operand rounding, and writes
//     the next A tile -- activations never leave the SM;
//   * the 3-wide output layer runs in float32 on the last hidden activation
//     straight from registers, followed by either the raw L' output or the
//     renderer's epilogue (decode 10^(-psi L') times albedo into the sample slot).
// All waits are bounded; a timeout sets the device error word, frees TMEM
// and returns.
#include "pf_internal.h"
#include "pf_field_common.cuh"
#include "pf_tc_ptx.cuh"
#include <algorithm>

using namespace pftc;

namespace {

constexpr int kThreads = 128;
constexpr int kFwdMaxThreads = 512;   // forward: up to four warpgroups
constexpr int kMaxLayers = 8;

struct TcLayer {
  uint32_t w_off;      // byte offset of the layer's packed weights in shared memory
  uint32_t kp;         // padded K (multiple of the MMA K step)
  float dequant;       // s_a * s_w (fp8), 1 otherwise
  float inv_s_in;      // 1 / s_a: scale applied when this layer's input is written (fp8), 1 otherwise
};

struct TcArgs {
  const uint8_t* wq;   // packed weights (global)
  uint32_t wq_bytes;
  const float* w_out;  // [3][H] float32 output layer
  int n_hidden, hidden, in_freqs, prec, kstep;  // kstep = 16 (16-bit) or 32 (fp8)
  int n_groups;        // forward: warpgroups (tiles in flight) per CTA
  uint32_t a_off, a_bytes, wout_off, ypart_off, bar_off, smem_bytes;
  float psi;
  TcLayer L[kMaxLayers];
};

// Operand encoding of one value for the A tile.
template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if (PREC == PF_PREC_BF16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(uint32_t*)&h;
  } else {
    __half2 h = __floats2half2_rn(a, b);
    return *(uint32_t*)&h;
  }
}
// Four e4m3 codes (round to nearest even, saturating), a in the low byte;
// two paired conversions, each the same rounding as pff::e4m3_code.
__device__ __forceinline__ uint32_t pack4_e4m3(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xFFFFu) | (hi << 16);
}

// Writes 16 bytes of row r at K-chunk c (16 bytes = one core-matrix row).
__device__ __forceinline__ void store_chunk(uint8_t* tile, uint32_t kp_bytes, int r, int c, uint4 v) {
  uint32_t off = (uint32_t)(r >> 3) * (kp_bytes / 16) * 128 + (uint32_t)c * 128 + (uint32_t)(r & 7) * 16;
  *(uint4*)(tile + off) = v;
}

// Takes 16 values of one row (already scaled) and stores them as operands:
// 16-bit types -> two 16-byte chunks, fp8 -> one chunk.  `col` is the first
// element's K index (multiple of 16).
template <int PREC>
__device__ __forceinline__ void store16(uint8_t* tile, uint32_t kp, int r, int col, const float v[16]) {
  if (PREC == PF_PREC_FP8) {
    uint4 q;
    q.x = pack4_e4m3(v[0], v[1], v[2], v[3]);
    q.y = pack4_e4m3(v[4], v[5], v[6], v[7]);
    q.z = pack4_e4m3(v[8], v[9], v[10], v[11]);
    q.w = pack4_e4m3(v[12], v[13], v[14], v[15]);
    store_chunk(tile, kp, r, col / 16, q);
  } else {
    uint4 q0, q1;
    q0.x = pack2<PREC>(v[0], v[1]); q0.y = pack2<PREC>(v[2], v[3]);
    q0.z = pack2<PREC>(v[4], v[5]); q0.w = pack2<PREC>(v[6], v[7]);
    q1.x = pack2<PREC>(v[8], v[9]); q1.y = pack2<PREC>(v[10], v[11]);
    q1.z = pack2<PREC>(v[12], v[13]); q1.w = pack2<PREC>(v[14], v[15]);
    store_chunk(tile, kp * 2, r, col / 8, q0);
    store_chunk(tile, kp * 2, r, col / 8 + 1, q1);
  }
}

// 16-bit operands of 16 values of row r with ReLU, applied to the rounded
// pairs (packed max with +0).
template <int PREC>
__device__ __forceinline__ void store16_relu(uint8_t* tile, uint32_t kp, int r, int col, const float v[16]) {
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (PREC == PF_PREC_BF16) {
      __nv_bfloat162 h = __hmax2(__floats2bfloat162_rn(v[2 * i], v[2 * i + 1]), __float2bfloat162_rn(0.f));
      w[i] = *(uint32_t*)&h;
    } else {
      __half2 h = __hmax2(__floats2half2_rn(v[2 * i], v[2 * i + 1]), __float2half2_rn(0.f));
      w[i] = *(uint32_t*)&h;
    }
  }
  store_chunk(tile, kp * 2, r, col / 8, make_uint4(w[0], w[1], w[2], w[3]));
  store_chunk(tile, kp * 2, r, col / 8 + 1, make_uint4(w[4], w[5], w[6], w[7]));
}

// Frequency encoding of one query (6 inputs x F frequencies, features ordered
// [input][k][sin, cos], each times s) into row r of an A tile with K extent
// kp, zero-padded to kp; features sin/cos(2^k pi v) by pff::freq_next.
// F = 12 (the usual width) is unrolled so that the 16-feature staging buffer
// stays in registers.
template <int PREC>
__device__ __forceinline__ void encode_query(uint8_t* tile, uint32_t kp, int r, const float qv[6], int F, float s) {
  if (F == 12) {
    float buf[16];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      float sn = 0.f, cs = 1.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        pff::freq_next(qv[d], k, sn, cs);
        const int f = 24 * d + 2 * k;       // feature index; 16 features per store
        buf[f % 16] = sn * s;
        buf[(f + 1) % 16] = cs * s;
        if ((f + 2) % 16 == 0) store16<PREC>(tile, kp, r, f + 2 - 16, buf);
      }
    }
    // features 144..kp-1: zero padding (144 = 9 x 16)
    for (int col = 144; col < (int)kp; col += 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) buf[i] = 0.f;
      store16<PREC>(tile, kp, r, col, buf);
    }
    return;
  }
  float buf[16];
  int nb = 0, col = 0;
  for (int d = 0; d < 6; ++d) {
    float sn = 0.f, cs = 1.f;
    for (int k = 0; k < F; ++k) {
      pff::freq_next(qv[d], k, sn, cs);
      buf[nb++] = sn * s;
      buf[nb++] = cs * s;
      if (nb == 16) { store16<PREC>(tile, kp, r, col, buf); col += 16; nb = 0; }
    }
  }
  while (col < (int)kp) {      // zero padding up to the MMA K step
    for (int i = nb; i < 16; ++i) buf[i] = 0.f;
    store16<PREC>(tile, kp, r, col, buf);
    col += 16;
    nb = 0;
  }
}

// Writes 8 values of row r as one 16-byte chunk (16-bit operand types);
// `chunk` is the K index / 8.
template <int PREC>
__device__ __forceinline__ void store8(uint8_t* tile, uint32_t kp, int r, int chunk, const float v[8]) {
  uint4 q;
  q.x = pack2<PREC>(v[0], v[1]); q.y = pack2<PREC>(v[2], v[3]);
  q.z = pack2<PREC>(v[4], v[5]); q.w = pack2<PREC>(v[6], v[7]);
  store_chunk(tile, kp * 2, r, chunk, q);
}

// Half of the frequency encoding of one query (16-bit operands, F = 12):
// inputs 3h..3h+2, i.e. features 72h..72h+71 of the row, the same values as
// encode_query writes there (nine 16-byte chunks).
template <int PREC>
__device__ __forceinline__ void encode_half(uint8_t* tile, uint32_t kp, int r, const float qv[3], int h) {
  float buf[8];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float sn = 0.f, cs = 1.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      pff::freq_next(qv[d], k, sn, cs);
      const int f = 24 * d + 2 * k;
      buf[f % 8] = sn;
      buf[(f + 1) % 8] = cs;
      if ((f + 2) % 8 == 0) store8<PREC>(tile, kp, r, (72 * h + f + 2 - 8) / 8, buf);
    }
  }
}

// TPR threads per tile row: 1, or 2 for 16-bit fields whose shared memory
// holds only two tiles in flight (the f16 / bf16 4 x 128 render field), so
// that the SM still has 16 warps to switch between.  With TPR = 2 the thread
// pair (r, r + 128) of a group owns row r; the two threads split the
// encoding (inputs 0-2 / 3-5) and the epilogue columns (halves of H), and the
// output layer's two partial sums meet in shared memory.
template <int PREC, int TPR>
__global__ void __launch_bounds__(kFwdMaxThreads, 1) k_tc_forward(TcArgs A, const float* __restrict__ q, int64_t B_max,
                                                            const uint32_t* __restrict__ B_dev, float* __restrict__ out,
                                                            const uint32_t* __restrict__ slot_idx,
                                                            const float* __restrict__ slot_alb,
                                                            float* __restrict__ slot_li, uint32_t* err) {
  constexpr bool FP8 = (PREC == PF_PREC_FP8);
  constexpr uint32_t EB = FP8 ? 1 : 2;
  constexpr uint32_t AB_TYPE = (PREC == PF_PREC_BF16) ? 1u : 0u;   // f16 = 0, bf16 = 1, e4m3 = 0
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int GT = 128 * TPR;                  // threads of a group
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wg = tid / GT, gtid = tid % GT;      // group; its thread
  const int ltid = gtid & 127, half = gtid >> 7; // row of the tile; column half (TPR = 2)
  const int NG = A.n_groups;
  uint8_t* a_tile = smem + A.a_off + (uint32_t)wg * A.a_bytes;
  float* w_out = (float*)(smem + A.wout_off);
  float* ypart = (float*)(smem + A.ypart_off) + (size_t)wg * 3 * kTileM;   // TPR = 2: [3][128] partial outputs
  uint64_t* bars = (uint64_t*)(smem + A.bar_off);          // [0] weights, [1 + g] MMAs of group g
  uint32_t* tmem_slot = (uint32_t*)(smem + A.bar_off + 48);
  int* abort_flag = (int*)(smem + A.bar_off + 52);
  const uint32_t bar_w = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1 + wg]);
  const int H = A.hidden;
  const uint32_t tmem_cols = (uint32_t)(NG * H);        // 128, 256 or 512

  if (tid == 0) {
    mbar_init(bar_w, 1);
    for (int g = 0; g < NG; ++g) mbar_init(smem_u32(&bars[1 + g]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 3 * H; i += blockDim.x) w_out[i] = A.w_out[i];
  if (warp == 0) tmem_alloc(tmem_slot, tmem_cols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot + (uint32_t)(wg * H);   // this group's accumulator columns
  // weights: one bulk copy (the packed block is contiguous and 16-byte sized)
  if (tid == 0) {
    mbar_expect_tx(bar_w, A.wq_bytes);
    bulk_g2s(smem_u32(smem), A.wq, A.wq_bytes, bar_w);
  }
  if (!mbar_wait(bar_w, 0)) {
    if (tid == 0) { atomicOr(err, PFE_ITER_CAP); *abort_flag = 1; }
  }
  __syncthreads();
  const int64_t B = B_dev ? (int64_t)*B_dev : B_max;
  const int64_t n_tiles = (B + kTileM - 1) / kTileM;
  uint32_t mma_phase = 0;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int F = A.in_freqs;
  const uint32_t kp0 = A.L[0].kp;

  // A timed-out wait sets abort_flag; the group stops at its next barrier,
  // all of its threads alike (the barrier ORs their reads of the flag).
  bool stop = false;
  // this thread's query inputs (3 with TPR = 2), loaded one tile ahead so
  // that the loads are in flight while the group works on the current tile
  constexpr int NQ = TPR == 2 ? 3 : 6;
  const int q0 = TPR == 2 ? 3 * half : 0;
  const int64_t t_step = (int64_t)gridDim.x * NG;
  float qn[NQ];
  auto load_q = [&](int64_t t) {
    const int64_t r = t * kTileM + ltid;
    const bool ok = t < n_tiles && r < B;
#pragma unroll
    for (int d = 0; d < NQ; ++d) qn[d] = ok ? __ldg(q + 6 * r + q0 + d) : 0.f;
  };
  load_q((int64_t)blockIdx.x * NG + wg);
  for (int64_t tile = (int64_t)blockIdx.x * NG + wg; tile < n_tiles; tile += t_step) {
    const int64_t row = tile * kTileM + ltid;
    const bool valid = row < B;
    float qv[NQ];
#pragma unroll
    for (int d = 0; d < NQ; ++d) qv[d] = qn[d];
    load_q(tile + t_step);
    // the render epilogue's inputs of this row, also in flight meanwhile
    uint32_t sl = 0;
    float al0 = 0.f, al1 = 0.f, al2 = 0.f;
    if (slot_idx && valid && half == 0) {
      sl = __ldg(slot_idx + row);
      al0 = __ldg(slot_alb + 3 * row + 0); al1 = __ldg(slot_alb + 3 * row + 1); al2 = __ldg(slot_alb + 3 * row + 2);
    }
    // ---- encoding of this thread's query into the A tile (K = kp0)
    if (TPR == 2) {
      encode_half<PREC>(a_tile, kp0, ltid, qv, half);
    } else {
      const float s = FP8 ? A.L[0].inv_s_in : 1.f;   // input scale of layer 0 (fp8)
      encode_query<PREC>(a_tile, kp0, ltid, qv, F, s);
    }
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
    for (int l = 0; l < A.n_hidden; ++l) {
      const TcLayer Ly = A.L[l];
      fence_proxy_async();
      tc_fence_before();
      stop = named_barrier_or(1 + wg, GT, *abort_flag != 0);
      tc_fence_after();
      if (stop) break;
      if (gtid == 0) {
        const uint32_t a0 = smem_u32(a_tile), b0 = smem_u32(smem + Ly.w_off);
        const uint32_t sbo = (Ly.kp * EB / 16) * 128;
        const uint32_t id = idesc(AB_TYPE, (uint32_t)H);
        const int nk = (int)(Ly.kp / A.kstep);
        for (int ks = 0; ks < nk; ++ks) {
          // a K step spans 32 bytes = two core matrices along K, so the start
          // address advances by 2 * LBO = 256 bytes
          const uint64_t ad = sdesc(a0 + ks * 256, 128, sbo);
          const uint64_t bd = sdesc(b0 + ks * 256, 128, sbo);
          mma<FP8>(tmem, ad, bd, id, ks > 0 ? 1u : 0u);
        }
        mma_commit(bar_mma);
      }
      if (!mbar_wait(bar_mma, mma_phase)) {
        atomicOr(err, PFE_ITER_CAP);
        *abort_flag = 1;
      }
      mma_phase ^= 1u;
      tc_fence_after();
      const bool last = (l == A.n_hidden - 1);
      const uint32_t kp_next = last ? 0u : A.L[l + 1].kp;
      // dequantisation and the next layer's input scale are powers of two
      // (fp8; 1 otherwise), so one product by their product is exact too
      const float s_next = (FP8 && !last) ? A.L[l + 1].inv_s_in : 1.f;
      const float sc = last ? Ly.dequant : Ly.dequant * s_next;
      const int c_lo = half * (H / TPR), c_hi = c_lo + H / TPR;
      for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);       // 32 columns, one wait
        if (FP8) {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] *= sc;           // power-of-two scales (1 for 16-bit fields)
        }
        if (last) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 w0 = *(const float4*)(w_out + c0 + i);
            const float4 w1 = *(const float4*)(w_out + H + c0 + i);
            const float4 w2 = *(const float4*)(w_out + 2 * H + c0 + i);
            const float a0 = fmaxf(v[i], 0.f), a1 = fmaxf(v[i + 1], 0.f);
            const float a2 = fmaxf(v[i + 2], 0.f), a3 = fmaxf(v[i + 3], 0.f);
            y0 = fmaf(a0, w0.x, y0); y0 = fmaf(a1, w0.y, y0);
            y0 = fmaf(a2, w0.z, y0); y0 = fmaf(a3, w0.w, y0);
            y1 = fmaf(a0, w1.x, y1); y1 = fmaf(a1, w1.y, y1);
            y1 = fmaf(a2, w1.z, y1); y1 = fmaf(a3, w1.w, y1);
            y2 = fmaf(a0, w2.x, y2); y2 = fmaf(a1, w2.y, y2);
            y2 = fmaf(a2, w2.z, y2); y2 = fmaf(a3, w2.w, y2);
          }
        } else if (FP8) {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
          store16<PREC>(a_tile, kp_next, ltid, c0, v);
          store16<PREC>(a_tile, kp_next, ltid, c0 + 16, v + 16);
        } else {
          // rounding is monotonic and 0 is exact, so ReLU after the
          // rounding equals ReLU before it: one packed max per two values
          store16_relu<PREC>(a_tile, kp_next, ltid, c0, v);
          store16_relu<PREC>(a_tile, kp_next, ltid, c0 + 16, v + 16);
        }
      }
    }
    if (stop) break;
    if (TPR == 2) {                    // the second half's partial sums join the first's
      if (half == 1) { ypart[ltid] = y0; ypart[kTileM + ltid] = y1; ypart[2 * kTileM + ltid] = y2; }
      named_barrier(1 + wg, GT);
      if (half == 1) continue;
      y0 = y0 + ypart[ltid]; y1 = y1 + ypart[kTileM + ltid]; y2 = y2 + ypart[2 * kTileM + ltid];
    }
    if (valid) {
      if (slot_idx) {
        slot_li[3 * (size_t)sl + 0] = al0 * exp10f(-A.psi * y0);
        slot_li[3 * (size_t)sl + 1] = al1 * exp10f(-A.psi * y1);
        slot_li[3 * (size_t)sl + 2] = al2 * exp10f(-A.psi * y2);
      } else {
        out[3 * row + 0] = y0;
        out[3 * row + 1] = y1;
        out[3 * row + 2] = y2;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(*tmem_slot, tmem_cols);
}

// ---------------------------------------------------------------- training step
// One fused pass per 128-query tile (bf16 / fp16 fields of width 64), two
// warpgroups splitting each row's columns:
//   forward  : encoding -> A_0; for each hidden layer l, tcgen05.mma
//              A_l x W_l^T -> TMEM, ReLU, operand rounding -> A_{l+1}
//              (every layer's input tile stays in shared memory);
//   output   : y = W_out h_L in float32 from registers; relative-MSE gradient
//              with loss scaling, dy = 2 (y - t) / (t^2 + 0.01) (3B times the
//              gradient of the mean; 1/(3B) is applied to the float32 dW sums
//              by k_reduce_partials), or a given dy; loss;
//              dW_out from registers: products dy_c h_n summed over each
//              warp's 32 rows by a butterfly reduce-scatter, then over the
//              four warps of the row quarters in order; dZ_{L-1} =
//              (W_out^T dy) * [h_L > 0];
//   backward : for l = L-1..0, tcgen05.mma dW_l += dZ_l^T x A_l (both operands
//              MN-major views of the row tiles, M padded to 128 neurons) into
//              a TMEM accumulator that persists across the CTA's tiles, and
//              dA_l = dZ_l x W_l (W_l as an MN-major B operand); epilogue
//              masks with [A_l > 0] and rounds into dZ_{l-1}.
// At the end each CTA writes its dW (float32) to its own partial row; a
// second kernel sums the partials in a fixed order.
struct TrArgs {
  TcArgs f;                 // forward plan (weights, A-tile K extents)
  uint32_t a_off[kMaxLayers];   // shared-memory byte offset of A_l
  uint32_t d_off;           // dZ tile (128 x 128 neurons, padded)
  uint32_t dwo_off;         // dW_out accumulator (3 x H float32)
  uint32_t part_off;        // dW_out partial sums: [8 warps][3][32] float32
  uint32_t dys_off;         // output-layer gradients of the tile (128 x 4 float32)
  uint32_t dw_col[kMaxLayers];  // TMEM column of dW_l
  uint32_t g_off;           // hash grids: [H] g weights, [H] dW of the g column, [128] g of the rows
  int64_t layer_off[kMaxLayers + 1];
  int64_t n_params;         // MLP weights (the partial rows' stride)
  // hash-grid fields: layer 0's operand is the nf = 2 L F table features
  // (x_in, [B][nf] in the field precision); g (fan0 = nf + 1 inputs) enters
  // on the CUDA cores; dx_out [B][nf] receives the features' gradient
  int hash, fan0, nf;
  const uint16_t* x_in;
  float* dx_out;
  const float* w0;          // layer 0 master weights [H][fan0]
};
constexpr uint32_t kTrainCols = 512;
constexpr int kTrainHidden = 64;
constexpr int kTrainThreads = 256;
constexpr uint32_t kDK = 128;       // padded neuron extent of the dZ tile


// One 16-bit operand (bf16 or f16 bits) as a float.
template <int PREC>
__device__ __forceinline__ float op_value(uint16_t h) {
  if (PREC == PF_PREC_BF16) return __bfloat162float(__ushort_as_bfloat16(h));
  return __half2float(__ushort_as_half(h));
}

// Fused forward + loss + backward for a 128-query tile, two warpgroups: the
// thread pair (r, r + 128) owns tile row r, and the two threads split the
// row's columns (encoding inputs 0-2 / 3-5, or the position / direction
// halves of the hash-grid features; neurons 0-31 / 32-63), so that each SM
// sub-partition has two warps to switch between while the other waits.
// TMEM lane quarter of warp w: w mod 4.
// HASH: layer 0's operand is the table features from x_in; g's term
// W_0[:, nf] g is added on the CUDA cores before the ReLU, its weight
// gradient summed on them too, and the features' gradient dZ_0 W_0 is
// written to dx_out for the table scatter.
template <int PREC, bool HASH>
__global__ void __launch_bounds__(kTrainThreads, 1) k_tc_train(TrArgs T, const float* __restrict__ q,
                                                               const float* __restrict__ targets,
                                                               const float* __restrict__ dy_in, int64_t B, float inv_n,
                                                               float* __restrict__ partial, float* __restrict__ loss,
                                                               uint32_t* err) {
  constexpr uint32_t AB_TYPE = (PREC == PF_PREC_BF16) ? 1u : 0u;
  constexpr int H = kTrainHidden;   // the only width planned for this kernel
  constexpr int HH = H / 2;         // columns per thread of a row pair
  extern __shared__ __align__(1024) uint8_t smem[];
  const TcArgs& A = T.f;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & (kTileM - 1), hf = tid >> 7;
  float* w_out = (float*)(smem + A.wout_off);
  float* dwo = (float*)(smem + T.dwo_off);
  uint8_t* dtile = smem + T.d_off;
  uint64_t* bars = (uint64_t*)(smem + A.bar_off);
  uint32_t* tmem_slot = (uint32_t*)(smem + A.bar_off + 16);
  int* abort_flag = (int*)(smem + A.bar_off + 20);
  const uint32_t bar_w = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  const int L = A.n_hidden;
  float* dwo_part = (float*)(smem + T.part_off);
  float* dys = (float*)(smem + T.dys_off);      // [128][4]: dy of the row
  float* ys = dys + 4 * kTileM;                  // [128][4]: second half's partial output
  float* wg = (float*)(smem + T.g_off);          // hash grids: [H] rounded g weights of layer 0
  float* dwg = wg + H;                           // [H] dW of layer 0's g column
  float* gs = dwg + H;                           // [128] rounded g of the tile's rows

  if (tid == 0) {
    mbar_init(bar_w, 1);
    mbar_init(bar_mma, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 3 * H; i += kTrainThreads) { w_out[i] = A.w_out[i]; dwo[i] = 0.f; }
  if (HASH)
    for (int i = tid; i < H; i += kTrainThreads) {
      const float wv = T.w0[(size_t)i * T.fan0 + T.nf];
      wg[i] = PREC == PF_PREC_BF16 ? pff::round_bf16(wv) : pff::round_f16(wv);
      dwg[i] = 0.f;
    }
  // zero the padded neuron columns of the dZ tile once (never written later)
  for (int i = tid; i < (int)(kTileM * kDK * 2 / 16); i += kTrainThreads) ((uint4*)dtile)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(tmem_slot, kTrainCols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    mbar_expect_tx(bar_w, A.wq_bytes);
    bulk_g2s(smem_u32(smem), A.wq, A.wq_bytes, bar_w);
  }
  if (!mbar_wait(bar_w, 0) && tid == 0) { atomicOr(err, PFE_ITER_CAP); *abort_flag = 1; }
  __syncthreads();
  const int64_t n_tiles = (B + kTileM - 1) / kTileM;
  uint32_t phase = 0;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int F = A.in_freqs;
  const uint32_t kp0 = A.L[0].kp;
  const uint32_t d_rg = (kDK * 2 / 16) * 128;       // dZ tile: bytes between 8-row groups
  bool first_tile = true;
  float lsum = 0.f;

  // A timed-out wait sets abort_flag; the CTA stops at the next MMA's
  // barrier, every thread alike (__syncthreads_or over their reads).
  auto sync_mma = [&]() {
    if (tid == 0) mma_commit(bar_mma);
    bool ok = mbar_wait(bar_mma, phase);
    phase ^= 1u;
    tc_fence_after();
    if (!ok) { atomicOr(err, PFE_ITER_CAP); *abort_flag = 1; }
  };
  auto pre_mma = [&]() -> bool {
    fence_proxy_async();
    tc_fence_before();
    const bool s = __syncthreads_or(*abort_flag != 0) != 0;
    tc_fence_after();
    return s;
  };
  bool stop = false;
  // the frequency-encoded rows' inputs (this thread's three) and targets,
  // loaded one tile ahead: the next tile's loads are issued after the loss,
  // so that they arrive during the backward pass
  const bool ahead = !HASH && F == 12;
  float qn[3] = {0.f, 0.f, 0.f}, tn[3] = {0.f, 0.f, 0.f};
  auto load_ahead = [&](int64_t tl) {
    const int64_t rw = tl * kTileM + r;
    const bool ok = tl < n_tiles && rw < B;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) qn[dd] = ok ? __ldg(q + 6 * rw + 3 * hf + dd) : 0.f;
    if (targets && hf == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) tn[c] = ok ? __ldg(targets + 3 * rw + c) : 0.f;
    }
  };
  if (ahead) load_ahead(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row = tile * kTileM + r;
    const bool valid = row < B;
    // ---- encoding -> A_0
    {
      uint8_t* a0 = smem + T.a_off[0];
      if (HASH) {
        // this thread: half hf of the row's table features, as 16-byte chunks
        const int nc = T.nf / 16;
        const uint4* src = (const uint4*)(T.x_in + (size_t)(valid ? row : 0) * T.nf);
        for (int c = hf * nc; c < (hf + 1) * nc; ++c)
          store_chunk(a0, kp0 * 2, r, c, valid ? __ldg(src + c) : make_uint4(0, 0, 0, 0));
        if (hf == 0) {
          const float gv = valid ? __ldg(q + 6 * row + 5) : 0.f;
          gs[r] = PREC == PF_PREC_BF16 ? pff::round_bf16(gv) : pff::round_f16(gv);
        }
      } else if (F == 12) {
        // this thread: inputs 3 hf .. 3 hf + 2 = features 72 hf .. 72 hf + 71
        float buf[8];
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
          const float v = qn[dd];
          float sn = 0.f, cs = 1.f;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            pff::freq_next(v, k, sn, cs);
            const int lf = 24 * dd + 2 * k;
            buf[lf % 8] = sn;
            buf[(lf + 1) % 8] = cs;
            if ((lf + 2) % 8 == 0) store8<PREC>(a0, kp0, r, (72 * hf + lf + 2 - 8) / 8, buf);
          }
        }
        // zero padding of K = 144 .. kp0 - 1, chunks split between the pair
#pragma unroll
        for (int i = 0; i < 8; ++i) buf[i] = 0.f;
        for (int c = 18 + hf; c < (int)(kp0 / 8); c += 2) store8<PREC>(a0, kp0, r, c, buf);
      } else if (hf == 0) {
        float qv[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) qv[d] = valid ? __ldg(q + 6 * row + d) : 0.f;
        encode_query<PREC>(a0, kp0, r, qv, F, 1.f);
      }
    }
    // ---- forward through the hidden layers
    float h[HH];
    for (int l = 0; l < L; ++l) {
      const TcLayer Ly = A.L[l];
      if ((stop = pre_mma())) break;
      if (tid == 0) {
        const uint32_t a0 = smem_u32(smem + T.a_off[l]), b0 = smem_u32(smem + Ly.w_off);
        const uint32_t sbo = (Ly.kp * 2 / 16) * 128;
        const uint32_t id = idesc(AB_TYPE, (uint32_t)H);
        for (int ks = 0; ks < (int)(Ly.kp / 16); ++ks)
          mma<false>(tmem, sdesc(a0 + ks * 256, 128, sbo), sdesc(b0 + ks * 256, 128, sbo), id, ks > 0 ? 1u : 0u);
      }
      sync_mma();
#pragma unroll
      for (int g = 0; g < HH / 16; ++g) {
        const int c0 = HH * hf + 16 * g;
        float v[16];
        tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
        if (HASH && l == 0) {
          const float gr = gs[r];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = fmaf(wg[c0 + i], gr, v[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
        if (l == L - 1) {
#pragma unroll
          for (int i = 0; i < 16; ++i) h[16 * g + i] = v[i];
        } else {
          store16<PREC>(smem + T.a_off[l + 1], (uint32_t)H, r, c0, v);
        }
      }
    }
    if (stop) break;
    // ---- output layer (float32 on the unrounded last activation), loss, dy
    {
      float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
      for (int j = 0; j < HH; ++j) {
        const int n = HH * hf + j;
        y0 = fmaf(h[j], w_out[n], y0);
        y1 = fmaf(h[j], w_out[H + n], y1);
        y2 = fmaf(h[j], w_out[2 * H + n], y2);
      }
      if (hf == 1) { ys[4 * r + 0] = y0; ys[4 * r + 1] = y1; ys[4 * r + 2] = y2; }
      __syncthreads();
      if (hf == 0) {
        const float y[3] = {y0 + ys[4 * r + 0], y1 + ys[4 * r + 1], y2 + ys[4 * r + 2]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float g = 0.f;
          if (valid) {
            if (targets) {
              const float t = ahead ? tn[c] : targets[3 * row + c];
              const float den = t * t + 0.01f;
              const float diff = y[c] - t;
              lsum += diff * diff / den;
              g = 2.f * diff / den;             // loss-scaled by 3B (see pf_tc_backward)
            } else {
              g = dy_in[3 * row + c];
            }
          }
          dys[4 * r + c] = g;
        }
      }
      __syncthreads();
    }
    if (ahead) load_ahead(tile + gridDim.x);
    const float dy0 = dys[4 * r + 0], dy1 = dys[4 * r + 1], dy2 = dys[4 * r + 2];
    // dW_out[c][n] += sum over the tile's rows of dy_c h_n.  Per warp (32
    // rows, this half's 32 columns) a butterfly reduce-scatter leaves lane j
    // holding column j's sum over the warp's rows; the four warps of the
    // half are then added in row order.  dy is 0 on rows past the batch.
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float dc = c == 0 ? dy0 : (c == 1 ? dy1 : dy2);
      float v[HH];
#pragma unroll
      for (int i = 0; i < HH; ++i) v[i] = dc * h[i];
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int off = 16 >> st;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
          const float send = up ? v[i] : v[off + i];
          const float keep = up ? v[off + i] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      dwo_part[(warp * 3 + c) * 32 + lane] = v[0];
    }
    __syncthreads();
    for (int o = tid; o < 3 * H; o += kTrainThreads) {
      const int c = o / H, n = o % H, hq = n / HH, j = n % HH;
      const float* pp = dwo_part + (4 * hq * 3 + c) * 32 + j;  // warps 4 hq .. 4 hq + 3, stride 3 x 32
      dwo[o] += ((pp[0] + pp[96]) + pp[192]) + pp[288];
    }
    // dZ_{L-1} = (dy W_out) * [rounded h > 0], this thread's columns
#pragma unroll
    for (int g = 0; g < HH / 16; ++g) {
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int j = 16 * g + i, n = HH * hf + j;
        const float dh = dy0 * w_out[n] + dy1 * w_out[H + n] + dy2 * w_out[2 * H + n];
        const float hr = PREC == PF_PREC_BF16 ? pff::round_bf16(h[j]) : pff::round_f16(h[j]);
        v[i] = hr > 0.f ? dh : 0.f;
      }
      store16<PREC>(dtile, kDK, r, HH * hf + 16 * g, v);
    }
    // ---- backward through the hidden layers
    for (int l = L - 1; l >= 0; --l) {
      const TcLayer Ly = A.L[l];
      if ((stop = pre_mma())) break;
      if (tid == 0) {
        // dW_l (+)= dZ_l^T A_l: A = dZ tile viewed MN-major (M = neurons, K = samples),
        // B = A_l viewed MN-major (N = input features, K = samples); K steps of 16 samples
        const uint32_t dz0 = smem_u32(dtile), al0 = smem_u32(smem + T.a_off[l]);
        const uint32_t a_rg = (Ly.kp * 2 / 16) * 128;      // A_l: bytes between 8-row groups
        const uint32_t idw = idesc(AB_TYPE, Ly.kp, 1u, 1u);
        for (int ks = 0; ks < kTileM / 16; ++ks) {
          const uint64_t ad = sdesc(dz0 + ks * 2 * d_rg, d_rg, 128);
          const uint64_t bd = sdesc(al0 + ks * 2 * a_rg, a_rg, 128);
          mma<false>(tmem + T.dw_col[l], ad, bd, idw, (first_tile && ks == 0) ? 0u : 1u);
        }
        if (l > 0) {
          // dA_l = dZ_l W_l: A = dZ tile K-major (K = the layer's H output neurons),
          // B = W_l viewed MN-major (N = input features, K = output neurons)
          const uint32_t w0 = smem_u32(smem + Ly.w_off);
          const uint32_t w_rg = (Ly.kp * 2 / 16) * 128;    // W_l: bytes between 8-neuron groups
          const uint32_t ida = idesc(AB_TYPE, Ly.kp, 0u, 1u);
          for (int ks = 0; ks < H / 16; ++ks) {
            const uint64_t ad = sdesc(dz0 + ks * 256, 128, d_rg);
            const uint64_t bd = sdesc(w0 + ks * 2 * w_rg, w_rg, 128);
            mma<false>(tmem, ad, bd, ida, ks > 0 ? 1u : 0u);
          }
        }
      }
      sync_mma();
      if (l > 0) {
        // dZ_{l-1} = dA_l * [A_l > 0], rounded; A_l is the layer's (rounded)
        // input tile (H wide for l > 0); the pair splits its column groups
        const uint8_t* al = smem + T.a_off[l];
        const uint32_t kpl = A.L[l].kp;
        for (int c0 = 16 * hf; c0 < (int)kpl; c0 += 32) {
          float v[16];
          tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint32_t off = (uint32_t)(r >> 3) * ((kpl * 2 / 16) * 128) + (uint32_t)(c0 / 8 + j) * 128 +
                                 (uint32_t)(r & 7) * 16;
            const uint4 raw = *(const uint4*)(al + off);
            const uint16_t* hv = (const uint16_t*)&raw;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const bool pos = (hv[i] & 0x8000u) == 0 && (hv[i] & 0x7FFFu) != 0;
              if (!pos) v[8 * j + i] = 0.f;
            }
          }
          store16<PREC>(dtile, kDK, r, c0, v);
        }
      }
      if (HASH && l == 0) {
        // dW of the g column: one owner thread per neuron over the tile's rows
        for (int n = tid; n < H; n += kTrainThreads) {
          float acc = 0.f;
          for (int rr = 0; rr < kTileM; ++rr) {
            const uint32_t off = (uint32_t)(rr >> 3) * d_rg + (uint32_t)(n >> 3) * 128 + (uint32_t)(rr & 7) * 16 +
                                 (uint32_t)(n & 7) * 2;
            acc = fmaf(op_value<PREC>(*(const uint16_t*)(dtile + off)), gs[rr], acc);
          }
          dwg[n] += acc;
        }
        // the features' gradient dZ_0 W_0 (W_0 rounded, as packed): this
        // thread's half of the row
        if (valid) {
          float dz[H];
#pragma unroll
          for (int c = 0; c < H / 8; ++c) {
            const uint4 raw = *(const uint4*)(dtile + (uint32_t)(r >> 3) * d_rg + (uint32_t)c * 128 +
                                              (uint32_t)(r & 7) * 16);
            const uint16_t* hv = (const uint16_t*)&raw;
#pragma unroll
            for (int i = 0; i < 8; ++i) dz[8 * c + i] = op_value<PREC>(hv[i]);
          }
          const uint8_t* w0p = smem + A.L[0].w_off;
          const int nc = T.nf / 16;
          float* dst = T.dx_out + (size_t)row * T.nf;
          for (int c = hf * nc; c < (hf + 1) * nc; ++c) {
            float acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll 8
            for (int n = 0; n < H; ++n) {
              const uint4 raw = *(const uint4*)(w0p + ((uint32_t)(n >> 3) * (kp0 / 8) + (uint32_t)c) * 128 +
                                                (uint32_t)(n & 7) * 16);
              const uint16_t* hv = (const uint16_t*)&raw;
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[i] = fmaf(dz[n], op_value<PREC>(hv[i]), acc[i]);
            }
            ((float4*)(dst + 8 * c))[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            ((float4*)(dst + 8 * c))[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
          }
        }
      }
    }
    if (stop) break;
    first_tile = false;
  }
  // ---- per-CTA partial dW: TMEM rows 0..H-1 (lane quarters 0..H/32-1), then dW_out
  tc_fence_before();
  const bool aborted = __syncthreads_or(*abort_flag != 0) != 0;
  tc_fence_after();
  float* part = partial + (size_t)blockIdx.x * (size_t)T.n_params;
  if (!aborted && (warp & 3) < H / 32) {
    const int m = (warp & 3) * 32 + lane;            // output neuron of this lane
    for (int l = 0; l < L; ++l) {
      const uint32_t kpl = A.L[l].kp;
      const int fan = l == 0 ? T.fan0 : H;           // row stride of W_l
      const int ncol = l == 0 ? T.nf : H;            // columns accumulated in TMEM
      for (uint32_t c0 = 16 * hf; c0 < kpl; c0 += 32) {
        float v[16];
        if (first_tile) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        } else {
          tmem_ld16(tmem + lane_base + T.dw_col[l] + c0, v);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if ((int)c0 + i < ncol) part[T.layer_off[l] + (int64_t)m * fan + c0 + i] = v[i];
      }
    }
  }
  __syncthreads();
  if (HASH)
    for (int n = tid; n < H; n += kTrainThreads) part[T.layer_off[0] + (int64_t)n * T.fan0 + T.nf] = dwg[n];
  for (int i = tid; i < 3 * H; i += kTrainThreads) part[T.layer_off[L] + i] = dwo[i];
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(loss, lsum * inv_n);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTrainCols);
}

// dW = scale * sum over CTAs of the partial rows: four running sums over the
// CTAs p = 0, 4, 8, ... / 1, 5, 9, ... / ..., each in CTA order, then
// (s0 + s1) + (s2 + s3) -- a fixed order, with four independent load chains.
__global__ void k_reduce_partials(const float* __restrict__ partial, int n_parts, int64_t n, float scale,
                                  float* __restrict__ dw) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int p = 0;
  for (; p + 4 <= n_parts; p += 4) {
    s0 += partial[(size_t)p * n + i];
    s1 += partial[(size_t)(p + 1) * n + i];
    s2 += partial[(size_t)(p + 2) * n + i];
    s3 += partial[(size_t)(p + 3) * n + i];
  }
  if (p < n_parts) s0 += partial[(size_t)p * n + i];
  if (p + 1 < n_parts) s1 += partial[(size_t)(p + 1) * n + i];
  if (p + 2 < n_parts) s2 += partial[(size_t)(p + 2) * n + i];
  dw[i] = ((s0 + s1) + (s2 + s3)) * scale;
}

// ---------------------------------------------------------------- training step, width 128
// Fields of width 128 (the render workloads' 4 x 128) do not fit the
// query-per-lane plan above: four resident weight matrices (132 KB) plus
// every layer's 128-query input tile exceed shared memory, and dW of all
// layers (144 + 3 x 128 columns) plus an accumulator exceed TMEM.  This
// kernel transposes the problem so that every MMA has M = 128 neurons (or
// input features) on the TMEM lanes and the tile's Q = 64 queries on the
// columns:
//   forward  : Z_l^T [n][q] = W_l [n][k] X_l^T [k][q]  (A = W_l K-major,
//              B = X_l; X_0 is stored query rows (K-major), X_{l>0} feature
//              rows with the queries contiguous (MN-major));
//              X_{l+1} = rnd(ReLU(Z_l)) written by the thread that owns
//              neuron n (one TMEM lane) as feature row n;
//   output   : y = W_out h on the CUDA cores from the unrounded last
//              activation, summed over the 128 neurons by a warp butterfly
//              per channel and over the four warps in shared memory;
//   backward : dW_l [n][k] += dZ_l [n][q] X_l [q][k]  (both K-major over q
//              for l > 0; X_0 MN-major), accumulated in TMEM across the
//              CTA's tiles for l > 0; dA_l^T [k][q] = W_l^T [k][n] dZ_l^T
//              [n][q] (A = W_l viewed MN-major, B = dZ_l MN-major), masked
//              by [X_l > 0] and rounded into dZ_{l-1};
//   dW_0     : 144 columns do not fit beside dW_1..3 (384) and the
//              accumulator (64), so each tile's dW_0 goes through the free
//              128 columns in two MMAs (features 0..127, then the rest) and
//              is summed in registers (72 per thread).
// TMEM: [0, 384) dW_1..3, [384, 448) accumulator, [448, 512) spare.
// Two warpgroups: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its neuron
// rows); warpgroup hf takes the query columns [32 hf, 32 hf + 32).
constexpr int kT128Threads = 256;
constexpr int kT128Q = 64;                         // queries per tile (MMA N)
constexpr uint32_t kT128RowGroup = kT128Q * 2 / 16 * 128;   // bytes between 8-row groups of a [row][q] tile
constexpr uint32_t kT128Acc = 384;                 // TMEM column of the forward / dA accumulator

struct T128Args {
  const uint8_t* wq;        // packed hidden-layer weights (k_pack_all layout)
  uint32_t wq_bytes;
  const float* w_out;       // [3][128] float32 output layer
  int n_hidden, in_freqs;
  uint32_t w_off[4], kp[4]; // packed layer offsets (bytes) and K extents
  uint32_t x_off[4];        // X_l tiles
  uint32_t dz_off, wout_off, dys_off, red_off, bar_off, smem_bytes;
  int64_t layer_off[6];
  int64_t n_params;
};

// 16 bytes (8 operands) of row r, query chunk c of a [row][q] tile (rows in
// groups of 8, the Q queries of a row contiguous in 16-byte chunks).
__device__ __forceinline__ uint32_t qrow_off(int r, int c) {
  return (uint32_t)(r >> 3) * kT128RowGroup + (uint32_t)c * 128 + (uint32_t)(r & 7) * 16;
}

template <int PREC>
__device__ __forceinline__ uint4 pack8(const float* v) {
  uint4 q;
  q.x = pack2<PREC>(v[0], v[1]); q.y = pack2<PREC>(v[2], v[3]);
  q.z = pack2<PREC>(v[4], v[5]); q.w = pack2<PREC>(v[6], v[7]);
  return q;
}

__device__ __forceinline__ bool op_positive(uint16_t h) { return (h & 0x8000u) == 0 && (h & 0x7FFFu) != 0; }

template <int PREC>
__global__ void __launch_bounds__(kT128Threads, 1) k_tc_train128(T128Args T, const float* __restrict__ q,
                                                                  const float* __restrict__ targets,
                                                                  const float* __restrict__ dy_in, int64_t B,
                                                                  float inv_n, float* __restrict__ partial,
                                                                  float* __restrict__ loss, uint32_t* err) {
  constexpr uint32_t AB = (PREC == PF_PREC_BF16) ? 1u : 0u;
  constexpr int H = 128;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int hf = warp >> 2, lq = warp & 3;
  const int n = lq * 32 + lane;                        // this thread's TMEM lane (neuron / feature row)
  const int L = T.n_hidden;
  float* w_out = (float*)(smem + T.wout_off);
  float* dys = (float*)(smem + T.dys_off);             // [Q][4] dy of the tile's queries
  float* red = (float*)(smem + T.red_off);             // [2][4][32][3] output-layer warp sums
  uint64_t* bars = (uint64_t*)(smem + T.bar_off);
  uint32_t* tmem_slot = (uint32_t*)(smem + T.bar_off + 16);
  int* abort_flag = (int*)(smem + T.bar_off + 20);
  const uint32_t bar_w = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  uint8_t* dz = smem + T.dz_off;

  if (tid == 0) {
    mbar_init(bar_w, 1);
    mbar_init(bar_mma, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 3 * H; i += kT128Threads) w_out[i] = T.w_out[i];
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    mbar_expect_tx(bar_w, T.wq_bytes);
    bulk_g2s(smem_u32(smem), T.wq, T.wq_bytes, bar_w);
  }
  if (!mbar_wait(bar_w, 0) && tid == 0) { atomicOr(err, PFE_ITER_CAP); *abort_flag = 1; }
  __syncthreads();

  const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
  const float wo0 = w_out[n], wo1 = w_out[H + n], wo2 = w_out[2 * H + n];
  constexpr int F = 12;                                // frequencies (the plan admits only 12)
  constexpr uint32_t kp0 = 12 * F;                     // 144 input features
  const uint32_t x0_rg = kp0 * 2 / 16 * 128;           // X_0: bytes between 8-query groups
  float dw0a[64], dw0b[8];
#pragma unroll
  for (int i = 0; i < 64; ++i) dw0a[i] = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) dw0b[i] = 0.f;
  float dwo0 = 0.f, dwo1 = 0.f, dwo2 = 0.f, lsum = 0.f;
  uint32_t phase = 0;
  bool first_tile = true;
  const int64_t n_tiles = (B + kT128Q - 1) / kT128Q;

  // A timed-out wait sets abort_flag; the CTA stops at the next MMA's
  // barrier, every thread alike (__syncthreads_or over their reads).
  auto pre_mma = [&]() -> bool {
    fence_proxy_async();
    tc_fence_before();
    const bool s = __syncthreads_or(*abort_flag != 0) != 0;
    tc_fence_after();
    return s;
  };
  auto commit_wait = [&]() {
    if (tid == 0) mma_commit(bar_mma);
    const bool ok = mbar_wait(bar_mma, phase);
    phase ^= 1u;
    tc_fence_after();
    if (!ok) { atomicOr(err, PFE_ITER_CAP); *abort_flag = 1; }
  };
  bool stop = false;
  // this thread's encoding inputs (items tid, tid + 256) and, for lane
  // quarter 0, its query's targets, loaded one tile ahead: the next tile's
  // loads are issued after the loss, so that they arrive during the backward
  constexpr int kItems = (kT128Q * 6 + kT128Threads - 1) / kT128Threads;
  float qn[kItems], tn[3] = {0.f, 0.f, 0.f};
  auto load_ahead = [&](int64_t tl) {
    const int64_t r0 = tl * kT128Q;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const int it = tid + j * kT128Threads;
      const int64_t row = r0 + (it & (kT128Q - 1));
      qn[j] = (tl < n_tiles && it < kT128Q * 6 && row < B) ? __ldg(q + 6 * row + it / kT128Q) : 0.f;
    }
    if (targets && lq == 0) {
      const int64_t row = r0 + 32 * hf + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c) tn[c] = (tl < n_tiles && row < B) ? __ldg(targets + 3 * row + c) : 0.f;
    }
  };
  load_ahead(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kT128Q;
    // ---- frequency encoding -> X_0 [q][k]: one (query, input) pair per item
    {
      uint8_t* x0 = smem + T.x_off[0];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const int it = tid + j * kT128Threads;
        if (it >= kT128Q * 6) break;
        const int qq = it & (kT128Q - 1), d = it / kT128Q;
        const float v = qn[j];
        float buf[8];
        float sn = 0.f, cs = 1.f;
#pragma unroll
        for (int k = 0; k < F; ++k) {
          pff::freq_next(v, k, sn, cs);
          buf[(2 * k) & 7] = sn;
          buf[(2 * k + 1) & 7] = cs;
          if (((2 * k + 2) & 7) == 0) {
            const int f0 = 2 * F * d + 2 * k + 2 - 8;             // first feature of the chunk
            *(uint4*)(x0 + (uint32_t)(qq >> 3) * x0_rg + (uint32_t)(f0 / 8) * 128 + (uint32_t)(qq & 7) * 16) =
                pack8<PREC>(buf);
          }
        }
      }
    }
    // ---- forward
    float h[32];
    for (int l = 0; l < L; ++l) {
      if ((stop = pre_mma())) break;
      if (tid == 0) {
        const uint32_t a0 = smem_u32(smem + T.w_off[l]), b0 = smem_u32(smem + T.x_off[l]);
        const uint32_t a_sbo = T.kp[l] * 2 / 16 * 128;
        const uint32_t id = idesc(AB, kT128Q, 0u, l > 0 ? 1u : 0u);
        for (int ks = 0; ks < (int)(T.kp[l] / 16); ++ks) {
          const uint64_t ad = sdesc(a0 + ks * 256, 128, a_sbo);
          const uint64_t bd = l == 0 ? sdesc(b0 + ks * 256, 128, x0_rg)
                                     : sdesc(b0 + ks * 2 * kT128RowGroup, kT128RowGroup, 128);
          mma<false>(tmem + kT128Acc, ad, bd, id, ks > 0 ? 1u : 0u);
        }
      }
      commit_wait();
      float v[32];
      tmem_ld32(lane_addr + kT128Acc + 32 * hf, v);
      if (l < L - 1) {
        uint8_t* xn = smem + T.x_off[l + 1];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float r[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) r[i] = fmaxf(v[8 * c + i], 0.f);
          *(uint4*)(xn + qrow_off(n, 4 * hf + c)) = pack8<PREC>(r);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) h[i] = fmaxf(v[i], 0.f);
      }
    }
    if (stop) break;
    // ---- output layer: y[q][c] = sum_n W_out[c][n] h[n][q] (butterfly over the
    // warp's 32 neurons, then the four warps in order)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float wc = c == 0 ? wo0 : (c == 1 ? wo1 : wo2);
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = wc * h[i];
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const int off = 16 >> s, half = 16 >> s;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
          const float send = up ? v[i] : v[half + i];
          const float keep = up ? v[half + i] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      red[((hf * 4 + lq) * 32 + lane) * 3 + c] = v[0];   // query 32 hf + lane, this warp's neurons
    }
    __syncthreads();
    if (lq == 0) {
      const int qq = 32 * hf + lane;
      const int64_t row = row0 + qq;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float y = ((red[((hf * 4 + 0) * 32 + lane) * 3 + c] + red[((hf * 4 + 1) * 32 + lane) * 3 + c]) +
                         red[((hf * 4 + 2) * 32 + lane) * 3 + c]) + red[((hf * 4 + 3) * 32 + lane) * 3 + c];
        float g = 0.f;
        if (row < B) {
          if (targets) {
            const float t = tn[c];
            const float den = t * t + 0.01f;
            const float diff = y - t;
            lsum += diff * diff / den;
            g = 2.f * diff / den;             // loss-scaled by 3B (see pf_tc_backward)
          } else {
            g = dy_in[3 * row + c];
          }
        }
        dys[4 * qq + c] = g;
      }
    }
    __syncthreads();
    load_ahead(tile + gridDim.x);
    // ---- dW_out (registers, across tiles) and dZ_{L-1} = rnd((dy W_out) * [rnd(h) > 0])
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float r[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int qi = 8 * c + i;
        const float4 dq = *(const float4*)(dys + 4 * (32 * hf + qi));
        dwo0 = fmaf(dq.x, h[qi], dwo0);
        dwo1 = fmaf(dq.y, h[qi], dwo1);
        dwo2 = fmaf(dq.z, h[qi], dwo2);
        const float dh = dq.x * wo0 + dq.y * wo1 + dq.z * wo2;
        const float hr = PREC == PF_PREC_BF16 ? pff::round_bf16(h[qi]) : pff::round_f16(h[qi]);
        r[i] = hr > 0.f ? dh : 0.f;
      }
      *(uint4*)(dz + qrow_off(n, 4 * hf + c)) = pack8<PREC>(r);
    }
    // ---- backward through the hidden layers l = L-1 .. 1
    for (int l = L - 1; l >= 1; --l) {
      if ((stop = pre_mma())) break;
      if (tid == 0) {
        const uint32_t dz0 = smem_u32(dz), xl = smem_u32(smem + T.x_off[l]), wl = smem_u32(smem + T.w_off[l]);
        // dW_l [n][k] (+)= dZ_l [n][q] X_l [q][k]: K = the tile's queries
        const uint32_t idw = idesc(AB, T.kp[l], 0u, 0u);
        const uint32_t dw_col = (uint32_t)(l - 1) * 128;
        for (int ks = 0; ks < kT128Q / 16; ++ks)
          mma<false>(tmem + dw_col, sdesc(dz0 + ks * 256, 128, kT128RowGroup), sdesc(xl + ks * 256, 128, kT128RowGroup),
                     idw, (first_tile && ks == 0) ? 0u : 1u);
        // dA_l^T [k][q] = W_l^T [k][n] dZ_l^T [n][q]: K = the layer's output neurons
        const uint32_t w_rg = T.kp[l] * 2 / 16 * 128;
        const uint32_t ida = idesc(AB, kT128Q, 1u, 1u);
        for (int ks = 0; ks < H / 16; ++ks)
          mma<false>(tmem + kT128Acc, sdesc(wl + ks * 2 * w_rg, w_rg, 128),
                     sdesc(dz0 + ks * 2 * kT128RowGroup, kT128RowGroup, 128), ida, ks > 0 ? 1u : 0u);
      }
      commit_wait();
      // dZ_{l-1} [k][q] = rnd(dA_l * [X_l > 0]), feature row k = this thread's lane
      float v[32];
      tmem_ld32(lane_addr + kT128Acc + 32 * hf, v);
      const uint8_t* xl = smem + T.x_off[l];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint4 raw = *(const uint4*)(xl + qrow_off(n, 4 * hf + c));
        const uint16_t* hv = (const uint16_t*)&raw;
        float r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = op_positive(hv[i]) ? v[8 * c + i] : 0.f;
        *(uint4*)(dz + qrow_off(n, 4 * hf + c)) = pack8<PREC>(r);
      }
    }
    if (stop) break;
    // ---- dW_0 of this tile through the free columns [384, 512): features
    // 0..127, then 128..143, each summed into registers
    {
      const uint32_t dz0 = smem_u32(dz), x0 = smem_u32(smem + T.x_off[0]);
      if ((stop = pre_mma())) break;
      if (tid == 0) {
        const uint32_t id = idesc(AB, 128, 0u, 1u);     // features 0..127
        for (int ks = 0; ks < kT128Q / 16; ++ks)
          mma<false>(tmem + kT128Acc, sdesc(dz0 + ks * 256, 128, kT128RowGroup),
                     sdesc(x0 + ks * 2 * x0_rg, x0_rg, 128), id, ks > 0 ? 1u : 0u);
      }
      commit_wait();
#pragma unroll
      for (int j = 0; j < 4; ++j) {                     // warpgroup hf: features 64 hf .. 64 hf + 63
        float v[16];
        tmem_ld16(lane_addr + kT128Acc + 64 * hf + 16 * j, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) dw0a[16 * j + i] += v[i];
      }
      {
        tc_fence_before();
        stop = __syncthreads_or(*abort_flag != 0) != 0;  // every thread has read the columns
        tc_fence_after();
        if (stop) break;
        if (tid == 0) {
          const uint32_t id = idesc(AB, 16, 0u, 1u);
          const uint32_t xb = x0 + (128 / 8) * 128;      // features 128.. (MN direction: 128 B per 8)
          for (int ks = 0; ks < kT128Q / 16; ++ks)
            mma<false>(tmem + kT128Acc, sdesc(dz0 + ks * 256, 128, kT128RowGroup),
                       sdesc(xb + ks * 2 * x0_rg, x0_rg, 128), id, ks > 0 ? 1u : 0u);
        }
        commit_wait();
        float v[16];
        tmem_ld16(lane_addr + kT128Acc, v);               // features 128..143; warpgroup hf takes 8 of them
#pragma unroll
        for (int i = 0; i < 8; ++i) dw0b[i] += v[8 * hf + i];
      }
    }
    first_tile = false;
  }
  // ---- this CTA's partial gradient row
  tc_fence_before();
  const bool aborted = __syncthreads_or(*abort_flag != 0) != 0;
  tc_fence_after();
  float* part = partial + (size_t)blockIdx.x * (size_t)T.n_params;
  if (!aborted) {
    for (int l = 1; l < L; ++l) {
      float* dst = part + T.layer_off[l] + (int64_t)n * H + 64 * hf;
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        if (first_tile) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        } else {
          tmem_ld16(lane_addr + (uint32_t)(l - 1) * 128 + 64 * hf + c0, v);
        }
#pragma unroll
        for (int i = 0; i < 16; i += 4) *(float4*)(dst + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
    }
    float* d0 = part + T.layer_off[0] + (int64_t)n * kp0;
#pragma unroll
    for (int i = 0; i < 64; i += 4) *(float4*)(d0 + 64 * hf + i) = make_float4(dw0a[i], dw0a[i + 1], dw0a[i + 2], dw0a[i + 3]);
#pragma unroll
    for (int i = 0; i < 8; i += 4) *(float4*)(d0 + 128 + 8 * hf + i) = make_float4(dw0b[i], dw0b[i + 1], dw0b[i + 2], dw0b[i + 3]);
  }
  // dW_out: the two warpgroups' sums, added in order
  __syncthreads();
  red[(hf * 3 + 0) * H + n] = dwo0;
  red[(hf * 3 + 1) * H + n] = dwo1;
  red[(hf * 3 + 2) * H + n] = dwo2;
  __syncthreads();
  if (!aborted)
    for (int i = tid; i < 3 * H; i += kT128Threads) part[T.layer_off[L] + i] = red[i] + red[3 * H + i];
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(loss, lsum * inv_n);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}


// ---------------------------------------------------------------- weight packing
// Hidden layer l packed K-major in 8 x 16-byte core matrices:
//   byte(n, k) = ((n/8) * (kp*eb/16) + (k*eb)/16) * 128 + (n%8) * 16 + (k*eb)%16
// values = operand rounding of W (fp8: code of W / s_w), zero for k >= fan_in.
struct Bounds { int64_t b[10]; float s_w[8]; int n; };

// All hidden layers packed in one launch (layout above): element e of the
// packed block belongs to layer l with first[l] <= e < first[l + 1] (H x kp_l elements
// each, in the order of k_pack).
struct PackAll {
  int64_t first[kMaxLayers + 1];
  int64_t w_off[kMaxLayers];
  uint32_t dst_off[kMaxLayers];
  int kp[kMaxLayers], fan_in[kMaxLayers];
  float inv_s[kMaxLayers];
  int n, prec;
};
__global__ void k_pack_all(const float* __restrict__ w, PackAll P, uint8_t* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.first[P.n]) return;
  int l = 0;
  while (l + 1 < P.n && e >= P.first[l + 1]) ++l;
  const int64_t le = e - P.first[l];
  const int kp = P.kp[l];
  const int n = (int)(le / kp), k = (int)(le % kp);
  const float x = k < P.fan_in[l] ? w[P.w_off[l] + (int64_t)n * P.fan_in[l] + k] : 0.f;
  const int eb = P.prec == PF_PREC_FP8 ? 1 : 2;
  uint8_t* d = dst + P.dst_off[l];
  const uint32_t off = (uint32_t)((n >> 3) * (kp * eb / 16) + (k * eb) / 16) * 128 + (uint32_t)(n & 7) * 16 +
                       (uint32_t)((k * eb) % 16);
  if (P.prec == PF_PREC_FP8) d[off] = pff::e4m3_code(x * P.inv_s[l]);
  else if (P.prec == PF_PREC_BF16) *(__nv_bfloat16*)(d + off) = __float2bfloat16_rn(x);
  else *(__half*)(d + off) = __float2half_rn(x);
}

// Hidden-layer weights rounded to the field precision (fp8: per-layer scale),
// as float values, for the SIMT path.
__global__ void k_round_weights(const float* __restrict__ w, float* __restrict__ wr, Bounds B, int prec) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.b[B.n]) return;
  int l = 0;
  while (l + 1 < B.n && i >= B.b[l + 1]) ++l;
  wr[i] = pff::round_prec(w[i], prec, B.s_w[l]);
}

// Shared-memory plan of a field for k_tc_forward (hash-grid fields: only as
// the first part of the training plan; their layer-0 operand is the 2 L F
// table features, g is added on the CUDA cores).
bool plan(const pf_field* f, TcArgs* A, bool for_train = false) {
  const int prec = f->desc.prec;
  if (prec == PF_PREC_F32) return false;
  const bool hash = f->desc.encoding == PF_ENC_HASHGRID;
  if (hash && (!for_train || (f->n_in - 1) % 16 != 0 || f->n_in - 1 > 256)) return false;
  const int H = f->desc.hidden;
  if (H != 64 && H != 128) return false;
  const int nh = f->n_layers - 1;
  if (nh < 1 || nh > kMaxLayers) return false;
  const uint32_t eb = prec == PF_PREC_FP8 ? 1 : 2;
  A->kstep = prec == PF_PREC_FP8 ? 32 : 16;
  A->n_hidden = nh;
  A->hidden = H;
  A->in_freqs = f->desc.in_freqs;
  A->prec = prec;
  A->psi = f->desc.psi;
  uint32_t off = 0, kmax = 0;
  for (int l = 0; l < nh; ++l) {
    uint32_t k = (uint32_t)f->fan_in[l];
    if (hash && l == 0) k -= 1;              // the g column is not an MMA operand
    uint32_t kp = (k + A->kstep - 1) / A->kstep * A->kstep;
    A->L[l].w_off = off;
    A->L[l].kp = kp;
    off += (uint32_t)H * kp * eb;
    kmax = std::max(kmax, kp);
    float s_a = prec == PF_PREC_FP8 ? f->scales_host[l] : 1.f;
    float s_w = prec == PF_PREC_FP8 ? f->scales_host[16 + l] : 1.f;
    A->L[l].dequant = s_a * s_w;
    A->L[l].inv_s_in = prec == PF_PREC_FP8 ? 1.f / s_a : 1.f;
  }
  A->wq_bytes = off;
  A->a_off = (off + 1023) / 1024 * 1024;
  A->a_bytes = kTileM * kmax * eb;
  // as many groups (tiles in flight) as TMEM (512 columns) and shared memory allow
  for (A->n_groups = 4; A->n_groups >= 1; A->n_groups /= 2) {
    A->wout_off = A->a_off + (uint32_t)A->n_groups * A->a_bytes;
    A->ypart_off = (A->wout_off + 3 * H * 4 + 15) / 16 * 16;
    A->bar_off = A->ypart_off + (uint32_t)A->n_groups * 3 * kTileM * 4;
    A->smem_bytes = A->bar_off + 64;
    if (A->n_groups * H <= 512 && A->smem_bytes <= 227 * 1024) break;
  }
  return A->n_groups >= 1;
}

}  // namespace

namespace {
// Shared-memory plan of k_tc_train128 (bf16 / f16, width 128, frequency
// encoding with 12 frequencies, 2..4 hidden layers).
bool plan_train128(const pf_field* f, T128Args* T) {
  if (f->desc.prec != PF_PREC_BF16 && f->desc.prec != PF_PREC_F16) return false;
  if (f->desc.hidden != 128 || f->desc.encoding == PF_ENC_HASHGRID) return false;
  const int F = f->desc.in_freqs;
  if (F != 12) return false;
  const int L = f->n_layers - 1;
  if (L < 2 || L > 4) return false;
  TcArgs A;
  if (!plan(f, &A, true)) return false;
  T->n_hidden = L;
  T->in_freqs = F;
  T->wq_bytes = A.wq_bytes;
  for (int l = 0; l < L; ++l) { T->w_off[l] = A.L[l].w_off; T->kp[l] = A.L[l].kp; }
  if (T->kp[0] != 144) return false;
  uint32_t off = (A.wq_bytes + 1023) / 1024 * 1024;
  T->x_off[0] = off;
  off += kT128Q * T->kp[0] * 2;
  for (int l = 1; l < L; ++l) { T->x_off[l] = off; off += kT128Q * 128 * 2; }
  T->dz_off = off;
  off += kT128Q * 128 * 2;
  T->wout_off = off;
  off += 3 * 128 * 4;
  T->dys_off = off;
  off += kT128Q * 4 * 4;
  T->red_off = off;
  off += 2 * 3 * 128 * 4;                          // >= [2][4][32][3] and [2][3][128] floats
  T->bar_off = (off + 15) / 16 * 16;
  T->smem_bytes = T->bar_off + 64;
  for (int l = 0; l <= f->n_layers; ++l) T->layer_off[l] = f->layer_off[l];
  T->n_params = f->layer_off[f->n_layers];
  return T->smem_bytes <= 227 * 1024;
}
}  // namespace

pf_status pf_tc_available(const pf_field* f) {
  TcArgs A;
  return plan(f, &A) ? PF_OK : PF_ERR_UNSUPPORTED;
}

pf_status pf_tc_forward(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B_max, const uint32_t* B_dev, float* out,
                        const uint32_t* slot_idx, const float* slot_alb, float* slot_li) {
  if (B_max <= 0) return PF_OK;
  TcArgs A;
  if (!plan(f, &A)) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "field shape not supported by the tensor-core path");
  A.wq = (const uint8_t*)f->wq;
  A.w_out = f->w + f->layer_off[f->n_layers - 1];
  int64_t tiles = (B_max + kTileM - 1) / kTileM;
  int grid = (int)std::min<int64_t>((tiles + A.n_groups - 1) / A.n_groups, (int64_t)ctx->num_sms);
  // two threads per row where shared memory holds at most two tiles in
  // flight (16-bit fields, 12 frequencies: the encoding splits at feature 72)
  const bool pair = f->desc.prec != PF_PREC_FP8 && A.n_groups <= 2 && A.in_freqs == 12 && A.L[0].kp == 144;
  const int tpr = pair ? 2 : 1;
  auto launch = [&](auto kern) -> pf_status {
    PF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A.smem_bytes));
    kern<<<grid, kThreads * tpr * A.n_groups, A.smem_bytes, ctx->stream>>>(A, q, B_max, B_dev, out, slot_idx,
                                                                            slot_alb, slot_li, ctx->err_dev);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  };
  if (f->desc.prec == PF_PREC_BF16)
    return pair ? launch(k_tc_forward<PF_PREC_BF16, 2>) : launch(k_tc_forward<PF_PREC_BF16, 1>);
  if (f->desc.prec == PF_PREC_F16)
    return pair ? launch(k_tc_forward<PF_PREC_F16, 2>) : launch(k_tc_forward<PF_PREC_F16, 1>);
  return launch(k_tc_forward<PF_PREC_FP8, 1>);
}

namespace {
bool plan_train(const pf_field* f, TrArgs* T) {
  if (f->desc.prec != PF_PREC_BF16 && f->desc.prec != PF_PREC_F16) return false;
  if (f->desc.hidden != kTrainHidden) return false;
  if (!plan(f, &T->f, true)) return false;
  const int L = T->f.n_hidden;
  const int H = T->f.hidden;
  T->hash = f->desc.encoding == PF_ENC_HASHGRID ? 1 : 0;
  T->fan0 = f->fan_in[0];
  T->nf = T->hash ? f->fan_in[0] - 1 : f->fan_in[0];
  uint32_t off = T->f.a_off;                 // weights first, then the activation tiles
  uint32_t col = (uint32_t)H;                // columns [0, H): forward and dA accumulators
  for (int l = 0; l < L; ++l) {
    T->a_off[l] = off;
    off += kTileM * T->f.L[l].kp * 2;
    T->dw_col[l] = col;
    col += T->f.L[l].kp;
  }
  if (col > kTrainCols) return false;
  off = (off + 1023) / 1024 * 1024;
  T->d_off = off;
  off += kTileM * kDK * 2;
  T->part_off = off;                         // dW_out partial sums of the 8 warps
  off += (kTrainThreads / 32) * 3 * 32 * 4;
  T->f.wout_off = off;
  off += 3 * H * 4;
  T->dwo_off = off;
  off += 3 * H * 4;
  T->g_off = off;                            // hash grids: g weights, g per row, dW of the g column
  off += (2 * H + kTileM) * 4;
  off = (off + 15) / 16 * 16;
  T->dys_off = off;
  off += 2 * kTileM * 4 * 4;                 // dy and the pair's partial outputs
  T->f.bar_off = (off + 15) / 16 * 16;
  T->f.smem_bytes = T->f.bar_off + 64;
  for (int l = 0; l <= f->n_layers; ++l) T->layer_off[l] = f->layer_off[l];
  T->n_params = f->layer_off[f->n_layers];   // the MLP's weights (hash tables are scattered separately)
  return T->f.smem_bytes <= 227 * 1024;
}
}  // namespace

pf_status pf_tc_backward_available(const pf_field* f) {
  TrArgs T;
  T128Args T2;
  return (plan_train(f, &T) || plan_train128(f, &T2)) ? PF_OK : PF_ERR_UNSUPPORTED;
}

pf_status pf_tc_backward(pf_ctx* ctx, const pf_field* f, const float* q, const float* dy, const float* targets,
                         int64_t B, float* dw, float* loss, const uint16_t* x_in, float* dx_out) {
  T128Args T2;
  if (plan_train128(f, &T2)) {
    T2.wq = (const uint8_t*)f->wq;
    T2.w_out = f->w + f->layer_off[f->n_layers - 1];
    const int64_t tiles = (B + kT128Q - 1) / kT128Q;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)ctx->num_sms);
    float* partial;
    PF_TRY(pf_scratch(ctx, WS_ACT, (size_t)grid * T2.n_params * sizeof(float), (void**)&partial));
    const float inv_n = targets ? 1.0f / (float)(3 * B) : 0.f;
    auto kern = f->desc.prec == PF_PREC_BF16 ? k_tc_train128<PF_PREC_BF16> : k_tc_train128<PF_PREC_F16>;
    PF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T2.smem_bytes));
    kern<<<grid, kT128Threads, T2.smem_bytes, ctx->stream>>>(T2, q, targets, dy, B, inv_n, partial, loss,
                                                             ctx->err_dev);
    PF_CUDA(ctx, cudaGetLastError());
    k_reduce_partials<<<(unsigned)((T2.n_params + 127) / 128), 128, 0, ctx->stream>>>(partial, grid, T2.n_params,
                                                                                     targets ? inv_n : 1.f, dw);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  }
  TrArgs T;
  if (!plan_train(f, &T)) return pf_fail(ctx, PF_ERR_UNSUPPORTED, "field shape not supported by the tensor-core backward");
  if (T.hash && (!x_in || !dx_out)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "hash-grid backward needs its features");
  T.f.wq = (const uint8_t*)f->wq;
  T.f.w_out = f->w + f->layer_off[f->n_layers - 1];
  T.x_in = x_in;
  T.dx_out = dx_out;
  T.w0 = f->w + f->layer_off[0];
  int64_t tiles = (B + kTileM - 1) / kTileM;
  int grid = (int)std::min<int64_t>(tiles, (int64_t)ctx->num_sms);
  float* partial;
  PF_TRY(pf_scratch(ctx, WS_ACT, (size_t)grid * T.n_params * sizeof(float), (void**)&partial));
  float inv_n = targets ? 1.0f / (float)(3 * B) : 0.f;
  auto launch = [&](auto kern) -> pf_status {
    PF_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T.f.smem_bytes));
    kern<<<grid, kTrainThreads, T.f.smem_bytes, ctx->stream>>>(T, q, targets, dy, B, inv_n, partial, loss,
                                                               ctx->err_dev);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  };
  if (T.hash) {
    if (f->desc.prec == PF_PREC_BF16) { PF_TRY(launch(k_tc_train<PF_PREC_BF16, true>)); }
    else { PF_TRY(launch(k_tc_train<PF_PREC_F16, true>)); }
  } else {
    if (f->desc.prec == PF_PREC_BF16) { PF_TRY(launch(k_tc_train<PF_PREC_BF16, false>)); }
    else { PF_TRY(launch(k_tc_train<PF_PREC_F16, false>)); }
  }
  k_reduce_partials<<<(unsigned)((T.n_params + 127) / 128), 128, 0, ctx->stream>>>(partial, grid, T.n_params,
                                                                                    targets ? inv_n : 1.f, dw);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

pf_status pf_field_pack(pf_ctx* ctx, pf_field* f) {
  if (f->desc.prec == PF_PREC_F32) return PF_OK;
  TcArgs A;
  const bool tc_fwd = plan(f, &A);
  TrArgs T;
  T128Args T2;
  const bool tc_bwd = f->desc.prec != PF_PREC_FP8 && (plan_train(f, &T) || plan_train128(f, &T2));
  // the float copy rounded to the field precision serves only the SIMT
  // kernels: needed unless every pass of this field runs on tcgen05
  const bool need_wr = !tc_fwd || (f->desc.prec != PF_PREC_FP8 && !tc_bwd);
  if (need_wr) {
    if (!f->wr) {
      // the MLP layers only (hash-grid tables are read from the master copy)
      const size_t nb = (size_t)f->layer_off[f->n_layers] * sizeof(float);
      if (cudaMalloc(&f->wr, nb) != cudaSuccess) return pf_fail(ctx, PF_ERR_OOM, "field pack");
      PF_CUDA(ctx, cudaMemsetAsync(f->wr, 0, nb, ctx->stream));
    }
    Bounds B;
    B.n = f->n_layers - 1;
    for (int l = 0; l <= B.n; ++l) B.b[l] = f->layer_off[l];
    for (int l = 0; l < 8; ++l) B.s_w[l] = f->scales_host[16 + l] > 0.f ? f->scales_host[16 + l] : 1.f;
    int64_t n = B.b[B.n];
    k_round_weights<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(f->w, f->wr, B, f->desc.prec);
    PF_CUDA(ctx, cudaGetLastError());
  }
  if (!tc_fwd && !tc_bwd) return PF_OK;
  if (!tc_fwd) A = T.f;                      // hash grids: packed for the training kernel only
  if (!f->wq || f->wq_bytes < A.wq_bytes) {
    cudaFree(f->wq);
    f->wq = nullptr;
    if (cudaMalloc(&f->wq, A.wq_bytes) != cudaSuccess) return pf_fail(ctx, PF_ERR_OOM, "field pack");
    f->wq_bytes = A.wq_bytes;
  }
  PackAll P;
  P.n = A.n_hidden;
  P.prec = f->desc.prec;
  P.first[0] = 0;
  for (int l = 0; l < A.n_hidden; ++l) {
    P.first[l + 1] = P.first[l] + (int64_t)A.hidden * A.L[l].kp;
    P.w_off[l] = f->layer_off[l];
    P.dst_off[l] = A.L[l].w_off;
    P.kp[l] = (int)A.L[l].kp;
    P.fan_in[l] = f->fan_in[l];
    const float s_w = f->desc.prec == PF_PREC_FP8 && f->scales_host[16 + l] > 0.f ? f->scales_host[16 + l] : 1.f;
    P.inv_s[l] = 1.f / s_w;
  }
  k_pack_all<<<(unsigned)((P.first[P.n] + 255) / 256), 256, 0, ctx->stream>>>(f->w, P, (uint8_t*)f->wq);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}
