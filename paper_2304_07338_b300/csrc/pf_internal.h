// Host-side internals of libpf: context, cache and field objects, scratch
// arena, error plumbing.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include "../../include/pf.h"

// Device error word codes (bitwise OR of all that happened).
enum : uint32_t { PFE_ITER_CAP = 1u, PFE_NONFINITE = 2u, PFE_OVERFLOW = 4u };

// Scratch slots of the context arena.
enum ScratchSlot {
  WS_REDUCE = 0, WS_SCAN, WS_QUERY, WS_TARGET, WS_ACT, WS_GRAD, WS_SAMPLES, WS_SLOT_LD, WS_SLOT_ALB,
  WS_SLOT_LI, WS_COMPACT_Q, WS_COMPACT_IDX, WS_LOSS, WS_MISC, WS_GRID, WS_COMPACT_DIR, WS_CELL_HIST, WS_CELL_OFF, WS_CELL_KEY, WS_CELL_PERM, WS_VMASK, WS_GRID_PRIMARY, WS_GRID_SHADOW, WS_HASH_X, WS_HASH_DX, WS_TRACE_SLOTS, WS_TRACE_POS, WS_TRACE_NREC, WS_TRACE_CURSOR, WS_TRACE_TALLY,
  WS_TRACE_OPOS, WS_NEE_CONTRIB, WS_KNN_LIST, WS_GRID_WALK, WS_GRID_PRIMARY_WALK, WS_GRID_SHADOW_WALK, WS_COUNT
};

struct pf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 148;
  uint32_t* err_dev = nullptr;        // device error word
  double* dbl_dev = nullptr;          // small FP64 scratch (reductions)
  unsigned long long* counters = nullptr;  // optional work counters (caller-owned)
  int timing = 0;                         // record per-stage CUDA events
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;                // recorded (stage, start, end) pairs
  std::vector<cudaEvent_t> event_pool;
  cudaStream_t aux = nullptr;             // second stream (training-batch prefetch), created on first use
  cudaEvent_t aux_ev[5] = {};             // its events: batch ready x2, batch consumed x2, fork
  void* ws[WS_COUNT] = {};
  size_t ws_size[WS_COUNT] = {};
  std::string last_error;
};

struct pf_cache {
  pf_ctx* ctx = nullptr;              // creating context (not dereferenced when freed)
  int device = 0;
  int res = 0, n_lights = 0, n_g = 0, max_bounces = 0;
  int64_t n_photons = 0, n_records = 0, n_keys = 0, n_occupied = 0;
  float g_set[16] = {};
  // device arrays
  uint32_t* counts = nullptr;         // [n_keys]
  uint64_t* offsets = nullptr;        // [n_keys + 1]
  float4* recs = nullptr;             // CSR records, 2 x float4 each
  float4* pos = nullptr;              // CSR record positions (x, y, z, record id bits)
  float* flux = nullptr;              // [n_keys * 3]
  uint32_t* occupied = nullptr;       // [n_occupied]
  float* cell_sigma = nullptr;        // [res^3]
  double tally[15] = {};
};

struct pf_field {
  pf_ctx* ctx = nullptr;              // creating context (not dereferenced when freed)
  int device = 0;
  pf_field_desc desc{};
  int n_in = 0, n_layers = 0;
  int64_t n_params = 0;
  int64_t layer_off[16] = {};         // offsets into the flat weight vector
  int fan_in[16] = {}, fan_out[16] = {};
  float* w = nullptr;                 // master weights f32 [n_params]
  float* m = nullptr;                 // Adam moments
  float* v = nullptr;
  void* wq = nullptr;                 // packed low-precision weights (tensor-core layout)
  float* wr = nullptr;                // hidden-layer weights rounded to the field precision (f32 values)
  size_t wq_bytes = 0;
  float* scales = nullptr;            // fp8: s_a[l], s_w[l] (device, 2 x 16)
  float scales_host[32] = {};
  int fp8_ready = 0;
  int step = 0;                       // Adam step counter
  // hash-grid encoding: per grid (0 position, 1 direction) and level the
  // cells per axis, table entries, dense flag (bit l) and the float offset of
  // the level's table in the flat parameters
  int hash_res[2][16] = {};
  uint32_t hash_entries[2][16] = {};
  uint32_t hash_dense[2] = {};
  int64_t hash_off[2][16] = {};
};

// Stage timing (PF_STAGE_* of pf.h): wraps a stage's launches in events.
struct StageTimer {
  pf_ctx* ctx; int stage; cudaEvent_t a = nullptr, b = nullptr;
  StageTimer(pf_ctx* c, int st);
  ~StageTimer();
};

// Status helpers.
pf_status pf_fail(pf_ctx* ctx, pf_status st, const char* fmt, ...);
pf_status pf_cuda_check(pf_ctx* ctx, cudaError_t e, const char* what);
#define PF_CUDA(ctx, call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return pf_cuda_check(ctx, e_, #call); } while (0)
#define PF_TRY(expr) do { pf_status s_ = (expr); if (s_ != PF_OK) return s_; } while (0)

// The context's second stream and its events, created on first use.
pf_status pf_aux_stream(pf_ctx* ctx);

// Scratch arena: returns a device buffer of at least `bytes` for `slot`.
pf_status pf_scratch(pf_ctx* ctx, int slot, size_t bytes, void** out);
// Enter the context's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) { cudaGetDevice(&prev); if (prev != dev) cudaSetDevice(dev); }
  ~DeviceGuard() { int cur; cudaGetDevice(&cur); if (prev >= 0 && cur != prev) cudaSetDevice(prev); }
};

// Volume validation and majorant.  The *_problem forms need no context: on a
// problem they write a message into buf and return true.
bool pf_volume_problem(const pf_volume* vol, char* buf, size_t len);
bool pf_lights_problem(const pf_light* lights, int n, char* buf, size_t len);
pf_status pf_check_volume(pf_ctx* ctx, const pf_volume* vol);
pf_status pf_majorant_impl(pf_ctx* ctx, const pf_volume* vol, float* out);
pf_status pf_check_lights(pf_ctx* ctx, const pf_light* lights, int n);
// Brick majorants of a volume: the caller's array, or computed into scratch.
pf_status pf_grid_for(pf_ctx* ctx, const pf_volume* vol, const float** grid);
// Copy of a brick-majorant grid (gx x gy x gz, x fastest) with a border of
// two zero bricks on every side, (gx + 4) x (gy + 4) x (gz + 4): the grid the
// trackers' walks read (scratch slot `slot`).  PF_ERR_INVALID_ARG when the
// bordered grid has 2^31 bricks or more.
pf_status pf_bordered_grid(pf_ctx* ctx, const float* grid, int gx, int gy, int gz, int slot, const float** out);

// Device-wide exclusive scan of u32 counts into u64 offsets (n+1 entries).
pf_status pf_scan_u32(pf_ctx* ctx, const uint32_t* in, uint64_t* out, int64_t n);
// Reads the error word; returns PF_ERR_TIMEOUT / PF_ERR_NUMERIC if set (and clears it).
pf_status pf_check_error_word(pf_ctx* ctx);

// Field internals used by the renderer and the trainer.
// Field forward over B_max query rows (B_dev, when given, holds the actual
// row count on the device).  out (nullable) receives L'; with slot_idx given,
// the render epilogue writes slot_li[slot] = albedo * 10^(-psi L') instead.
pf_status pf_field_forward_impl(pf_ctx* ctx, const pf_field* f, const float* q, int64_t B_max,
                                const uint32_t* B_dev, float* out, const uint32_t* slot_idx,
                                const float* slot_alb, float* slot_li);
pf_status pf_field_pack(pf_ctx* ctx, pf_field* f);
// KNN radiance estimate (see pf_estimate_targets_knn) on `stream`; ls, lp,
// k_out, r_out nullable.
pf_status pf_knn_targets_impl(pf_ctx* ctx, const pf_cache* c, const float* q, int64_t B, int K, float r_max, float psi,
                              float* ls, float* lp, int32_t* k_out, float* r_out, cudaStream_t stream);
