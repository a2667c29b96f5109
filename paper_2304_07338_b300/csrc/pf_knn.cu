// Phase-selective k-nearest-neighbour radiance estimate (Sec. 3.3.1) over the
// photon records, the training targets of the paper's estimator:
//
//   L_s(x, w, g) = sum_{K nearest records of phase g} p_g(dir_n . w) Phi_n
//                  / ((4/3) pi r^3 sigma_cell(x))
//
// with r the K-th distance when the search ball (radius r_max, the staggered
// schedule's cap) holds at least K records and r_max otherwise.
//
// One warp per query.  The records of one (light, phase) are grouped by cache
// cell (CSR by key = (l*n_g + g)*res^3 + cell, cells x-fastest), so the cells
// of one row (fixed y, z) are one contiguous record range.  The ball is
// covered by the rows whose (y, z) cell rectangle meets it, each cut to the
// x-range of cells the ball reaches.  Passes over those ranges:
//   count      records in the rows, from the offsets alone: at most K means
//              every record within r_max is used (r = r_max, or the largest
//              distance if they are exactly K);
//   histogram  256 bins of d^3 / r_max^3 (monotone in d2) over the records
//              within r_max; at most K of them: all are used, as above;
//              else bin b* holds the K-th, and m more are needed from it;
//   refine     only if b* holds more than the selection list: radix rounds
//              on the 64-bit key (d2 bits, record id) inside b*, 8 bits at a
//              time, until the records sharing the key prefix fit the list;
//   select     accumulate the records below the prefix, gather the prefix's
//              records into shared memory, sort them by key (bitonic), and
//              accumulate the first m; r = sqrt(d2) of the m-th.
// "Nearest" is the order of (d2, record id) with d2 = (dx^2 + dy^2) + dz^2 in
// float32, each operation rounded: the selection is a pure function of the
// records, and the record id (photon << 4 | interaction slot) breaks ties.
#include "pf_internal.h"
#include <algorithm>
#include <cstdint>

namespace {

constexpr int kWarps = 8;      // queries per block (five blocks per SM: 48 registers)
constexpr int kBins = 256;     // histogram bins over d^3 / r_max^3
constexpr int kList = 256;     // selection list capacity (a power of two)

struct KnnArgs {
  const uint64_t* offsets;
  const float4* recs;          // 2 x float4 per record: (key, id, dir.x, dir.y), (dir.z, Phi)
  const float4* pos;           // (x, y, z, id bits) per record
  const float* cell_sigma;
  const float* q;
  int64_t B;
  int res, n_lights, n_g, K;
  float r_max, psi;
  float g_set[16];
  float* ls;
  float* lp;
  int32_t* k_out;
  float* r_out;
  const uint32_t* list;        // warp kernel: the queries to do (nullptr: all B, one warp each)
  const uint32_t* list_count;
};

struct Query {
  float x, y, z, r2, hs;       // position, r_max^2, histogram scale kBins / r_max^3
  float wx, wy, wz;            // outgoing direction
  float c0, c1, c2;            // HG: p = c0 / (c1 - c2 mu)^1.5
  int gi, ylo, yhi, zlo, zhi;
};

// Cells [lo, hi] along an axis that a ball of half-width rr around c can
// reach, widened by 1e-3 cells so that rounding never drops one.
__device__ __forceinline__ void axis_range(float c, float rr, int R, int* lo, int* hi) {
  const int l = (int)floorf((c - rr) * (float)R - 1e-3f);
  const int h = (int)floorf((c + rr) * (float)R + 1e-3f);
  *lo = max(l, 0);
  *hi = min(h, R - 1);
}

// Squared distance from c to the cell interval [i/R, (i+1)/R] (R a power of
// two: the products by 1/R are exact).
__device__ __forceinline__ float gap2(float c, int i, float inv_r) {
  const float lo = (float)i * inv_r, hi = (float)(i + 1) * inv_r;
  const float d = fmaxf(0.f, fmaxf(lo - c, c - hi));
  return d * d;
}

// Record range of row ri of the query's cover (ri -> light, z, y), or an
// empty range when the row's (y, z) rectangle misses the ball.
__device__ __forceinline__ void row_range(const KnnArgs& A, const Query& Q, int ri, int ny, int nz, uint64_t* s,
                                          uint32_t* len) {
  const int R = A.res;
  const int per_l = ny * nz;
  const int l = ri / per_l, rem = ri - l * per_l;
  const int cz = Q.zlo + rem / ny, cy = Q.ylo + rem % ny;
  *s = 0;
  *len = 0;
  const float inv_r = 1.0f / (float)R;
  const float gyz = (gap2(Q.z, cz, inv_r) + gap2(Q.y, cy, inv_r)) * (1.f - 1e-5f);
  if (gyz > Q.r2) return;
  const float rx = sqrtf(Q.r2 - gyz) * (1.f + 1e-5f) + 1e-7f;
  int xlo, xhi;
  axis_range(Q.x, rx, R, &xlo, &xhi);
  if (xlo > xhi) return;
  const int64_t row = (int64_t)(l * A.n_g + Q.gi) * ((int64_t)R * R * R) + (int64_t)R * (cy + (int64_t)R * cz);
  const uint64_t a = A.offsets[row + xlo], b = A.offsets[row + xhi + 1];
  *s = a;
  *len = (uint32_t)(b - a);
}

// Rows r0 .. r0+31 of the cover, one per lane: the lane's record range
// [s, s + len) and the running total inc over lanes 0..lane.
struct Chunk {
  uint64_t s;
  uint32_t len, inc, total;
};

__device__ __forceinline__ Chunk chunk_at(const KnnArgs& A, const Query& Q, int lane, int r0, int n_rows, int ny,
                                          int nz) {
  Chunk c;
  c.s = 0;
  c.len = 0;
  if (r0 + lane < n_rows) row_range(A, Q, r0 + lane, ny, nz, &c.s, &c.len);
  c.inc = c.len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, c.inc, o);
    if (lane >= o) c.inc += v;
  }
  c.total = __shfl_sync(0xffffffffu, c.inc, 31);
  return c;
}

// Calls f(n, d2, id) for the records of a chunk with d2 <= r_max^2.  The
// lanes walk the concatenation of the chunk's record ranges, each lane
// finding its row by a binary search over the lanes' running totals, so short
// rows leave no lane idle.
template <typename F>
__device__ __forceinline__ void walk_chunk(const KnnArgs& A, const Query& Q, int lane, const Chunk& c, F&& f) {
  for (uint32_t t0 = 0; t0 < c.total; t0 += 32) {
    const uint32_t t = t0 + lane;
    int j = 0;                                    // first lane whose running total exceeds t
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (__shfl_sync(0xffffffffu, c.inc, j + step - 1) <= t) j += step;
    const uint32_t inc_j = __shfl_sync(0xffffffffu, c.inc, j), len_j = __shfl_sync(0xffffffffu, c.len, j);
    const uint64_t s_j = __shfl_sync(0xffffffffu, c.s, j);
    if (t < c.total) {
      const uint64_t n = s_j + (t - (inc_j - len_j));
      const float4 p = __ldg(&A.pos[n]);
      const float dx = __fsub_rn(p.x, Q.x), dy = __fsub_rn(p.y, Q.y), dz = __fsub_rn(p.z, Q.z);
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      if (d2 <= Q.r2) f(n, d2, __float_as_uint(p.w));
    }
  }
}

// Calls f(n, d2, id) for every record n of the query's phase (all lights)
// with d2 <= r_max^2, the cover's rows taken 32 at a time (their offsets
// load in parallel).
template <typename F>
__device__ __forceinline__ void for_candidates(const KnnArgs& A, const Query& Q, int lane, F&& f) {
  const int ny = Q.yhi - Q.ylo + 1, nz = Q.zhi - Q.zlo + 1;
  if (ny <= 0 || nz <= 0) return;
  const int n_rows = A.n_lights * ny * nz;
  for (int r0 = 0; r0 < n_rows; r0 += 32) walk_chunk(A, Q, lane, chunk_at(A, Q, lane, r0, n_rows, ny, nz), f);
}

// Records in the rows covering the ball (offsets only).
__device__ __forceinline__ uint64_t row_total(const KnnArgs& A, const Query& Q, int lane) {
  const int ny = Q.yhi - Q.ylo + 1, nz = Q.zhi - Q.zlo + 1;
  if (ny <= 0 || nz <= 0) return 0;
  const int n_rows = A.n_lights * ny * nz;
  uint64_t T = 0;
  for (int ri = lane; ri < n_rows; ri += 32) {
    uint64_t s;
    uint32_t len;
    row_range(A, Q, ri, ny, nz, &s, &len);
    T += len;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) T += __shfl_xor_sync(0xffffffffu, T, o);
  return T;
}

__device__ __forceinline__ int bin_of(const Query& Q, float d2) {
  const float t = __fmul_rn(__fmul_rn(d2, __fsqrt_rn(d2)), Q.hs);
  return min((int)t, kBins - 1);
}

__device__ __forceinline__ uint64_t key_of(float d2, uint32_t id) {
  return ((uint64_t)__float_as_uint(d2) << 32) | id;
}

// The first bucket of h[0..nb) (nb = 32 * per) at which the running count
// reaches `need`; *below = the count in the buckets before it.
__device__ __forceinline__ int find_bucket(const uint32_t* h, int per, uint32_t need, int lane, uint32_t* below) {
  uint32_t mine = 0;
  for (int i = 0; i < per; ++i) mine += h[lane * per + i];
  uint32_t inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  const uint32_t exc = inc - mine;
  const unsigned hit = __ballot_sync(0xffffffffu, exc < need && need <= inc);
  const int src = __ffs(hit) - 1;
  int bucket = 0;
  uint32_t b = 0;
  if (lane == src) {
    uint32_t c = exc;
    for (int i = 0; i < per; ++i) {
      const uint32_t v = h[lane * per + i];
      if (c + v >= need) { bucket = lane * per + i; break; }
      c += v;
    }
    b = c;
  }
  bucket = __shfl_sync(0xffffffffu, bucket, src);
  *below = __shfl_sync(0xffffffffu, b, src);
  return bucket;
}

// The query's parameters: position, outgoing direction, phase, HG
// constants, r_max^2, histogram scale and the cover's cell ranges.
__device__ __forceinline__ Query make_query(const KnnArgs& A, int64_t b) {
  Query Q;
  const float* qb = A.q + 6 * b;
  Q.x = qb[0]; Q.y = qb[1]; Q.z = qb[2];
  float st, ct, sp, cp;
  sincospif(qb[3], &st, &ct);
  sincospif(2.0f * qb[4], &sp, &cp);
  Q.wx = st * cp; Q.wy = st * sp; Q.wz = ct;
  Q.gi = 0;
  for (int i = 0; i < A.n_g; ++i)
    if (A.g_set[i] == qb[5]) Q.gi = i;
  const float g = A.g_set[Q.gi];
  Q.c0 = 0.0795774715459476678f * (1.f - g * g);
  Q.c1 = 1.f + g * g;
  Q.c2 = 2.f * g;
  const float r_max = A.r_max;
  Q.r2 = __fmul_rn(r_max, r_max);
  Q.hs = (float)kBins / (Q.r2 * sqrtf(Q.r2));
  const int R = A.res;
  axis_range(Q.y, r_max, R, &Q.ylo, &Q.yhi);
  axis_range(Q.z, r_max, R, &Q.zlo, &Q.zhi);
  return Q;
}

// Mean sigma_t of the query's cache cell.
__device__ __forceinline__ float query_sigma(const KnnArgs& A, const Query& Q) {
  const int R = A.res;
  return A.cell_sigma[min(max((int)floorf(Q.x * (float)R), 0), R - 1) +
                      (int64_t)R * (min(max((int)floorf(Q.y * (float)R), 0), R - 1) +
                                    (int64_t)R * min(max((int)floorf(Q.z * (float)R), 0), R - 1))];
}

// L_s (and L') of query b from its sums, records used and radius.
__device__ __forceinline__ void write_query(const KnnArgs& A, int64_t b, float sig, float r, float a0, float a1,
                                            float a2, uint32_t kc) {
  const float vol = 4.18879032f * r * r * r;
  const float norm = (sig > 0.f && vol > 0.f) ? 1.0f / (vol * sig) : 0.f;
  const float L[3] = {a0 * norm, a1 * norm, a2 * norm};
  const float thr = exp10f(-A.psi);
  for (int c = 0; c < 3; ++c) {
    if (A.ls) A.ls[3 * b + c] = L[c];
    if (A.lp) A.lp[3 * b + c] = L[c] > thr ? -log10f(L[c]) / A.psi : 1.0f;
  }
  if (A.k_out) A.k_out[b] = (int32_t)kc;
  if (A.r_out) A.r_out[b] = r;
}

// One query on one warp (the histogram / selection passes of the file's
// header).
__device__ __forceinline__ void knn_warp(const KnnArgs& A, int64_t b, int lane, uint32_t* hist,
                                         unsigned long long* lkey, uint32_t* lidx, uint32_t* cnt_slot) {
  __syncwarp();                            // the previous query's shared-memory reads are done
  const Query Q = make_query(A, b);
  const float r_max = A.r_max;
  const int R = A.res;

  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  uint32_t kc = 0;
  auto add = [&](uint64_t n) {
    const float4 r0 = __ldg(&A.recs[2 * n]), r1 = __ldg(&A.recs[2 * n + 1]);
    const float mu = r0.z * Q.wx + r0.w * Q.wy + r1.x * Q.wz;
    const float den = Q.c1 - Q.c2 * mu;
    const float p = Q.c0 / (den * sqrtf(den));
    a0 = fmaf(p, r1.y, a0); a1 = fmaf(p, r1.z, a1); a2 = fmaf(p, r1.w, a2);
    kc += 1;
  };
  float r = r_max;
  const uint32_t K = (uint32_t)A.K;
  const float sig = query_sigma(A, Q);
  (void)R;
  // a cover of at most 32 rows is one chunk: its ranges stay in registers,
  // and if it holds at most K records they are all used at once
  const int ny = Q.yhi - Q.ylo + 1, nz = Q.zhi - Q.zlo + 1;
  const int n_rows = (ny > 0 && nz > 0) ? A.n_lights * ny * nz : 0;
  bool all, done = false;
  float dmax = 0.f;            // all-records path: largest d2 used (the K-th when exactly K)
  if (n_rows <= 32) {
    const Chunk c0 = chunk_at(A, Q, lane, 0, n_rows, ny, nz);
    all = c0.total <= K;
    if (all) {
      walk_chunk(A, Q, lane, c0, [&](uint64_t n, float d2, uint32_t) { add(n); dmax = fmaxf(dmax, d2); });
      done = true;
    }
  } else {
    all = row_total(A, Q, lane) <= (uint64_t)K;
  }
  int bstar = 0;
  uint32_t need = 0;
  if (!all) {
    for (int i = lane; i < kBins; i += 32) hist[i] = 0;
    __syncwarp();
    for_candidates(A, Q, lane, [&](uint64_t, float d2, uint32_t) { atomicAdd(&hist[bin_of(Q, d2)], 1u); });
    __syncwarp();
    uint32_t below = 0;
    uint32_t tot = 0;
    for (int i = lane; i < kBins; i += 32) tot += hist[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    all = tot <= K;
    if (!all) {
      bstar = find_bucket(hist, kBins / 32, K, lane, &below);
      need = K - below;
    }
  }
  if (all) {
    if (!done)
      for_candidates(A, Q, lane, [&](uint64_t n, float d2, uint32_t) { add(n); dmax = fmaxf(dmax, d2); });
  } else {
    // narrow bin b* by radix rounds on the key until its share fits the list
    uint32_t inF = hist[bstar];
    uint64_t prefix = 0;
    int shift = 64;
    __syncwarp();
    while (inF > (uint32_t)kList && shift > 0) {
      for (int i = lane; i < 256; i += 32) hist[i] = 0;
      __syncwarp();
      const int sh = shift - 8;
      for_candidates(A, Q, lane, [&](uint64_t, float d2, uint32_t id) {
        if (bin_of(Q, d2) != bstar) return;
        const uint64_t key = key_of(d2, id);
        if (shift < 64 && (key >> shift) != prefix) return;
        atomicAdd(&hist[(key >> sh) & 255u], 1u);
      });
      __syncwarp();
      uint32_t below = 0;
      const int bk = find_bucket(hist, 8, need, lane, &below);
      inF = hist[bk];
      need -= below;
      prefix = (prefix << 8) | (uint64_t)bk;
      shift = sh;
      __syncwarp();
    }
    if (lane == 0) *cnt_slot = 0;
    __syncwarp();
    for_candidates(A, Q, lane, [&](uint64_t n, float d2, uint32_t id) {
      const int bn = bin_of(Q, d2);
      if (bn < bstar) { add(n); return; }
      if (bn > bstar) return;
      const uint64_t key = key_of(d2, id);
      const uint64_t kp = shift < 64 ? (key >> shift) : 0;
      if (kp < prefix) { add(n); return; }
      if (kp > prefix) return;
      const uint32_t slot = atomicAdd(cnt_slot, 1u);
      if (slot < (uint32_t)kList) { lkey[slot] = key; lidx[slot] = (uint32_t)n; }
    });
    __syncwarp();
    const uint32_t cnt = min(*cnt_slot, (uint32_t)kList);
    int P2 = 32;
    while (P2 < (int)cnt) P2 <<= 1;
    for (int i = (int)cnt + lane; i < P2; i += 32) { lkey[i] = ~0ull; lidx[i] = 0; }
    __syncwarp();
    // bitonic sort of the list, ascending by key
    for (int kk = 2; kk <= P2; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P2; i += 32) {
          const int ij = i ^ j;
          if (ij > i) {
            const unsigned long long x = lkey[i], y = lkey[ij];
            const bool up = (i & kk) == 0;
            if ((x > y) == up) {
              lkey[i] = y; lkey[ij] = x;
              const uint32_t t = lidx[i]; lidx[i] = lidx[ij]; lidx[ij] = t;
            }
          }
        }
        __syncwarp();
      }
    const uint32_t take = min(need, cnt);
    for (uint32_t i = lane; i < take; i += 32) add(lidx[i]);
    if (take > 0) r = __fsqrt_rn(__uint_as_float((uint32_t)(lkey[take - 1] >> 32)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    kc += __shfl_xor_sync(0xffffffffu, kc, o);
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  if (all && kc >= K) r = __fsqrt_rn(dmax);
  if (lane == 0) write_query(A, b, sig, r, a0, a1, a2, kc);
}

// One warp per query.
__global__ void __launch_bounds__(32 * kWarps, 5) k_knn(KnnArgs A) {
  __shared__ uint32_t s_hist[kWarps][kBins];
  __shared__ unsigned long long s_key[kWarps][kList];
  __shared__ uint32_t s_idx[kWarps][kList];
  __shared__ uint32_t s_cnt[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kWarps + warp;
  if (b < A.B) knn_warp(A, b, lane, s_hist[warp], s_key[warp], s_idx[warp], &s_cnt[warp]);
}

// Persistent warps over the listed queries (those k_knn_thread passed on).
__global__ void __launch_bounds__(32 * kWarps, 5) k_knn_list(KnnArgs A) {
  __shared__ uint32_t s_hist[kWarps][kBins];
  __shared__ unsigned long long s_key[kWarps][kList];
  __shared__ uint32_t s_idx[kWarps][kList];
  __shared__ uint32_t s_cnt[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = *A.list_count;
  for (uint32_t i = blockIdx.x * kWarps + warp; i < n; i += gridDim.x * kWarps)
    knn_warp(A, (int64_t)A.list[i], lane, s_hist[warp], s_key[warp], s_idx[warp], &s_cnt[warp]);
}

// One thread per query: a query whose cover rows hold at most K records
// (offsets alone) uses every record within r_max, summed in row and record
// order; the others are listed for the warp kernel.  Most queries of the
// staggered schedule's small radii take this path.
__global__ void __launch_bounds__(128) k_knn_thread(KnnArgs A, uint32_t* __restrict__ list,
                                                   uint32_t* __restrict__ list_count) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  const Query Q = make_query(A, b);
  const int ny = Q.yhi - Q.ylo + 1, nz = Q.zhi - Q.zlo + 1;
  const int n_rows = (ny > 0 && nz > 0) ? A.n_lights * ny * nz : 0;
  uint64_t T = 0;
  for (int ri = 0; ri < n_rows; ++ri) {
    uint64_t s0;
    uint32_t len;
    row_range(A, Q, ri, ny, nz, &s0, &len);
    T += len;
  }
  if (T > (uint64_t)A.K) {
    list[atomicAdd(list_count, 1u)] = (uint32_t)b;
    return;
  }
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, dmax = 0.f;
  uint32_t kc = 0;
  for (int ri = 0; ri < n_rows; ++ri) {
    uint64_t s0;
    uint32_t len;
    row_range(A, Q, ri, ny, nz, &s0, &len);
    for (uint64_t n = s0; n < s0 + len; ++n) {
      const float4 p = __ldg(&A.pos[n]);
      const float dx = __fsub_rn(p.x, Q.x), dy = __fsub_rn(p.y, Q.y), dz = __fsub_rn(p.z, Q.z);
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      if (!(d2 <= Q.r2)) continue;
      const float4 r0 = __ldg(&A.recs[2 * n]), r1 = __ldg(&A.recs[2 * n + 1]);
      const float mu = r0.z * Q.wx + r0.w * Q.wy + r1.x * Q.wz;
      const float den = Q.c1 - Q.c2 * mu;
      const float ph = Q.c0 / (den * sqrtf(den));
      a0 = fmaf(ph, r1.y, a0); a1 = fmaf(ph, r1.z, a1); a2 = fmaf(ph, r1.w, a2);
      dmax = fmaxf(dmax, d2);
      ++kc;
    }
  }
  const float r = kc >= (uint32_t)A.K ? __fsqrt_rn(dmax) : A.r_max;
  write_query(A, b, query_sigma(A, Q), r, a0, a1, a2, kc);
}

}  // namespace

pf_status pf_knn_targets_impl(pf_ctx* ctx, const pf_cache* c, const float* q, int64_t B, int K, float r_max, float psi,
                              float* ls, float* lp, int32_t* k_out, float* r_out, cudaStream_t stream) {
  if (B == 0) return PF_OK;
  KnnArgs A;
  A.offsets = c->offsets; A.recs = c->recs; A.pos = c->pos; A.cell_sigma = c->cell_sigma;
  A.q = q; A.B = B; A.res = c->res; A.n_lights = c->n_lights; A.n_g = c->n_g; A.K = K;
  A.r_max = r_max; A.psi = psi;
  for (int i = 0; i < 16; ++i) A.g_set[i] = c->g_set[i];
  A.ls = ls; A.lp = lp; A.k_out = k_out; A.r_out = r_out;
  A.list = nullptr; A.list_count = nullptr;
  if (r_max * (float)c->res > 1.0f) {
    // covers wider than a cell in every direction: one warp per query
    k_knn<<<(unsigned)((B + kWarps - 1) / kWarps), 32 * kWarps, 0, stream>>>(A);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  }
  // small covers: one thread per query first; the queries with more than K
  // records in their cover go to the warp kernel through a list
  uint32_t* list;
  PF_TRY(pf_scratch(ctx, WS_KNN_LIST, ((size_t)B + 64) * sizeof(uint32_t), (void**)&list));
  uint32_t* count = list + B + 32;
  PF_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(uint32_t), stream));
  k_knn_thread<<<(unsigned)((B + 127) / 128), 128, 0, stream>>>(A, list, count);
  PF_CUDA(ctx, cudaGetLastError());
  A.list = list; A.list_count = count;
  const int64_t blocks = std::min<int64_t>((B + kWarps - 1) / kWarps, (int64_t)ctx->num_sms * 5);
  k_knn_list<<<(unsigned)blocks, 32 * kWarps, 0, stream>>>(A);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

extern "C" pf_status pf_estimate_targets_knn(pf_ctx* ctx, const pf_cache* c, const float* q, int64_t B, int K,
                                             float r_max, float psi, float* ls, float* lp, int32_t* k_out,
                                             float* r_out) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  if (!c || (!q && B > 0) || B < 0 || B >= (1ll << 40) || !(psi > 0.f))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "bad KNN estimate arguments");
  if (K < 1 || K > (1 << 20)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "K must be in [1, 2^20]");
  if (!(r_max > 0.f && r_max <= 2.f)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "r_max must be in (0, 2]");
  DeviceGuard dg(ctx->device);
  return pf_knn_targets_impl(ctx, c, q, B, K, r_max, psi, ls, lp, k_out, r_out, ctx->stream);
}
