// Multi-phase photon tracing (Algorithm 1, Sec. 3.2) and the photon caches
// the training-sample generator reads (Sec. 3.3).
//
// Pipeline (all stream-ordered, no host round trip except two scalars):
//   k_trace_photons  persistent warps, one photon per lane at a time (lanes
//                    refill from a global counter); emission, delta tracking,
//                    HG scattering, Russian roulette; record j (j >= 2) goes to
//                    the photon's own slot p*(max_bounces-1) + j-2 -- so no
//                    global append counter -- and bumps counts[key]; the
//                    interaction position goes to a parallel slot array;
//   scan(counts)     -> CSR offsets;
//   k_scatter        slot records -> CSR order (position within a key taken
//                    by an atomic cursor), positions with them (x, y, z, id)
//                    for the KNN estimate;
//   k_key_flux       per-key power sums in FP64 -> float (thread per key);
//   k_cell_sigma     mean sigma_t over the voxel centres of every cache cell;
//   k_occupancy + scan + k_occupied_list -> ascending occupied cells.
// Compiled with -fmad=false: see pf_device.cuh.
#include "pf_internal.h"
#include "pf_device.cuh"
#include <algorithm>
#include <cmath>

using namespace pfd;

namespace {

struct TraceArgs {
  Vol V;
  DevLights L;
  float g_set[16];
  int n_g, max_bounces, res, use_rr;
  uint64_t N, seed, n_photons;
};

// Persistent warps (one per block) that refill: a photon path's length
// varies a lot (most photons leave the box after zero or one collision, a
// few scatter a dozen times), so a thread per photon leaves most lanes idle
// while the warp's longest path finishes.  Here every lane carries one photon
// at a time and the loop body advances each lane by one interaction; a lane
// whose photon is finished takes the next photon id from a global counter
// (one atomic per warp and round).  A photon's arithmetic and random numbers
// are those of a thread-per-photon tracer (its Philox stream is its id), so
// records and bins do not depend on which lane traced it.  FP64 tallies
// accumulate per lane in shared memory; each block writes one row of
// tally_part, summed by k_tally_reduce.
constexpr int kTraceThreads = 32;
template <int DT>
__global__ void __launch_bounds__(kTraceThreads, 32) k_trace_photons(TraceArgs A, float4* __restrict__ slots,
                                                       float4* __restrict__ slot_pos, uint8_t* __restrict__ nrec, uint32_t* __restrict__ counts,
                                                       unsigned long long* __restrict__ next, double* __restrict__ tally_part,
                                                       uint32_t* err) {
  __shared__ double s_t[15][kTraceThreads];        // emitted, escaped, absorbed, truncated, RR net (x 3 channels)
  const int lane = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 15; ++i) s_t[i][lane] = 0.0;
  const Vol& V = A.V;
  const int S = A.max_bounces - 1 > 0 ? A.max_bounces - 1 : 1;
  const uint32_t R = (uint32_t)A.res;
  bool has = false;
  uint64_t p = 0;
  int l = 0, gi = 0, j = 0, n = 0;
  float g = 0.f, t = 0.f, t1 = 0.f, P0 = 0.f, P1 = 0.f, P2 = 0.f, pe_max = 1.f;
  V3 o = v3(0.f, 0.f, 0.f), d = o;
  Rng rng(0, 0, 0, 0);
  uint32_t nfetch = 0;
  auto finish = [&](bool escaped) {
    if (escaped) { s_t[3][lane] += P0; s_t[4][lane] += P1; s_t[5][lane] += P2; }
    nrec[p] = (uint8_t)n;
    has = false;
  };
  for (;;) {
    // refill the lanes without a photon
    const unsigned need = __ballot_sync(0xffffffffu, !has);
    bool exhausted = false;
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      exhausted = base + (unsigned long long)__popc(need) >= A.n_photons;
      if (!has) {
        const uint64_t qid = base + (uint64_t)__popc(need & ((1u << lane) - 1u));
        if (qid < A.n_photons) {
          p = qid;
          has = true;
          l = (int)(p / ((uint64_t)A.n_g * A.N));
          gi = (int)((p / A.N) % (uint64_t)A.n_g);
          const DevLight& Lt = A.L.l[l];
          g = A.g_set[gi];
          rng = Rng(A.seed, TAG_PHOTON, p, 0);
          float u[4]; rng.uni4(u);
          if (Lt.kind == 0) {
            V3 v = normalize(v3(Lt.v[0], Lt.v[1], Lt.v[2]));
            V3 e1, e2; onb(v, &e1, &e2);
            float side = 1.7320508075688772f;
            float a = (u[0] - 0.5f) * side, b = (u[1] - 0.5f) * side;
            o = v3(0.5f + v.x + a * e1.x + b * e2.x, 0.5f + v.y + a * e1.y + b * e2.y, 0.5f + v.z + a * e1.z + b * e2.z);
            d = v3(-v.x, -v.y, -v.z);
            P0 = Lt.rgb[0] * 3.0f / (float)A.N; P1 = Lt.rgb[1] * 3.0f / (float)A.N; P2 = Lt.rgb[2] * 3.0f / (float)A.N;
          } else {
            float z = 1.0f - 2.0f * u[0];
            float r = sqrtf(mx(0.0f, 1.0f - z * z));
            float sp, cp; own_sincos2pif(u[1], &sp, &cp);
            d = v3(r * cp, r * sp, z);
            o = v3(Lt.v[0], Lt.v[1], Lt.v[2]);
            const float fpi = 12.566370614359172f;
            P0 = Lt.rgb[0] * fpi / (float)A.N; P1 = Lt.rgb[1] * fpi / (float)A.N; P2 = Lt.rgb[2] * fpi / (float)A.N;
          }
          s_t[0][lane] += P0; s_t[1][lane] += P1; s_t[2][lane] += P2;
          pe_max = mx(P0, mx(P1, P2));
          n = 0; j = 0;
          float t0_ = 0.f, t1_ = 0.f;
          if (box_hit(o, d, &t0_, &t1_)) { t = t0_; t1 = t1_; }
          else finish(true);                       // misses the box: escapes at once
        }
      }
    }
    // a warp leaves only when it is idle and the counter has run out (its
    // new photons may all have missed the box and finished at once)
    if (!__any_sync(0xffffffffu, has)) {
      if (exhausted) break;
      continue;
    }
    if (!has) continue;
    // one interaction of this lane's photon
    float th;
    if (!delta_track<DT>(V, o, d, t, t1, rng, &th, err, nfetch)) { finish(true); continue; }
    const V3 x = along(o, d, th);
    j = j + 1;
    float sig; V3 alb;
    medium_at<DT>(V, x, &sig, &alb);
    if (j >= 2) {
      int bx = (int)floorf(x.x * (float)A.res), by = (int)floorf(x.y * (float)A.res), bz = (int)floorf(x.z * (float)A.res);
      bx = min(max(bx, 0), A.res - 1); by = min(max(by, 0), A.res - 1); bz = min(max(bz, 0), A.res - 1);
      const uint32_t bin = (uint32_t)bx + R * ((uint32_t)by + R * (uint32_t)bz);
      const uint32_t key = (uint32_t)(l * A.n_g + gi) * (R * R * R) + bin;
      float4* my = slots + 2 * (size_t)p * S;
      my[2 * n + 0] = make_float4(__uint_as_float(key), __uint_as_float((uint32_t)(p << 4) | (uint32_t)n), d.x, d.y);
      my[2 * n + 1] = make_float4(d.z, P0, P1, P2);
      slot_pos[(size_t)p * S + n] = make_float4(x.x, x.y, x.z, 0.0f);
      atomicAdd(&counts[key], 1u);
      n = n + 1;
    }
    const float Q0 = P0 * alb.x, Q1 = P1 * alb.y, Q2 = P2 * alb.z;
    s_t[6][lane] += (double)P0 - (double)Q0; s_t[7][lane] += (double)P1 - (double)Q1; s_t[8][lane] += (double)P2 - (double)Q2;
    P0 = Q0; P1 = Q1; P2 = Q2;
    if (j == A.max_bounces) {
      s_t[9][lane] += P0; s_t[10][lane] += P1; s_t[11][lane] += P2;
      finish(false);
      continue;
    }
    float w[4]; rng.uni4(w);
    const V3 nd = hg_sample(g, d, w[0], w[1]);
    if (A.use_rr && j >= 3) {
      float q = mx(P0, mx(P1, P2)) / pe_max;
      if (q > 1.0f) q = 1.0f;
      if (!(w[2] < q)) {
        s_t[12][lane] += P0; s_t[13][lane] += P1; s_t[14][lane] += P2;
        finish(false);
        continue;
      }
      const float n0 = P0 / q, n1 = P1 / q, n2 = P2 / q;
      s_t[12][lane] -= (double)n0 - (double)P0; s_t[13][lane] -= (double)n1 - (double)P1; s_t[14][lane] -= (double)n2 - (double)P2;
      P0 = n0; P1 = n1; P2 = n2;
    }
    o = x; d = nd;
    float a0, a1;
    if (!box_hit(o, d, &a0, &a1)) { finish(true); continue; }
    t = 0.0f; t1 = a1;
  }
  // the block's (warp's) FP64 tallies: one row of tally_part
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    double v = s_t[i][lane];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) tally_part[(size_t)blockIdx.x * 15 + i] = v;
  }
}

// tally[i] += sum over the rows of tally_part (FP64; tally zeroed first).
// The rows are read as one contiguous array; with 240 threads per block and a
// grid stride that is a multiple of 15, every thread always meets the same
// tally index.
constexpr int kTallyThreads = 240;
__global__ void __launch_bounds__(kTallyThreads) k_tally_reduce(const double* __restrict__ part, int64_t rows,
                                                              double* __restrict__ tally) {
  __shared__ double s[15];
  if (threadIdx.x < 15) s[threadIdx.x] = 0.0;
  __syncthreads();
  const int64_t n = rows * 15;
  const int64_t stride = (int64_t)gridDim.x * kTallyThreads;
  double v = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kTallyThreads + threadIdx.x; e < n; e += stride) v += part[e];
  atomicAdd(&s[threadIdx.x % 15], v);
  __syncthreads();
  if (threadIdx.x < 15) atomicAdd(&tally[threadIdx.x], s[threadIdx.x]);
}

// Move slot records into CSR order.
__global__ void k_scatter(const float4* __restrict__ slots, const float4* __restrict__ slot_pos,
                          const uint8_t* __restrict__ nrec, uint64_t n_photons, int S,
                          const uint64_t* __restrict__ offsets, uint32_t* __restrict__ cursor, float4* __restrict__ recs,
                          float4* __restrict__ rpos) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t p = i / (uint64_t)S;
  int s = (int)(i % (uint64_t)S);
  if (p >= n_photons || s >= (int)nrec[p]) return;
  float4 a = slots[2 * i], b = slots[2 * i + 1];
  uint32_t key = __float_as_uint(a.x);
  uint64_t pos = offsets[key] + atomicAdd(&cursor[key], 1u);
  recs[2 * pos] = a;
  recs[2 * pos + 1] = b;
  float4 x = slot_pos[i];
  x.w = a.y;                                   // record id: the KNN tie-break
  rpos[pos] = x;
}

// Per-key power sums: one thread per key (keys hold few records on average),
// FP64, rounded once.
__global__ void k_key_flux(const float4* __restrict__ recs, const uint64_t* __restrict__ offsets, int64_t n_keys,
                           float* __restrict__ flux) {
  const int64_t key = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (key >= n_keys) return;
  double s0 = 0, s1 = 0, s2 = 0;
  for (uint64_t n = offsets[key]; n < offsets[key + 1]; ++n) {
    const float4 b = recs[2 * n + 1];
    s0 += b.y; s1 += b.z; s2 += b.w;
  }
  flux[3 * key] = (float)s0; flux[3 * key + 1] = (float)s1; flux[3 * key + 2] = (float)s2;
}

// First voxel index whose centre lies in cache cell c (axis of n voxels, res cells).
__device__ __forceinline__ int cell_lo(int c, int n, int res) {
  long long a = 2LL * n * c - res;
  if (a <= 0) return 0;
  return (int)((a + 2LL * res - 1) / (2LL * res));
}

template <int DT>
__global__ void k_cell_sigma(Vol V, int res, float* __restrict__ out) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nc = (int64_t)res * res * res;
  if (c >= nc) return;
  int cx = (int)(c % res), cy = (int)((c / res) % res), cz = (int)(c / ((int64_t)res * res));
  int x0 = cell_lo(cx, V.nx, res), x1 = cx + 1 < res ? cell_lo(cx + 1, V.nx, res) : V.nx;
  int y0 = cell_lo(cy, V.ny, res), y1 = cy + 1 < res ? cell_lo(cy + 1, V.ny, res) : V.ny;
  int z0 = cell_lo(cz, V.nz, res), z1 = cz + 1 < res ? cell_lo(cz + 1, V.nz, res) : V.nz;
  float sum = 0.f;
  int cnt = 0;
  for (int k = z0; k < z1; ++k)
    for (int j = y0; j < y1; ++j)
      for (int i = x0; i < x1; ++i) {
        sum += V.sigma_scale * tf_alpha(V, voxel<DT>(V, i, j, k));
        ++cnt;
      }
  if (cnt > 0) out[c] = sum / (float)cnt;
  else out[c] = sigma_at<DT>(V, v3((cx + 0.5f) / res, (cy + 0.5f) / res, (cz + 0.5f) / res));
}

__global__ void k_occupancy(const uint32_t* __restrict__ counts, const float* __restrict__ csig, int64_t nc, int nlg,
                            uint32_t* __restrict__ flag) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  uint32_t tot = 0;
  for (int a = 0; a < nlg; ++a) tot += counts[(int64_t)a * nc + c];
  flag[c] = (tot > 0 && csig[c] > 0.f) ? 1u : 0u;
}

__global__ void k_occupied_list(const uint32_t* __restrict__ flag, const uint64_t* __restrict__ pos, int64_t nc,
                                uint32_t* __restrict__ occ) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || !flag[c]) return;
  occ[pos[c]] = (uint32_t)c;
}

// Brick majorant: min / max density over the brick plus a one-voxel apron
// (and 0 on the box boundary), largest TF alpha over that range, margin 2^-10.
template <int DT>
__global__ void k_brick_majorants(Vol V, float* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)V.gx * V.gy * V.gz;
  if (b >= nb) return;
  const int bx = (int)(b % V.gx), by = (int)((b / V.gx) % V.gy), bz = (int)(b / ((int64_t)V.gx * V.gy));
  float dmin = __int_as_float(0x7f800000), dmax = -dmin;
  const int B = V.B;
  for (int k = max(B * bz - 1, 0); k <= min(B * bz + B, V.nz - 1); ++k)
    for (int j = max(B * by - 1, 0); j <= min(B * by + B, V.ny - 1); ++j)
      for (int i = max(B * bx - 1, 0); i <= min(B * bx + B, V.nx - 1); ++i) {
        const float d = voxel<DT>(V, i, j, k);
        if (d < dmin) dmin = d;
        if (d > dmax) dmax = d;
      }
  if (bx == 0 || by == 0 || bz == 0 || bx == V.gx - 1 || by == V.gy - 1 || bz == V.gz - 1)
    if (0.0f < dmin) dmin = 0.0f;
  out[b] = V.sigma_scale * tf_alpha_max(V, dmin, dmax) * 1.0009765625f;
}

// The same majorant with one block per brick (large bricks): warps take the
// (y, z) rows of the brick plus apron, lanes the voxels along x; min and max
// are combined by comparisons, so the order does not change the result.
template <int DT>
__global__ void __launch_bounds__(256) k_brick_majorants_block(Vol V, float* __restrict__ out) {
  __shared__ float s_min[8], s_max[8];
  const int64_t b = blockIdx.x;
  const int bx = (int)(b % V.gx), by = (int)((b / V.gx) % V.gy), bz = (int)(b / ((int64_t)V.gx * V.gy));
  const int B = V.B;
  const int i0 = max(B * bx - 1, 0), i1 = min(B * bx + B, V.nx - 1);
  const int j0 = max(B * by - 1, 0), j1 = min(B * by + B, V.ny - 1);
  const int k0 = max(B * bz - 1, 0), k1 = min(B * bz + B, V.nz - 1);
  const int nj = j1 - j0 + 1, rows = nj * (k1 - k0 + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float dmin = __int_as_float(0x7f800000), dmax = -dmin;
  for (int r = warp; r < rows; r += nw) {
    const int j = j0 + r % nj, k = k0 + r / nj;
    for (int i = i0 + lane; i <= i1; i += 32) {
      const float d = voxel<DT>(V, i, j, k);
      if (d < dmin) dmin = d;
      if (d > dmax) dmax = d;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float a = __shfl_xor_sync(0xffffffffu, dmin, off), c = __shfl_xor_sync(0xffffffffu, dmax, off);
    if (a < dmin) dmin = a;
    if (c > dmax) dmax = c;
  }
  if (lane == 0) { s_min[warp] = dmin; s_max[warp] = dmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      if (s_min[w] < dmin) dmin = s_min[w];
      if (s_max[w] > dmax) dmax = s_max[w];
    }
    if (bx == 0 || by == 0 || bz == 0 || bx == V.gx - 1 || by == V.gy - 1 || bz == V.gz - 1)
      if (0.0f < dmin) dmin = 0.0f;
    out[b] = V.sigma_scale * tf_alpha_max(V, dmin, dmax) * 1.0009765625f;
  }
}

}  // namespace

pf_status pf_brick_majorants_impl(pf_ctx* ctx, const pf_volume* vol, float* out) {
  Vol V = pf_make_vol(vol, 0.f, nullptr);
  const int64_t nb = (int64_t)V.gx * V.gy * V.gz;
  if (V.B >= 64) {   // (B + 2)^3 voxels per brick: a block each (measured faster from B = 64)
    const unsigned grd = (unsigned)nb;
    if (vol->dtype == PF_F32) k_brick_majorants_block<0><<<grd, 256, 0, ctx->stream>>>(V, out);
    else if (vol->dtype == PF_F16) k_brick_majorants_block<1><<<grd, 256, 0, ctx->stream>>>(V, out);
    else k_brick_majorants_block<2><<<grd, 256, 0, ctx->stream>>>(V, out);
  } else {
    const unsigned grd = (unsigned)((nb + 127) / 128);
    if (vol->dtype == PF_F32) k_brick_majorants<0><<<grd, 128, 0, ctx->stream>>>(V, out);
    else if (vol->dtype == PF_F16) k_brick_majorants<1><<<grd, 128, 0, ctx->stream>>>(V, out);
    else k_brick_majorants<2><<<grd, 128, 0, ctx->stream>>>(V, out);
  }
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

pf_status pf_grid_for(pf_ctx* ctx, const pf_volume* vol, const float** grid) {
  if (vol->brick_majorants_dev) { *grid = vol->brick_majorants_dev; return PF_OK; }
  const int B = vol->brick > 0 ? vol->brick : 8;
  const int64_t nb = (int64_t)((vol->nx + B - 1) / B) * ((vol->ny + B - 1) / B) * ((vol->nz + B - 1) / B);
  float* g;
  PF_TRY(pf_scratch(ctx, WS_GRID, (size_t)nb * sizeof(float), (void**)&g));
  PF_TRY(pf_brick_majorants_impl(ctx, vol, g));
  *grid = g;
  return PF_OK;
}

namespace {
__global__ void k_border_grid(const float* __restrict__ g, int gx, int gy, int gz, int64_t n, float* __restrict__ out) {
  const int px = gx + 2 * kBorder, py = gy + 2 * kBorder;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % px) - kBorder, j = (int)((e / px) % py) - kBorder, k = (int)(e / ((int64_t)px * py)) - kBorder;
    const bool in = i >= 0 && i < gx && j >= 0 && j < gy && k >= 0 && k < gz;
    out[e] = in ? __ldg(g + (int64_t)i + (int64_t)gx * ((int64_t)j + (int64_t)gy * k)) : 0.0f;
  }
}
}  // namespace

pf_status pf_bordered_grid(pf_ctx* ctx, const float* grid, int gx, int gy, int gz, int slot, const float** out) {
  const int64_t n = (int64_t)(gx + 2 * kBorder) * (gy + 2 * kBorder) * (gz + 2 * kBorder);
  if (n >= (1ll << 31)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "brick grid too large for the walks (2^31 bricks)");
  float* b;
  PF_TRY(pf_scratch(ctx, slot, (size_t)n * sizeof(float), (void**)&b));
  k_border_grid<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
      grid, gx, gy, gz, n, b);
  PF_CUDA(ctx, cudaGetLastError());
  *out = b;
  return PF_OK;
}

namespace {
// Tiled copy: one thread per destination element (tile-major, 64 per tile).
template <typename T>
__global__ void k_tile_volume(const T* __restrict__ src, int nx, int ny, int nz, int tnx, int tny, int64_t n,
                              T* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t tile = e >> 6;
  const int w = (int)(e & 63);
  const int i = (int)(tile % tnx) * 4 + (w & 3);
  const int j = (int)((tile / tnx) % tny) * 4 + ((w >> 2) & 3);
  const int k = (int)(tile / ((int64_t)tnx * tny)) * 4 + (w >> 4);
  dst[e] = (i < nx && j < ny && k < nz) ? src[(size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k)] : T(0);
}
}  // namespace

extern "C" pf_status pf_volume_tile(pf_ctx* ctx, const pf_volume* vol, void* out_dev) {
  if (!ctx || !out_dev) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, vol));
  const int tnx = (vol->nx + 3) / 4, tny = (vol->ny + 3) / 4, tnz = (vol->nz + 3) / 4;
  const int64_t n = (int64_t)tnx * tny * tnz * 64;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (vol->dtype == PF_F32)
    k_tile_volume<float><<<grid, 256, 0, ctx->stream>>>((const float*)vol->data_dev, vol->nx, vol->ny, vol->nz, tnx,
                                                         tny, n, (float*)out_dev);
  else if (vol->dtype == PF_F16)
    k_tile_volume<uint16_t><<<grid, 256, 0, ctx->stream>>>((const uint16_t*)vol->data_dev, vol->nx, vol->ny, vol->nz,
                                                            tnx, tny, n, (uint16_t*)out_dev);
  else
    k_tile_volume<uint8_t><<<grid, 256, 0, ctx->stream>>>((const uint8_t*)vol->data_dev, vol->nx, vol->ny, vol->nz,
                                                           tnx, tny, n, (uint8_t*)out_dev);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

extern "C" pf_status pf_volume_brick_majorants(pf_ctx* ctx, const pf_volume* vol, float* out_dev) {
  if (!ctx || !out_dev) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, vol));
  return pf_brick_majorants_impl(ctx, vol, out_dev);
}

static void free_cache(pf_cache* c) {
  if (!c) return;
  cudaFree(c->counts); cudaFree(c->offsets); cudaFree(c->recs); cudaFree(c->pos); cudaFree(c->flux);
  cudaFree(c->occupied); cudaFree(c->cell_sigma);
  delete c;
}

extern "C" pf_status pf_build_photon_cache(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights,
                                           const float* g_set, int n_g, uint64_t N, int max_bounces, int res,
                                           uint64_t seed, int use_rr, pf_cache** out) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (!out) return pf_fail(ctx, PF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  PF_TRY(pf_check_volume(ctx, vol));
  PF_TRY(pf_check_lights(ctx, lights, n_lights));
  if (!g_set || n_g < 1 || n_g > 16) return pf_fail(ctx, PF_ERR_INVALID_ARG, "n_g must be in [1, 16]");
  for (int i = 0; i < n_g; ++i)
    if (!(g_set[i] > -1.f && g_set[i] < 1.f)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "g values must lie in (-1, 1)");
  if (max_bounces < 2 || max_bounces > 16) return pf_fail(ctx, PF_ERR_INVALID_ARG, "max_bounces must be in [2, 16]");
  if (res < 1 || res > 256 || (res & (res - 1))) return pf_fail(ctx, PF_ERR_INVALID_ARG, "cache_res must be a power of two in [1, 256]");
  uint64_t P = (uint64_t)n_lights * (uint64_t)n_g * N;
  if (N == 0 || P >= (1ull << 28)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "total photon count must be in [1, 2^28)");
  int64_t nc = (int64_t)res * res * res;
  int64_t n_keys = (int64_t)n_lights * n_g * nc;
  if (n_keys >= (1ll << 32)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "too many cache keys");
  const float* grid;
  PF_TRY(pf_grid_for(ctx, vol, &grid));

  pf_cache* c = new pf_cache();
  c->ctx = ctx; c->device = ctx->device; c->res = res; c->n_lights = n_lights; c->n_g = n_g; c->max_bounces = max_bounces;
  c->n_photons = (int64_t)P; c->n_keys = n_keys;
  for (int i = 0; i < n_g; ++i) c->g_set[i] = g_set[i];
  int S = max_bounces - 1;
  auto fail = [&](pf_status s) { free_cache(c); return s; };
  float4* slots = nullptr;
  float4* slot_pos = nullptr;
  uint8_t* nrec = nullptr;
  uint32_t* cursor = nullptr;
  double* tally_dev = nullptr;
  // the temporaries live in the context's scratch arena (reused by the next
  // build); the cache's own arrays are allocated for it
#define CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return fail(pf_cuda_check(ctx, e_, #call)); } while (0)
#define ST(call) do { pf_status s_ = (call); if (s_ != PF_OK) return fail(s_); } while (0)
  ST(pf_scratch(ctx, WS_TRACE_SLOTS, (size_t)P * S * 2 * sizeof(float4), (void**)&slots));
  ST(pf_scratch(ctx, WS_TRACE_POS, (size_t)P * S * sizeof(float4), (void**)&slot_pos));
  ST(pf_scratch(ctx, WS_TRACE_NREC, (size_t)P, (void**)&nrec));
  CK(cudaMalloc(&c->counts, (size_t)n_keys * sizeof(uint32_t)));
  ST(pf_scratch(ctx, WS_TRACE_CURSOR, (size_t)std::max<int64_t>(n_keys, nc) * sizeof(uint32_t), (void**)&cursor));
  CK(cudaMalloc(&c->offsets, (size_t)(n_keys + 1) * sizeof(uint64_t)));
  // persistent tracing warps: as many one-warp blocks as fit on the device
  int per_sm = 0;
  if (vol->dtype == PF_F32) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_photons<0>, kTraceThreads, 0));
  else if (vol->dtype == PF_F16) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_photons<1>, kTraceThreads, 0));
  else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_photons<2>, kTraceThreads, 0));
  const int64_t trace_blocks = std::max<int64_t>(
      1, std::min<int64_t>((int64_t)ctx->num_sms * std::max(per_sm, 1), (int64_t)((P + kTraceThreads - 1) / kTraceThreads)));
  // per-block tally rows, the 15 sums, and the photon counter
  ST(pf_scratch(ctx, WS_TRACE_TALLY, (size_t)(trace_blocks + 2) * 15 * sizeof(double), (void**)&tally_dev));
  CK(cudaMemsetAsync(c->counts, 0, (size_t)n_keys * sizeof(uint32_t), ctx->stream));


  StageTimer tm(ctx, PF_STAGE_PHOTONS);
  TraceArgs A;
  A.V = pf_make_vol(vol, 0.f, grid);
  ST(pf_bordered_grid(ctx, grid, A.V.gx, A.V.gy, A.V.gz, WS_GRID_WALK, &A.V.mgw));
  A.L = pf_make_lights(lights, n_lights);
  for (int i = 0; i < 16; ++i) A.g_set[i] = i < n_g ? g_set[i] : 0.f;
  A.n_g = n_g; A.max_bounces = max_bounces; A.res = res; A.use_rr = use_rr; A.N = N; A.seed = seed; A.n_photons = P;
  const unsigned grd = (unsigned)trace_blocks;
  double* tally_sum = tally_dev + (size_t)trace_blocks * 15;
  unsigned long long* next = (unsigned long long*)(tally_sum + 15);
  CK(cudaMemsetAsync(next, 0, sizeof(unsigned long long), ctx->stream));
  if (vol->dtype == PF_F32)
    k_trace_photons<0><<<grd, kTraceThreads, 0, ctx->stream>>>(A, slots, slot_pos, nrec, c->counts, next, tally_dev,
                                                                ctx->err_dev);
  else if (vol->dtype == PF_F16)
    k_trace_photons<1><<<grd, kTraceThreads, 0, ctx->stream>>>(A, slots, slot_pos, nrec, c->counts, next, tally_dev,
                                                                ctx->err_dev);
  else
    k_trace_photons<2><<<grd, kTraceThreads, 0, ctx->stream>>>(A, slots, slot_pos, nrec, c->counts, next, tally_dev,
                                                                ctx->err_dev);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(tally_sum, 0, 15 * sizeof(double), ctx->stream));
  k_tally_reduce<<<(unsigned)std::min<int64_t>((trace_blocks * 15 + kTallyThreads - 1) / kTallyThreads,
                                               (int64_t)ctx->num_sms * 8),
                   kTallyThreads, 0, ctx->stream>>>(tally_dev, trace_blocks, tally_sum);
  CK(cudaGetLastError());
  ST(pf_scan_u32(ctx, c->counts, c->offsets, n_keys));
  uint64_t n_rec = 0;
  CK(cudaMemcpyAsync(&n_rec, c->offsets + n_keys, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(c->tally, tally_sum, 15 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  c->n_records = (int64_t)n_rec;
  CK(cudaMalloc(&c->recs, (size_t)std::max<uint64_t>(n_rec, 1) * 2 * sizeof(float4)));
  CK(cudaMalloc(&c->pos, (size_t)std::max<uint64_t>(n_rec, 1) * sizeof(float4)));
  CK(cudaMemsetAsync(cursor, 0, (size_t)n_keys * sizeof(uint32_t), ctx->stream));
  uint64_t n_slots = P * (uint64_t)S;
  k_scatter<<<(unsigned)((n_slots + 255) / 256), 256, 0, ctx->stream>>>(slots, slot_pos, nrec, P, S, c->offsets, cursor,
                                                                        c->recs, c->pos);
  CK(cudaGetLastError());
  CK(cudaMalloc(&c->flux, (size_t)n_keys * 3 * sizeof(float)));
  k_key_flux<<<(unsigned)((n_keys + 255) / 256), 256, 0, ctx->stream>>>(c->recs, c->offsets, n_keys, c->flux);
  CK(cudaGetLastError());
  CK(cudaMalloc(&c->cell_sigma, (size_t)nc * sizeof(float)));
  unsigned gc = (unsigned)((nc + 127) / 128);
  if (vol->dtype == PF_F32) k_cell_sigma<0><<<gc, 128, 0, ctx->stream>>>(A.V, res, c->cell_sigma);
  else if (vol->dtype == PF_F16) k_cell_sigma<1><<<gc, 128, 0, ctx->stream>>>(A.V, res, c->cell_sigma);
  else k_cell_sigma<2><<<gc, 128, 0, ctx->stream>>>(A.V, res, c->cell_sigma);
  CK(cudaGetLastError());
  // occupancy flags reuse `cursor`; their exclusive scan gets its own buffer
  uint64_t* opos = nullptr;
  ST(pf_scratch(ctx, WS_TRACE_OPOS, (size_t)(nc + 1) * sizeof(uint64_t), (void**)&opos));
  k_occupancy<<<gc, 128, 0, ctx->stream>>>(c->counts, c->cell_sigma, nc, n_lights * n_g, cursor);
  CK(cudaGetLastError());
  ST(pf_scan_u32(ctx, cursor, opos, nc));
  uint64_t n_occ = 0;
  CK(cudaMemcpyAsync(&n_occ, opos + nc, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  c->n_occupied = (int64_t)n_occ;
  CK(cudaMalloc(&c->occupied, (size_t)std::max<uint64_t>(n_occ, 1) * sizeof(uint32_t)));
  k_occupied_list<<<gc, 128, 0, ctx->stream>>>(cursor, opos, nc, c->occupied);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
#undef CK
#undef ST
  pf_status es = pf_check_error_word(ctx);
  if (es != PF_OK) { free_cache(c); return es; }
  *out = c;
  return PF_OK;
}

extern "C" pf_status pf_cache_info(pf_ctx* ctx, const pf_cache* c, pf_cache_info_t* out) {
  if (!ctx || !c || !out) return PF_ERR_INVALID_ARG;
  out->n_photons = c->n_photons; out->n_records = c->n_records; out->n_keys = c->n_keys;
  out->n_occupied = c->n_occupied; out->res = c->res; out->n_lights = c->n_lights; out->n_g = c->n_g;
  out->max_bounces = c->max_bounces;
  for (int i = 0; i < 15; ++i) out->tally[i] = c->tally[i];
  return PF_OK;
}

namespace {
__global__ void k_export_recs(const float4* __restrict__ recs, const float4* __restrict__ rpos, int64_t n, uint32_t* key,
                              uint32_t* id, float* dir, float* phi, float* pos) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = recs[2 * i], b = recs[2 * i + 1];
  if (pos) { float4 x = rpos[i]; pos[3 * i] = x.x; pos[3 * i + 1] = x.y; pos[3 * i + 2] = x.z; }
  if (key) key[i] = __float_as_uint(a.x);
  if (id) id[i] = __float_as_uint(a.y);
  if (dir) { dir[3 * i] = a.z; dir[3 * i + 1] = a.w; dir[3 * i + 2] = b.x; }
  if (phi) { phi[3 * i] = b.y; phi[3 * i + 1] = b.z; phi[3 * i + 2] = b.w; }
}
}  // namespace

extern "C" pf_status pf_cache_export(pf_ctx* ctx, const pf_cache* c, uint32_t* counts_dev, float* flux_dev,
                                     uint32_t* rec_key_dev, uint32_t* rec_id_dev, float* rec_dir_dev,
                                     float* rec_phi_dev, float* rec_pos_dev, uint32_t* occupied_dev,
                                     float* cell_sigma_dev) {
  if (!ctx || !c) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = ctx->stream;
  if (counts_dev) PF_CUDA(ctx, cudaMemcpyAsync(counts_dev, c->counts, c->n_keys * 4, cudaMemcpyDeviceToDevice, s));
  if (flux_dev) PF_CUDA(ctx, cudaMemcpyAsync(flux_dev, c->flux, c->n_keys * 12, cudaMemcpyDeviceToDevice, s));
  if (occupied_dev && c->n_occupied)
    PF_CUDA(ctx, cudaMemcpyAsync(occupied_dev, c->occupied, c->n_occupied * 4, cudaMemcpyDeviceToDevice, s));
  if (cell_sigma_dev)
    PF_CUDA(ctx, cudaMemcpyAsync(cell_sigma_dev, c->cell_sigma, (size_t)c->res * c->res * c->res * 4, cudaMemcpyDeviceToDevice, s));
  if ((rec_key_dev || rec_id_dev || rec_dir_dev || rec_phi_dev || rec_pos_dev) && c->n_records) {
    k_export_recs<<<(unsigned)((c->n_records + 255) / 256), 256, 0, s>>>(c->recs, c->pos, c->n_records, rec_key_dev,
                                                                           rec_id_dev, rec_dir_dev, rec_phi_dev,
                                                                           rec_pos_dev);
    PF_CUDA(ctx, cudaGetLastError());
  }
  return PF_OK;
}

extern "C" pf_status pf_cache_free(pf_cache* c) {
  if (!c) return PF_OK;
  DeviceGuard dg(c->device);
  cudaDeviceSynchronize();
  free_cache(c);
  return PF_OK;
}
