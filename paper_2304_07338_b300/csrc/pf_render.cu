// Neural volumetric path tracing (Algorithm 2) and the plain path tracer.
//
// Wavefront organisation on B300:
//   k_camera_samples  one thread per (pixel, sample): RayGeneration and free
//                     flight (VolumeSampling); appends the samples that
//                     scatter to a compacted list (one atomic per warp) with
//                     their field query, direction and albedo.  In marching
//                     mode it also does the next-event estimation itself;
//   k_place           (tracking mode) orders the compacted list by a 64^3
//                     Morton cell of the scattering position (counting sort:
//                     histogram in k_camera_samples, scan, placement);
//   k_nee             (tracking mode) DirectIllumination over the ordered
//                     list: one thread per scattering sample traces its
//                     ratio-tracked shadow rays, so the ~90% of samples that
//                     leave the volume do not hold idle lanes while the
//                     others trace eight shadow rays each, and the lanes of
//                     a warp start from nearby points: towards one light
//                     their rays cross the same bricks in step;
//   field forward     over the compacted list only (the paper's compaction
//                     of the sample buffer), decode, times albedo, written
//                     back to the sample's slot;
//   k_compose         one thread per pixel, sums its samples in order.
// The path tracer uses the same slot layout and an in-order per-pixel sum,
// processed in chunks of samples so that any spp fits in bounded scratch.
//
// Compiled with -fmad=false: see pf_device.cuh.
#include "pf_internal.h"
#include "pf_device.cuh"
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>
#include <algorithm>

using namespace pfd;

namespace {

// Morton index of the 64^3 cell holding x (positions in [0,1]^3).
constexpr int kCellBits = 6;
constexpr uint32_t kCells = 1u << (3 * kCellBits);
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t morton_cell(V3 x) {
  const float s = (float)(1 << kCellBits);
  const uint32_t cx = (uint32_t)min(max((int)(x.x * s), 0), (1 << kCellBits) - 1);
  const uint32_t cy = (uint32_t)min(max((int)(x.y * s), 0), (1 << kCellBits) - 1);
  const uint32_t cz = (uint32_t)min(max((int)(x.z * s), 0), (1 << kCellBits) - 1);
  return spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
}

// Coarser majorant grid: each cell the largest majorant of its f x f x f
// group of bricks (exact; it bounds sigma_t over the group).
__global__ void k_pool_majorants(const float* __restrict__ fine, int gx, int gy, int gz, int f, int px, int py,
                                 int pz, float* __restrict__ coarse) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (int64_t)px * py * pz) return;
  const int I = (int)(c % px), J = (int)((c / px) % py), K = (int)(c / ((int64_t)px * py));
  float m = 0.0f;
  for (int k = K * f; k < min(K * f + f, gz); ++k)
    for (int j = J * f; j < min(J * f + f, gy); ++j)
      for (int i = I * f; i < min(I * f + f, gx); ++i) m = fmaxf(m, fine[i + (int64_t)gx * (j + (int64_t)gy * k)]);
  coarse[c] = m;
}

// Counting-sort placement: entry i goes to off[key] + (its rank among the
// entries of that key, in atomic order).
__global__ void k_place(const uint32_t* __restrict__ ckey, const uint32_t* __restrict__ ccount,
                        const uint64_t* __restrict__ off, uint32_t* __restrict__ fill, uint32_t* __restrict__ perm) {
  const uint32_t n = *ccount;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = ckey[i];
    perm[off[k] + atomicAdd(fill + k, 1u)] = i;
  }
}

// Segments of the ray marcher whose density lookups are issued together.
constexpr int kMarchAhead = 4;

// -------------------------------------------------------------- camera samples
// Sample k of pixel pix = (px, py) for slot = pix * spp + k, in 32-bit
// arithmetic when every slot index fits (the same quotients as in 64 bits).
__device__ __forceinline__ void slot_pixel(int64_t slot, int64_t n_slots, int spp, int W, int* k, int64_t* pix,
                                           int* px, int* py) {
  if (n_slots <= (int64_t)0xffffffffll) {
    const uint32_t s = (uint32_t)slot, sp = (uint32_t)spp, w = (uint32_t)W;
    const uint32_t p = s / sp, y = p / w;
    *k = (int)(s - p * sp);
    *pix = (int64_t)p;
    *py = (int)y;
    *px = (int)(p - y * w);
  } else {
    *k = (int)(slot % spp);
    *pix = slot / spp;
    *px = (int)(*pix % W);
    *py = (int)(*pix / W);
  }
}

// stats (nullable): stats[0] += density lookups, stats[1] += valid samples
// (= field queries) of the launch.
template <int DT, bool MARCH>
__device__ __forceinline__ void camera_samples(Vol V, DevLights L, CamF cam, float g, int spp, float h,
                                               uint64_t seed, int64_t n_slots, float* __restrict__ slot_ld,
                                               float* __restrict__ slot_li, float* __restrict__ cq,
                                               float* __restrict__ calb, float* __restrict__ cdir,
                                               uint32_t* __restrict__ cidx, uint32_t* __restrict__ ccount,
                                               uint32_t* __restrict__ ckey, uint32_t* __restrict__ chist,
                                               uint32_t* __restrict__ vmask, uint32_t* err,
                                               unsigned long long* stats) {
  int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = slot < n_slots;
  uint32_t nfetch = 0;
  int valid = 0;
  V3 x = v3(0.f, 0.f, 0.f), wo = x, alb = x, Ld = x;
  if (active) {
    int k, px, py;
    int64_t pix;
    slot_pixel(slot, n_slots, spp, cam.W, &k, &pix, &px, &py);
    Rng rng(seed, TAG_CAMERA, (uint64_t)pix, (uint32_t)k);
    float b0[4]; rng.uni4(b0);
    V3 o, d;
    camera_ray(cam, px, py, b0[0], b0[1], &o, &d);
    wo = v3(-d.x, -d.y, -d.z);
    float t0, t1;
    if (box_hit(o, d, &t0, &t1)) {
      float th = 0.f;
      bool hit = false;
      float jl[16];
      if (MARCH) {
        for (int b = 0; b < (L.n + 3) / 4; ++b) {
          float w[4]; rng.uni4(w);
#pragma unroll
          for (int i = 0; i < 4; ++i) if (4 * b + i < 16) jl[4 * b + i] = w[i];
        }
        // Target optical depth tau* = -ln(1-u).  The interaction point is
        // s0 + (tau* - tau)/sigma: where sigma is small, one float32 ulp of
        // tau* or tau moves it by ulp/sigma, so tau* (one log per sample) and
        // that final remainder are evaluated in FP64; the march itself and
        // its compensated (Kahan) optical-depth sum stay float32.
        const double tau_star_d = -log1p(-(double)b0[3]);
        const float tau_star = (float)tau_star_d;
        float tau = 0.f, comp = 0.f;
        const int nseg = (int)ceilf((t1 - t0) / h);
        // kMarchAhead segments' lookups are issued together (independent
        // loads in flight), then taken in order by the same float steps as a
        // one-at-a-time loop; lookups past the interaction are discarded
        // (a point beyond the ray's box exit reads density 0)
        for (int s = 0; s < nseg && !hit; s += kMarchAhead) {
          float sg[kMarchAhead], s0v[kMarchAhead], lenv[kMarchAhead];
#pragma unroll
          for (int j = 0; j < kMarchAhead; ++j) {
            s0v[j] = t0 + (float)(s + j) * h;
            lenv[j] = mn(t0 + (float)(s + j + 1) * h, t1) - s0v[j];
            sg[j] = sigma_at<DT>(V, along(o, d, s0v[j] + b0[2] * lenv[j]));
          }
#pragma unroll
          for (int j = 0; j < kMarchAhead; ++j) {
            if (s + j >= nseg || hit) break;
            const float len = lenv[j];
            if (!(len > 0.f)) continue;
            ++nfetch;
            const float dtau = sg[j] * len;
            if (sg[j] > 0.f && (tau - comp) + dtau >= tau_star) {
              const double rem = tau_star_d - ((double)tau - (double)comp);
              const float dl = (float)(rem / (double)sg[j]);
              th = s0v[j] + mn(mx(dl, 0.f), len);
              hit = true;
              break;
            }
            const float y = dtau - comp;
            const float t = tau + y;
            comp = (t - tau) - y;
            tau = t;
          }
        }
      } else {
        hit = delta_track<DT>(V, o, d, t0, t1, rng, &th, err, nfetch);
      }
      if (hit) {
        x = along(o, d, th);
        float sig;
        medium_at<DT>(V, x, &sig, &alb);
        ++nfetch;
        for (int l = 0; MARCH && l < L.n; ++l) {
          V3 wl, E; float dist;
          light_geom(L.l[l], x, &wl, &dist, &E);
          float a0, a1, tend = 0.f;
          if (box_hit(x, wl, &a0, &a1)) tend = mn(a1, dist);
          float T;
          {
            float tau = 0.f, comp = 0.f;
            if (tend > 0.f) {
              const int nseg = (int)ceilf(tend / h);
              for (int s = 0; s < nseg; s += kMarchAhead) {   // lookups ahead, sums in order
                float sg[kMarchAhead], lenv[kMarchAhead];
#pragma unroll
                for (int j = 0; j < kMarchAhead; ++j) {
                  const float s0 = (float)(s + j) * h;
                  lenv[j] = mn((float)(s + j + 1) * h, tend) - s0;
                  sg[j] = sigma_at<DT>(V, along(x, wl, s0 + jl[l] * lenv[j]));
                }
#pragma unroll
                for (int j = 0; j < kMarchAhead; ++j) {
                  if (s + j >= nseg) break;
                  if (!(lenv[j] > 0.f)) continue;
                  const float y = sg[j] * lenv[j] - comp;
                  ++nfetch;
                  const float t = tau + y;
                  comp = (t - tau) - y;
                  tau = t;
                }
              }
            }
            T = expf(-(tau - comp));
          }
          float ph = hg_eval(g, dot(d, wl));
          Ld = v3(Ld.x + ph * T * E.x, Ld.y + ph * T * E.y, Ld.z + ph * T * E.z);
        }
        valid = 1;
      }
    }
    if (MARCH && valid) {  // tracking mode: k_nee writes L_d of the valid slots
      slot_ld[3 * slot + 0] = alb.x * Ld.x;
      slot_ld[3 * slot + 1] = alb.y * Ld.y;
      slot_ld[3 * slot + 2] = alb.z * Ld.z;
    }
  }
  // one validity bit per slot (the warp's 32 slots are one aligned word);
  // compose reads only the valid slots, so no slot is zero-filled
  const unsigned ball = __ballot_sync(0xffffffffu, valid);
  if ((threadIdx.x & 31) == 0 && slot < n_slots) vmask[slot >> 5] = ball;
  if (stats) {
    unsigned long long v = nfetch;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    unsigned nv = __popc(__ballot_sync(0xffffffffu, valid));
    if ((threadIdx.x & 31) == 0) {
      if (v) atomicAdd(stats, v);
      if (nv) atomicAdd(stats + 1, (unsigned long long)nv);
    }
  }
  if (cq == nullptr) return;
  // warp-aggregated append of the valid samples' queries
  if (ball == 0) return;
  int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(ccount, (uint32_t)__popc(ball));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (valid) {
    uint32_t i = base + __popc(ball & ((1u << lane) - 1u));
    float th, ph;
    query_angles(wo.x, wo.y, wo.z, &th, &ph);
    cq[6 * (size_t)i + 0] = x.x; cq[6 * (size_t)i + 1] = x.y; cq[6 * (size_t)i + 2] = x.z;
    cq[6 * (size_t)i + 3] = th;  cq[6 * (size_t)i + 4] = ph;  cq[6 * (size_t)i + 5] = g;
    calb[3 * (size_t)i + 0] = alb.x; calb[3 * (size_t)i + 1] = alb.y; calb[3 * (size_t)i + 2] = alb.z;
    if (!MARCH) {
      cdir[3 * (size_t)i + 0] = -wo.x; cdir[3 * (size_t)i + 1] = -wo.y; cdir[3 * (size_t)i + 2] = -wo.z;
      const uint32_t key = morton_cell(x);
      ckey[i] = key;
      atomicAdd(chist + key, 1u);
    }
    cidx[i] = (uint32_t)slot;
  }
}

// The two modes as separate kernels: the tracking body is lean and gains from
// 8 resident blocks per SM (64 registers), the marched body (shadow rays
// marched in the same kernel) needs its registers.
#define PF_CAMERA_ARGS                                                                                              \
  Vol V, DevLights L, CamF cam, float g, int spp, float h, uint64_t seed, int64_t n_slots, float* __restrict__ slot_ld, \
      float* __restrict__ slot_li, float* __restrict__ cq, float* __restrict__ calb, float* __restrict__ cdir,       \
      uint32_t* __restrict__ cidx, uint32_t* __restrict__ ccount, uint32_t* __restrict__ ckey,                      \
      uint32_t* __restrict__ chist, uint32_t* __restrict__ vmask, uint32_t* err, unsigned long long* stats
#define PF_CAMERA_PASS \
  V, L, cam, g, spp, h, seed, n_slots, slot_ld, slot_li, cq, calb, cdir, cidx, ccount, ckey, chist, vmask, err, stats
template <int DT>
__global__ void __launch_bounds__(128, 8) k_camera_samples(PF_CAMERA_ARGS) { camera_samples<DT, false>(PF_CAMERA_PASS); }
template <int DT>
__global__ void __launch_bounds__(128, 5) k_camera_samples_march(PF_CAMERA_ARGS) {
  camera_samples<DT, true>(PF_CAMERA_PASS);
}
#undef PF_CAMERA_ARGS
#undef PF_CAMERA_PASS

// Majorant of the brick of V holding x, its index clamped into brick `widx`
// of the coarser grid Vw (so that it never exceeds Vw's majorant there);
// widx indexes Vw's bordered copy (the walk's), and names a brick inside the
// grid (a tentative collision never lies in a border brick).
__device__ __forceinline__ float thin_majorant(const Vol& V, const Vol& Vw, int widx, V3 x) {
  const int f = Vw.B / V.B;
  const int wx = widx % Vw.pgx - kBorder, wy = (widx / Vw.pgx) % Vw.pgy - kBorder,
            wz = widx / (Vw.pgx * Vw.pgy) - kBorder;
  const int cx = min(max((int)floorf(x.x / V.wx), wx * f), min(wx * f + f, V.gx) - 1);
  const int cy = min(max((int)floorf(x.y / V.wy), wy * f), min(wy * f + f, V.gy) - 1);
  const int cz = min(max((int)floorf(x.z / V.wz), wz * f), min(wz * f + f, V.gz) - 1);
  return __ldg(V.mg + (cx + V.gx * (cy + V.gy * cz)));
}

// Next-event estimation of the scattering samples (tracking mode): one shadow
// ray per (light, scattering sample), ratio tracked on the ray's own stream;
// k_nee_sum then forms L_d = sum over lights, in order, of p(d . w_l) T_l E_l
// and slot_ld[slot] = albedo * L_d.  stats[0] and stats[2] += its lookups.
//
// Work items are the shadow rays, in windows of kNeeWindow cell-sorted
// samples and light-major inside a window, so a warp's rays share a light and
// start close together, and a window's voxels serve all lights while they are
// in L2.  Warps are persistent and refill: a lane whose ray is done takes
// the next item from a global counter (one atomic per warp and pass), so a
// warp no longer idles while its longest ray finishes.
//
// Ratio tracking's tentative collisions do not depend on the density, only
// the weights 1 - sigma_t/majorant do.  A warp therefore traces its rays in
// passes: each lane walks its ray, recording up to kNeePool collisions
// (distance, majorant) in the warp's shared-memory pool; then all 32 lanes
// evaluate the pooled density lookups together, whatever ray they belong to;
// then each lane multiplies its own factors in collision order.  The floats
// are those of a walk with the lookups inline (same operations, same order per
// ray); only the lane doing each lookup changes, so the lanes stay busy while
// the rays' collision counts differ.  The pool lives in shared memory, which
// the SM carves out of the same storage as the L1 cache that serves the
// density gathers; it is kept small.
constexpr int kNeePool = 8;                                                // collisions per lane per pass (the budget ring bounds them too)
constexpr int kNeeTau = 8;                                                 // buffered budgets per lane (ring)
constexpr int kNeeWarpFloats =
    32 * kNeePool * 2 + 32 * kNeePool / 2 + 32 * 6 + 32 * kNeeTau;  // t/factor, majorant, u16 map; x, w_l; budgets
constexpr int kNeeWarps = 4;
constexpr uint64_t kNeeWindow = 4096;   // sorted samples whose shadow rays (all lights) run together

// THIN: the rays walk Vw (the brick grid max-pooled by f = Vw.B / V.B) and a
// tentative collision of that walk at x is kept with probability
// m_V(x) / m_Vw (one more uniform after its budget), m_V(x) the majorant of
// the brick of V holding x, clamped into the current brick of Vw: the kept
// collisions are those of ratio tracking over V's bricks.
// contrib [n_lights][n][2]: (p(d . w_l) T_l, |p_l - x|^2) of sorted sample j for
// light l; k_nee_sum forms E_l from the second (point lights) and multiplies.
template <int DT, bool THIN>
__global__ void __launch_bounds__(128, 8) k_nee(Vol V, Vol Vw, DevLights L, float g, int spp, uint64_t seed,
                                             const float* __restrict__ cq, const float* __restrict__ cdir,
                                             const uint32_t* __restrict__ cidx, const uint32_t* __restrict__ ccount,
                                             const uint32_t* __restrict__ perm, unsigned long long* __restrict__ next,
                                             float* __restrict__ contrib, uint32_t* err, unsigned long long* stats) {
  extern __shared__ float pf_nee_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* pool = pf_nee_smem + warp * kNeeWarpFloats;
  float* pt = pool;                                        // collision distance, then its factor
  float* pm = pool + 32 * kNeePool;                        // majorant at the collision
  uint16_t* pmap = (uint16_t*)(pool + 64 * kNeePool);      // pooled entry -> lane * kNeePool + index
  float* pxw = pool + 64 * kNeePool + 16 * kNeePool;       // per lane: origin x (3), direction w_l (3)
  float* ptau = pxw + 32 * 6 + lane * kNeeTau;             // this lane's ring of budgets -ln(1 - u)
  const uint64_t n = *ccount;
  const uint64_t n_items = n * (uint64_t)L.n;
  uint32_t nfetch = 0;
  // the lane's shadow ray
  bool has = false, done = true;
  uint64_t item = 0;
  V3 x = v3(0.5f, 0.5f, 0.5f), wl = v3(0.f, 0.f, 1.f), E = v3(0.f, 0.f, 0.f);
  float ph = 0.f, T = 1.0f, t = 0.0f, tau = 0.0f, tc = 0.0f, tend = 0.0f, d2l = 0.0f;
  int it = 0;
  Walk<true> W;
  Uniforms U;                   // THIN: uniforms drawn in the walk
  int un = 0, ur = 0;           // !THIN: budgets buffered in ptau, read position
  bool need_tau = false;        // !THIN: the next budget is still to be taken
  Rng rs(0, 0, 0, 0);
  for (;;) {
    // refill: lanes whose ray is done take the next items
    const unsigned need = __ballot_sync(0xffffffffu, !has);
    bool exhausted = false;
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      exhausted = base + (unsigned long long)__popc(need) >= n_items;
      if (!has) {
        const uint64_t q = base + (uint64_t)__popc(need & ((1u << lane) - 1u));
        if (q < n_items) {
          has = true;
          // windows of kNeeWindow sorted samples, light-major inside a window:
          // the rays of all lights of a window run while its voxels are in L2
          const uint64_t per_w = (uint64_t)kNeeWindow * (uint64_t)L.n;
          const uint64_t full = n / kNeeWindow;
          uint64_t j;
          int l;
          if (n_items <= 0xffffffffull) {  // the same split in 32-bit arithmetic
            const uint32_t q32 = (uint32_t)q, pw = (uint32_t)per_w, f32 = (uint32_t)full;
            if (q32 < f32 * pw) {
              const uint32_t w = q32 / pw, r = q32 - w * pw;
              l = (int)(r / (uint32_t)kNeeWindow);
              j = (uint64_t)w * kNeeWindow + r % (uint32_t)kNeeWindow;
            } else {
              const uint32_t r = q32 - f32 * pw, rem = (uint32_t)(n - full * kNeeWindow);
              const uint32_t lq = r / rem;
              l = (int)lq;
              j = full * kNeeWindow + (r - lq * rem);
            }
          } else if (q < full * per_w) {
            const uint64_t r = q % per_w;
            l = (int)(r / kNeeWindow);
            j = (q / per_w) * kNeeWindow + r % kNeeWindow;
          } else {
            const uint64_t r = q - full * per_w, rem = n - full * kNeeWindow;
            l = (int)(r / rem);
            j = full * kNeeWindow + r % rem;
          }
          item = (uint64_t)l * n + j;                    // contrib index (light-major)
          const uint32_t i = perm[j];
          x = v3(cq[6 * (size_t)i + 0], cq[6 * (size_t)i + 1], cq[6 * (size_t)i + 2]);
          const V3 d = v3(cdir[3 * (size_t)i + 0], cdir[3 * (size_t)i + 1], cdir[3 * (size_t)i + 2]);
          const uint32_t slot = cidx[i];
          const uint64_t pix = slot / (uint32_t)spp;
          const uint32_t k = slot % (uint32_t)spp;
          float dist;
          light_geom(L.l[l], x, &wl, &dist, &E);
          if (L.l[l].kind == 0) d2l = 0.0f;
          else {
            const V3 dv = v3(L.l[l].v[0] - x.x, L.l[l].v[1] - x.y, L.l[l].v[2] - x.z);
            d2l = dot(dv, dv);                             // as light_geom forms it
          }
          float a0, a1;
          tend = 0.f;
          if (box_hit(x, wl, &a0, &a1)) tend = mn(a1, dist);
          ph = hg_eval(g, dot(d, wl));
          rs = Rng(seed, TAG_SHADOW, shadow_item(pix, 1, l), k);
          W.init(THIN ? Vw : V, x, wl, 0.0f);
          U = Uniforms();
          T = 1.0f;
          t = 0.0f;
          if (THIN) tau = -own_lnf(1.0f - U.next(rs));
          else { un = 0; ur = 0; need_tau = true; }   // the first budget comes with the pass's draws
          tc = mn(W.exit_t(), tend);
          done = false;
          it = 0;
          pxw[6 * lane + 0] = x.x; pxw[6 * lane + 1] = x.y; pxw[6 * lane + 2] = x.z;
          pxw[6 * lane + 3] = wl.x; pxw[6 * lane + 4] = wl.y; pxw[6 * lane + 5] = wl.z;
        }
      }
    }
    if (!__any_sync(0xffffffffu, has)) {
      if (exhausted) break;
      continue;
    }
    // !THIN: every uniform of a shadow ray is a budget.  The lanes draw the
    // Philox blocks of the budgets this pass may need here, together (two
    // blocks at most, keeping at least five budgets in the ring), instead of
    // one lane at a time inside the divergent walk; the budgets and their
    // order are those of drawing them one by one.  A lane whose ring runs dry
    // within a pass waits for the next one.
    if (!THIN && has && !done) {
#pragma unroll 1
      for (int b = 0; b < 2 && un <= 4; ++b) {
        float u[4];
        rs.uni4(u);
#pragma unroll
        for (int i = 0; i < 4; ++i) ptau[(ur + un + i) & (kNeeTau - 1)] = -own_lnf(1.0f - u[i]);
        un += 4;
      }
      if (need_tau) {
        tau = ptau[ur];
        ur = (ur + 1) & (kNeeTau - 1);
        --un;
        need_tau = false;
      }
    }
    // walk: record up to kNeePool tentative collisions of this lane's ray
    int cnt = 0;
    while (has && !done && !need_tau && cnt < kNeePool) {
      float seg = tc - t;
      if (seg < 0.0f) seg = 0.0f;
      if (tau < W.m * seg) {           // tau >= 0: never true in a brick of majorant 0
        const float m = W.m;
        t = t + tau / m;
        if (THIN) {
          const float ut = U.next(rs);
          const float mf = thin_majorant(V, Vw, W.idx, along(x, wl, t));
          if (ut * m < mf) {
            pt[lane * kNeePool + cnt] = t;
            pm[lane * kNeePool + cnt] = mf;
            ++cnt;
          }
        } else {
          pt[lane * kNeePool + cnt] = t;
          pm[lane * kNeePool + cnt] = m;
          ++cnt;
        }
        if (THIN) {
          tau = -own_lnf(1.0f - U.next(rs));
        } else if (un > 0) {
          tau = ptau[ur];
          ur = (ur + 1) & (kNeeTau - 1);
          --un;
        } else {
          need_tau = true;
        }
      } else {
        tau = tau - W.m * seg;
        t = tc;
        if (t >= tend || !W.step(THIN ? Vw : V)) done = true;
        else tc = mn(W.exit_t(), tend);
      }
      if (++it >= kMaxTrackSteps) { atomicOr(err, 1u); done = true; }
    }
    // pool the warp's collisions
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int c = 0; c < cnt; ++c) pmap[incl - cnt + c] = (uint16_t)(lane * kNeePool + c);
    __syncwarp();
    for (int e = lane; e < total; e += 32) {
      const int si = pmap[e];
      const int o = si / kNeePool;
      const V3 xo = v3(pxw[6 * o + 0], pxw[6 * o + 1], pxw[6 * o + 2]);
      const V3 wo = v3(pxw[6 * o + 3], pxw[6 * o + 4], pxw[6 * o + 5]);
      pt[si] = 1.0f - sigma_at<DT>(V, along(xo, wo, pt[si])) / pm[si];
      ++nfetch;
    }
    __syncwarp();
    for (int c = 0; c < cnt; ++c) T = T * mx(0.0f, pt[lane * kNeePool + c]);
    __syncwarp();
    if (has && done) {
      reinterpret_cast<float2*>(contrib)[item] = make_float2(ph * T, d2l);
      has = false;
    }
  }
  if (stats) {
    unsigned long long v = nfetch;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0 && v) {
      atomicAdd(stats, v);
      atomicAdd(stats + 2, v);
    }
  }
}

// L_d of sorted sample j: the lights' contributions summed in light order;
// slot_ld[slot] = albedo * L_d.
// Per light, E_l = rgb (directional) or rgb / d^2 (point) as light_geom forms
// it, and the term w E_l is rounded before it is added, as when k_nee wrote
// the three products itself.
__global__ void k_nee_sum(const float* __restrict__ contrib, DevLights L, const float* __restrict__ calb,
                          const uint32_t* __restrict__ cidx, const uint32_t* __restrict__ ccount,
                          const uint32_t* __restrict__ perm, float* __restrict__ slot_ld) {
  const uint64_t n = *ccount;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int l = 0; l < L.n; ++l) {
      const float2 c = reinterpret_cast<const float2*>(contrib)[(size_t)l * n + j];
      const DevLight& ll = L.l[l];
      float e0 = ll.rgb[0], e1 = ll.rgb[1], e2 = ll.rgb[2];
      if (ll.kind != 0) { e0 = e0 / c.y; e1 = e1 / c.y; e2 = e2 / c.y; }
      a0 = a0 + c.x * e0; a1 = a1 + c.x * e1; a2 = a2 + c.x * e2;
    }
    const uint32_t i = perm[j];
    const uint32_t slot = cidx[i];
    slot_ld[3 * (size_t)slot + 0] = calb[3 * (size_t)i + 0] * a0;
    slot_ld[3 * (size_t)slot + 1] = calb[3 * (size_t)i + 1] * a1;
    slot_ld[3 * (size_t)slot + 2] = calb[3 * (size_t)i + 2] * a2;
  }
}

// Pixel = (1/spp) sum over its samples, in order, of albedo (L_d + L_i).  A
// sample that did not scatter contributes exactly zero and is skipped (the
// running sums are non-negative, so adding +0 would not change a bit);
// slot_li is NULL when no field was queried.
__global__ void k_compose(const float* __restrict__ slot_ld, const float* __restrict__ slot_li,
                          const uint32_t* __restrict__ vmask, int64_t n_pix, int spp, float* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int k = 0; k < spp; ++k) {
    const size_t sl = (size_t)p * spp + k;
    if (!((__ldg(vmask + (sl >> 5)) >> (sl & 31)) & 1u)) continue;
    const size_t s = 3 * sl;
    float l0 = slot_ld[s + 0], l1 = slot_ld[s + 1], l2 = slot_ld[s + 2];
    if (slot_li) { l0 = l0 + slot_li[s + 0]; l1 = l1 + slot_li[s + 1]; l2 = l2 + slot_li[s + 2]; }
    a0 = a0 + l0;
    a1 = a1 + l1;
    a2 = a2 + l2;
  }
  out[3 * p + 0] = a0 / (float)spp;
  out[3 * p + 1] = a1 / (float)spp;
  out[3 * p + 2] = a2 / (float)spp;
}

// -------------------------------------------------------------- path tracer
template <int DT>
__global__ void __launch_bounds__(128, 8) k_path_samples(Vol V, DevLights L, CamF cam, float g, int spp, int k0, int kc,
                                                      int max_bounces, int use_rr, uint64_t seed, int64_t n_items,
                                                      float* __restrict__ slot_rad, uint32_t* err,
                                                      unsigned long long* stats) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  int k, px, py;
  int64_t pix;
  slot_pixel(it, n_items, kc, cam.W, &k, &pix, &px, &py);
  k += k0;
  Rng rng(seed, TAG_CAMERA, (uint64_t)pix, (uint32_t)k);
  float b0[4]; rng.uni4(b0);
  V3 o, d;
  camera_ray(cam, px, py, b0[0], b0[1], &o, &d);
  V3 rad = v3(0.f, 0.f, 0.f);
  uint32_t nfetch = 0;
  float beta0 = 1.f, beta1 = 1.f, beta2 = 1.f;
  float t0, t1;
  if (box_hit(o, d, &t0, &t1)) {
    float t = t0;
    for (int j = 1; j <= max_bounces; ++j) {
      float th;
      if (!delta_track<DT, false>(V, o, d, t, t1, rng, &th, err, nfetch)) break;
      V3 x = along(o, d, th);
      float sig; V3 alb;
      medium_at<DT>(V, x, &sig, &alb);
      V3 Lr = v3(0.f, 0.f, 0.f);
      for (int l = 0; l < L.n; ++l) {
        V3 wl, E; float dist;
        light_geom(L.l[l], x, &wl, &dist, &E);
        float a0, a1, tend = 0.f;
        if (box_hit(x, wl, &a0, &a1)) tend = mn(a1, dist);
        Rng rs(seed, TAG_SHADOW, shadow_item((uint64_t)pix, j, l), (uint32_t)k);
        float T = ratio_track<DT, false>(V, x, wl, tend, rs, err, nfetch);
        float ph = hg_eval(g, dot(d, wl));
        Lr = v3(Lr.x + ph * T * E.x, Lr.y + ph * T * E.y, Lr.z + ph * T * E.z);
      }
      float c0 = beta0 * alb.x, c1 = beta1 * alb.y, c2 = beta2 * alb.z;
      rad = v3(rad.x + c0 * Lr.x, rad.y + c1 * Lr.y, rad.z + c2 * Lr.z);
      beta0 = c0; beta1 = c1; beta2 = c2;
      if (j == max_bounces) break;
      float w[4]; rng.uni4(w);
      V3 nd = hg_sample(g, d, w[0], w[1]);
      if (use_rr && j >= 3) {
        float q = mx(beta0, mx(beta1, beta2));
        if (q > 1.f) q = 1.f;
        if (!(w[2] < q)) break;
        beta0 = beta0 / q; beta1 = beta1 / q; beta2 = beta2 / q;
      }
      o = x; d = nd;
      float a0, a1;
      if (!box_hit(o, d, &a0, &a1)) break;
      t = 0.f; t1 = a1;
    }
  }
  slot_rad[3 * it + 0] = rad.x;
  slot_rad[3 * it + 1] = rad.y;
  slot_rad[3 * it + 2] = rad.z;
  if (stats) atomicAdd(stats, (unsigned long long)nfetch);
}

// acc[p] += r[p][k] for the chunk's samples in order; on the last chunk,
// out = acc / spp.
// The path tracer proper: persistent warps (a block's four warps refill
// independently) in which each lane carries one camera sample's path at a
// time and the loop body advances every lane by one interaction (free flight
// to the next real collision, next-event estimation towards every light,
// Henyey-Greenstein continuation, Russian roulette); a lane whose path ended
// takes the next sample from a global counter.  Paths differ widely in
// length, so a thread per sample leaves most lanes idle while the warp's
// longest path finishes.  A sample's arithmetic and random streams are those
// of k_path_samples (its streams are keyed by pixel and sample), so the
// per-sample radiance is the same bit for bit.
template <int DT>
__global__ void __launch_bounds__(128, 8) k_path_persistent(Vol V, DevLights L, CamF cam, float g, int spp, int k0, int kc,
                                                      int max_bounces, int use_rr, uint64_t seed, int64_t n_items,
                                                      float* __restrict__ slot_rad, unsigned long long* __restrict__ next,
                                                      uint32_t* err) {
  const int lane = threadIdx.x & 31;
  bool has = false;
  int64_t it = 0;
  int64_t pix = 0;
  int k = 0, j = 0;
  V3 o = v3(0.f, 0.f, 0.f), d = o, rad = o;
  float beta0 = 1.f, beta1 = 1.f, beta2 = 1.f, t = 0.f, t1 = 0.f;
  Rng rng(0, 0, 0, 0);
  uint32_t nfetch = 0;
  auto finish = [&]() {
    slot_rad[3 * it + 0] = rad.x; slot_rad[3 * it + 1] = rad.y; slot_rad[3 * it + 2] = rad.z;
    has = false;
  };
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !has);
    bool exhausted = false;
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      exhausted = (int64_t)(base + (unsigned long long)__popc(need)) >= n_items;
      if (!has) {
        const int64_t q = (int64_t)(base + (unsigned long long)__popc(need & ((1u << lane) - 1u)));
        if (q < n_items) {
          it = q; has = true;
          int px, py;
          slot_pixel(it, n_items, kc, cam.W, &k, &pix, &px, &py);
          k += k0;
          rng = Rng(seed, TAG_CAMERA, (uint64_t)pix, (uint32_t)k);
          float b0[4]; rng.uni4(b0);
          camera_ray(cam, px, py, b0[0], b0[1], &o, &d);
          rad = v3(0.f, 0.f, 0.f);
          beta0 = beta1 = beta2 = 1.f;
          j = 0;
          float t0_, t1_;
          if (box_hit(o, d, &t0_, &t1_)) { t = t0_; t1 = t1_; } else finish();
        }
      }
    }
    if (!__any_sync(0xffffffffu, has)) {
      if (exhausted) break;
      continue;
    }
    if (!has) continue;
    j = j + 1;
    float th;
    if (!delta_track<DT>(V, o, d, t, t1, rng, &th, err, nfetch)) { finish(); continue; }
    const V3 x = along(o, d, th);
    float sig; V3 alb;
    medium_at<DT>(V, x, &sig, &alb);
    V3 Lr = v3(0.f, 0.f, 0.f);
    for (int l = 0; l < L.n; ++l) {
      V3 wl, E; float dist;
      light_geom(L.l[l], x, &wl, &dist, &E);
      float a0, a1, tend = 0.f;
      if (box_hit(x, wl, &a0, &a1)) tend = mn(a1, dist);
      Rng rs(seed, TAG_SHADOW, shadow_item((uint64_t)pix, j, l), (uint32_t)k);
      float T = ratio_track<DT>(V, x, wl, tend, rs, err, nfetch);
      float ph = hg_eval(g, dot(d, wl));
      Lr = v3(Lr.x + ph * T * E.x, Lr.y + ph * T * E.y, Lr.z + ph * T * E.z);
    }
    const float c0 = beta0 * alb.x, c1 = beta1 * alb.y, c2 = beta2 * alb.z;
    rad = v3(rad.x + c0 * Lr.x, rad.y + c1 * Lr.y, rad.z + c2 * Lr.z);
    beta0 = c0; beta1 = c1; beta2 = c2;
    if (j == max_bounces) { finish(); continue; }
    float w[4]; rng.uni4(w);
    const V3 nd = hg_sample(g, d, w[0], w[1]);
    if (use_rr && j >= 3) {
      float q = mx(beta0, mx(beta1, beta2));
      if (q > 1.f) q = 1.f;
      if (!(w[2] < q)) { finish(); continue; }
      beta0 = beta0 / q; beta1 = beta1 / q; beta2 = beta2 / q;
    }
    o = x; d = nd;
    float a0, a1;
    if (!box_hit(o, d, &a0, &a1)) { finish(); continue; }
    t = 0.f; t1 = a1;
  }
}

__global__ void k_path_accumulate(const float* __restrict__ slot_rad, int64_t n_pix, int kc, int first, int last,
                                  int spp, float* __restrict__ acc, float* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  float a0 = first ? 0.f : acc[3 * p], a1 = first ? 0.f : acc[3 * p + 1], a2 = first ? 0.f : acc[3 * p + 2];
  for (int k = 0; k < kc; ++k) {
    size_t s = 3 * ((size_t)p * kc + k);
    a0 = a0 + slot_rad[s]; a1 = a1 + slot_rad[s + 1]; a2 = a2 + slot_rad[s + 2];
  }
  if (last) {
    out[3 * p] = a0 / (float)spp; out[3 * p + 1] = a1 / (float)spp; out[3 * p + 2] = a2 / (float)spp;
  } else {
    acc[3 * p] = a0; acc[3 * p + 1] = a1; acc[3 * p + 2] = a2;
  }
}

// Camera frame in double on the host, rounded once to float.
CamF make_cam(const pf_camera* c) {
  double eye[3] = {c->eye[0], c->eye[1], c->eye[2]};
  double f[3] = {(double)c->at[0] - eye[0], (double)c->at[1] - eye[1], (double)c->at[2] - eye[2]};
  double up[3] = {c->up[0], c->up[1], c->up[2]};
  double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int i = 0; i < 3; ++i) f[i] /= fn;
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int i = 0; i < 3; ++i) r[i] /= rn;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  double th = std::tan(0.5 * (double)c->fovy_deg * M_PI / 180.0);
  CamF o;
  for (int i = 0; i < 3; ++i) { o.eye[i] = (float)eye[i]; o.f[i] = (float)f[i]; o.r[i] = (float)r[i]; o.u[i] = (float)u[i]; }
  o.sy = (float)th;
  o.sx = (float)(th * (double)c->width / (double)c->height);
  o.W = c->width; o.H = c->height;
  return o;
}

// ---- ray marching with the field at every step (Sec. 3.6) -----------------
// Camera sample k of pixel p: the ray from block 0 of (seed, tag 1, p, k)
// (pixel jitter, march offset u in lane 2).  Segment s covers
// [t0 + s h, min(t0 + (s+1) h, t1)); its sample point sits at fraction u,
// with sigma_s and albedo_s there; weight a_s = exp(-tau_s) (1 - exp(-sigma_s
// len_s)), tau_s the (compensated) optical depth before the segment.  L_d
// towards every light by a marched shadow ray whose jitter is lane l % 4 of
// Philox block 4 s + l / 4 of (seed, tag 6, p, k).  A segment with sigma_s > 0
// asks one field query (x_s, -d, g) with weight a_s albedo_s.
constexpr uint32_t kTagMarch = 6;

// EMIT = false: count the queries of each ray; EMIT = true: write them (at
// off[ray] - base, when q is given) and each ray's direct part.
template <int DT, bool EMIT>
__global__ void __launch_bounds__(128) k_raymarch(Vol V, DevLights L, CamF cam, float g, int spp, float h,
                                                  uint64_t seed, int64_t r0, int64_t n_rays,
                                                  uint32_t* __restrict__ counts, const uint64_t* __restrict__ off,
                                                  uint64_t base, float* __restrict__ q, float* __restrict__ wgt,
                                                  float* __restrict__ direct) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rays) return;
  const int64_t ray = r0 + i;
  int k, px, py;
  int64_t pix;
  slot_pixel(ray, r0 + n_rays, spp, cam.W, &k, &pix, &px, &py);
  Rng rng(seed, TAG_CAMERA, (uint64_t)pix, (uint32_t)k);
  float b0[4];
  rng.uni4(b0);
  V3 o, d;
  camera_ray(cam, px, py, b0[0], b0[1], &o, &d);
  uint32_t n = 0;
  V3 D = v3(0.f, 0.f, 0.f);
  uint64_t j = (EMIT && q) ? off[ray] - base : 0;
  const uint64_t j_end = (EMIT && q) ? off[ray + 1] - base : 0;   // the ray's range (the count pass's)
  float t0, t1;
  if (box_hit(o, d, &t0, &t1)) {
    float qth, qph;
    query_angles(-d.x, -d.y, -d.z, &qth, &qph);
    float tau = 0.f, comp = 0.f;
    const int nseg = (int)ceilf((t1 - t0) / h);
    for (int s = 0; s < nseg; ++s) {
      const float s0 = t0 + (float)s * h;
      const float s1 = mn(t0 + (float)(s + 1) * h, t1);
      const float len = s1 - s0;
      if (!(len > 0.f)) continue;
      const V3 x = along(o, d, s0 + b0[2] * len);
      float sg;
      V3 alb;
      medium_at<DT>(V, x, &sg, &alb);
      if (sg > 0.f) {
        ++n;
        if (EMIT) {
          const float a = expf(-(tau - comp)) * -expm1f(-sg * len);
          V3 Ld = v3(0.f, 0.f, 0.f);
          Rng rs(seed, kTagMarch, (uint64_t)pix, (uint32_t)k);
          for (int gq = 0; 4 * gq < L.n; ++gq) {
            rs.c3 = (uint32_t)(4 * s + gq);
            float jit[4];
            rs.uni4(jit);
            for (int ii = 0; ii < 4 && 4 * gq + ii < L.n; ++ii) {
              V3 wl, E;
              float dist;
              light_geom(L.l[4 * gq + ii], x, &wl, &dist, &E);
              float a0, a1, tend = 0.f;
              if (box_hit(x, wl, &a0, &a1)) tend = mn(a1, dist);
              float st = 0.f, sc = 0.f;
              if (tend > 0.f) {
                const int ns = (int)ceilf(tend / h);
                for (int m = 0; m < ns; m += kMarchAhead) {    // lookups ahead, sums in order
                  float sg4[kMarchAhead], ml4[kMarchAhead];
#pragma unroll
                  for (int u = 0; u < kMarchAhead; ++u) {
                    const float m0 = (float)(m + u) * h;
                    ml4[u] = mn((float)(m + u + 1) * h, tend) - m0;
                    sg4[u] = sigma_at<DT>(V, along(x, wl, m0 + jit[ii] * ml4[u]));
                  }
#pragma unroll
                  for (int u = 0; u < kMarchAhead; ++u) {
                    if (m + u >= ns) break;
                    if (!(ml4[u] > 0.f)) continue;
                    const float y = sg4[u] * ml4[u] - sc;
                    const float t = st + y;
                    sc = (t - st) - y;
                    st = t;
                  }
                }
              }
              const float T = expf(-(st - sc));
              const float ph = hg_eval(g, dot(d, wl));
              Ld = v3(Ld.x + ph * T * E.x, Ld.y + ph * T * E.y, Ld.z + ph * T * E.z);
            }
          }
          const V3 w = v3(a * alb.x, a * alb.y, a * alb.z);
          D = v3(D.x + w.x * Ld.x, D.y + w.y * Ld.y, D.z + w.z * Ld.z);
          if (EMIT && q && j < j_end) {
            q[6 * j + 0] = x.x; q[6 * j + 1] = x.y; q[6 * j + 2] = x.z;
            q[6 * j + 3] = qth; q[6 * j + 4] = qph; q[6 * j + 5] = g;
            wgt[3 * j + 0] = w.x; wgt[3 * j + 1] = w.y; wgt[3 * j + 2] = w.z;
            ++j;
          }
        }
      }
      const float y = sg * len - comp;
      const float t = tau + y;
      comp = (t - tau) - y;
      tau = t;
    }
  }
  if (!EMIT) {
    counts[i] = n;
  } else {
    direct[3 * i + 0] = D.x; direct[3 * i + 1] = D.y; direct[3 * i + 2] = D.z;
  }
}

// out[p] = off[p * spp], p <= n_pix: the query offsets at pixel boundaries.
__global__ void k_pixel_offsets(const uint64_t* __restrict__ off, int spp, int64_t n_pix, uint64_t* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= n_pix) out[p] = off[p * spp];
}

__global__ void k_iota(uint32_t* __restrict__ v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

// Pixel p0 + i: the mean over its samples of the direct part plus the
// weighted field values of the sample's queries (li, nullable).
__global__ void k_raymarch_compose(const float* __restrict__ direct, const float* __restrict__ li,
                                   const uint64_t* __restrict__ off, uint64_t base, int64_t p0, int64_t n_pix,
                                   int spp, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pix) return;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int k = 0; k < spp; ++k) {
    const int64_t rl = i * spp + k;                  // ray within the chunk
    a0 += direct[3 * rl]; a1 += direct[3 * rl + 1]; a2 += direct[3 * rl + 2];
    if (li) {
      const int64_t ray = p0 * spp + rl;
      for (uint64_t jj = off[ray] - base; jj < off[ray + 1] - base; ++jj) {
        a0 += li[3 * jj]; a1 += li[3 * jj + 1]; a2 += li[3 * jj + 2];
      }
    }
  }
  const float inv = 1.0f / (float)spp;
  const int64_t p = p0 + i;
  out[3 * p] = a0 * inv; out[3 * p + 1] = a1 * inv; out[3 * p + 2] = a2 * inv;
}

// Launches k_nee as a grid-stride loop over the compacted list with as many
// blocks as fit on the device at once.
template <int DT>
pf_status launch_nee(pf_ctx* ctx, const Vol& V, const Vol& Vw, const DevLights& L, float g, int spp, uint64_t seed,
                     int64_t n_max, const float* cq, const float* cdir, const float* calb, const uint32_t* cidx,
                     const uint32_t* ccount, const uint32_t* perm, float* ld) {
  const size_t bytes = (size_t)kNeeWarps * kNeeWarpFloats * sizeof(float);
  const bool thin = Vw.B > V.B;
  // per-(light, sample) contributions, sized for the worst case (every slot
  // scatters), and the work counter (in the bytes after the sample count)
  float* contrib;
  PF_TRY(pf_scratch(ctx, WS_NEE_CONTRIB, (size_t)L.n * (size_t)n_max * 2 * sizeof(float), (void**)&contrib));
  unsigned long long* next = (unsigned long long*)((char*)ccount + 64);
  PF_CUDA(ctx, cudaMemsetAsync(next, 0, sizeof(unsigned long long), ctx->stream));
  int o = 0;  // resident blocks per SM
  if (thin) PF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nee<DT, true>, 32 * kNeeWarps, bytes));
  else PF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nee<DT, false>, 32 * kNeeWarps, bytes));
  const unsigned nb = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n_max * L.n + 127) / 128, (int64_t)ctx->num_sms * std::max(o, 1)));
  if (thin)
    k_nee<DT, true><<<nb, 32 * kNeeWarps, bytes, ctx->stream>>>(V, Vw, L, g, spp, seed, cq, cdir, cidx, ccount, perm,
                                                                next, contrib, ctx->err_dev, ctx->counters);
  else
    k_nee<DT, false><<<nb, 32 * kNeeWarps, bytes, ctx->stream>>>(V, Vw, L, g, spp, seed, cq, cdir, cidx, ccount, perm,
                                                                 next, contrib, ctx->err_dev, ctx->counters);
  PF_CUDA(ctx, cudaGetLastError());
  k_nee_sum<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n_max + 255) / 256, (int64_t)ctx->num_sms * 8)), 256, 0,
              ctx->stream>>>(contrib, L, calb, cidx, ccount, perm, ld);
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

}  // namespace

// A finite, non-degenerate camera frame: eye, at and up finite, eye != at,
// up not parallel to at - eye (the trackers' walks rely on finite rays).
static bool cam_frame_ok(const pf_camera* cam) {
  double f[3], up[3], fn = 0.0, un = 0.0;
  for (int i = 0; i < 3; ++i) {
    if (!std::isfinite(cam->eye[i]) || !std::isfinite(cam->at[i]) || !std::isfinite(cam->up[i])) return false;
    f[i] = (double)cam->at[i] - (double)cam->eye[i];
    up[i] = cam->up[i];
    fn += f[i] * f[i];
    un += up[i] * up[i];
  }
  const double r0 = f[1] * up[2] - f[2] * up[1], r1 = f[2] * up[0] - f[0] * up[2], r2 = f[0] * up[1] - f[1] * up[0];
  return fn > 0.0 && r0 * r0 + r1 * r1 + r2 * r2 > 1e-12 * fn * un;
}

static pf_status check_cam(pf_ctx* ctx, const pf_camera* cam, int spp) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0 || spp > (1 << 24))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "camera size and spp must be positive (spp < 2^24)");
  if (!(cam->fovy_deg > 0.f && cam->fovy_deg < 180.f))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "fovy_deg must lie in (0, 180)");
  if (!cam_frame_ok(cam))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "camera needs finite eye, at, up with eye != at and up not parallel to at - eye");
  return PF_OK;
}

extern "C" pf_status pf_render_neural(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights,
                                      float g, const pf_camera* cam, int spp, float step_vox, uint64_t seed,
                                      const pf_field* field, float* out_rgb_dev) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, vol));
  PF_TRY(pf_check_lights(ctx, lights, n_lights));
  PF_TRY(check_cam(ctx, cam, spp));
  if (!out_rgb_dev) return pf_fail(ctx, PF_ERR_INVALID_ARG, "out_rgb_dev is NULL");
  if (!(step_vox == 0.f || (step_vox >= 0.05f && step_vox <= 64.f)) || !(g > -1.f && g < 1.f))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "need step_vox = 0 or in [0.05, 64] voxels, and |g| < 1");
  if (field && field->ctx != ctx) return pf_fail(ctx, PF_ERR_INVALID_ARG, "field belongs to another context");
  const float* grid = nullptr;
  if (step_vox == 0.f) PF_TRY(pf_grid_for(ctx, vol, &grid));
  int64_t n_pix = (int64_t)cam->width * cam->height;
  int64_t n_slots = n_pix * spp;
  if (n_slots > (int64_t)0xFFFFFFFFll) return pf_fail(ctx, PF_ERR_INVALID_ARG, "width*height*spp must be < 2^32");
  bool march = step_vox > 0.f;
  float *ld, *li, *cq = nullptr, *calb = nullptr, *cdir = nullptr;
  uint32_t *cidx = nullptr, *ccount = nullptr;
  PF_TRY(pf_scratch(ctx, WS_SLOT_LD, n_slots * 3 * sizeof(float), (void**)&ld));
  PF_TRY(pf_scratch(ctx, WS_SLOT_LI, n_slots * 3 * sizeof(float), (void**)&li));
  if (field || !march) {
    PF_TRY(pf_scratch(ctx, WS_COMPACT_Q, n_slots * 6 * sizeof(float), (void**)&cq));
    PF_TRY(pf_scratch(ctx, WS_SLOT_ALB, n_slots * 3 * sizeof(float), (void**)&calb));
    PF_TRY(pf_scratch(ctx, WS_COMPACT_IDX, n_slots * sizeof(uint32_t), (void**)&cidx));
    PF_TRY(pf_scratch(ctx, WS_MISC, 256, (void**)&ccount));
    PF_CUDA(ctx, cudaMemsetAsync(ccount, 0, sizeof(uint32_t), ctx->stream));
  }
  uint32_t *ckey = nullptr, *chist = nullptr, *cfill = nullptr, *perm = nullptr, *vmask = nullptr;
  PF_TRY(pf_scratch(ctx, WS_VMASK, (size_t)((n_slots + 31) / 32) * sizeof(uint32_t), (void**)&vmask));
  uint64_t* coff = nullptr;
  if (!march) {
    PF_TRY(pf_scratch(ctx, WS_COMPACT_DIR, n_slots * 3 * sizeof(float), (void**)&cdir));
    PF_TRY(pf_scratch(ctx, WS_CELL_KEY, n_slots * sizeof(uint32_t), (void**)&ckey));
    PF_TRY(pf_scratch(ctx, WS_CELL_PERM, n_slots * sizeof(uint32_t), (void**)&perm));
    PF_TRY(pf_scratch(ctx, WS_CELL_HIST, 2 * kCells * sizeof(uint32_t), (void**)&chist));
    PF_TRY(pf_scratch(ctx, WS_CELL_OFF, (kCells + 1) * sizeof(uint64_t), (void**)&coff));
    cfill = chist + kCells;
    PF_CUDA(ctx, cudaMemsetAsync(chist, 0, 2 * kCells * sizeof(uint32_t), ctx->stream));
  }
  Vol V = pf_make_vol(vol, 0.f, grid);
  // coarser grids, max-pooled from the brick grid: the camera rays' free
  // flight (brick_primary) and the shadow rays' walk (brick_shadow)
  auto pooled_vol = [&](int edge, int slot, Vol* out) -> pf_status {
    *out = V;
    if (march || edge <= V.B) return PF_OK;
    const int f = edge / V.B;
    const int px = (V.gx + f - 1) / f, py = (V.gy + f - 1) / f, pz = (V.gz + f - 1) / f;
    const int64_t np = (int64_t)px * py * pz;
    float* pooled;
    PF_TRY(pf_scratch(ctx, slot, (size_t)np * sizeof(float), (void**)&pooled));
    k_pool_majorants<<<(unsigned)((np + 127) / 128), 128, 0, ctx->stream>>>(grid, V.gx, V.gy, V.gz, f, px, py, pz,
                                                                           pooled);
    PF_CUDA(ctx, cudaGetLastError());
    *out = pf_make_vol(vol, 0.f, pooled, edge);
    return PF_OK;
  };
  Vol Vp, Vs;
  PF_TRY(pooled_vol(vol->brick_primary, WS_GRID_PRIMARY, &Vp));
  PF_TRY(pooled_vol(vol->brick_shadow, WS_GRID_SHADOW, &Vs));
  if (!march) {   // the walks' bordered copies, one per distinct grid
    PF_TRY(pf_bordered_grid(ctx, V.mg, V.gx, V.gy, V.gz, WS_GRID_WALK, &V.mgw));
    if (Vp.mg == V.mg) Vp.mgw = V.mgw;
    else PF_TRY(pf_bordered_grid(ctx, Vp.mg, Vp.gx, Vp.gy, Vp.gz, WS_GRID_PRIMARY_WALK, &Vp.mgw));
    if (Vs.mg == V.mg) Vs.mgw = V.mgw;
    else PF_TRY(pf_bordered_grid(ctx, Vs.mg, Vs.gx, Vs.gy, Vs.gz, WS_GRID_SHADOW_WALK, &Vs.mgw));
  }
  DevLights L = pf_make_lights(lights, n_lights);
  CamF C = make_cam(cam);
  int nmax = std::max(vol->nx, std::max(vol->ny, vol->nz));
  float h = step_vox > 0.f ? step_vox / (float)nmax : 0.f;
  dim3 blk(128), grd((unsigned)((n_slots + 127) / 128));
  {
  StageTimer tm(ctx, PF_STAGE_CAMERA);
#define LAUNCH_CS(DT)                                                                                              \
  if (march) k_camera_samples_march<DT><<<grd, blk, 0, ctx->stream>>>(Vp, L, C, g, spp, h, seed, n_slots, ld, li, cq, \
                                                                      calb, cdir, cidx, ccount, ckey, chist, vmask, \
                                                                      ctx->err_dev, ctx->counters);                 \
  else k_camera_samples<DT><<<grd, blk, 0, ctx->stream>>>(Vp, L, C, g, spp, h, seed, n_slots, ld, li, cq, calb, \
                                                                 cdir, cidx, ccount, ckey, chist, vmask,            \
                                                                 ctx->err_dev, ctx->counters);
  if (vol->dtype == PF_F32) { LAUNCH_CS(0) } else if (vol->dtype == PF_F16) { LAUNCH_CS(1) } else { LAUNCH_CS(2) }
#undef LAUNCH_CS
  }
  PF_CUDA(ctx, cudaGetLastError());
  if (!march) {
    StageTimer tm(ctx, PF_STAGE_NEE);
    PF_TRY(pf_scan_u32(ctx, chist, coff, kCells));
    k_place<<<(unsigned)std::min<int64_t>((n_slots + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
        ckey, ccount, coff, cfill, perm);
    PF_CUDA(ctx, cudaGetLastError());
    if (vol->dtype == PF_F32)
      PF_TRY(launch_nee<0>(ctx, V, Vs, L, g, spp, seed, n_slots, cq, cdir, calb, cidx, ccount, perm, ld));
    else if (vol->dtype == PF_F16)
      PF_TRY(launch_nee<1>(ctx, V, Vs, L, g, spp, seed, n_slots, cq, cdir, calb, cidx, ccount, perm, ld));
    else
      PF_TRY(launch_nee<2>(ctx, V, Vs, L, g, spp, seed, n_slots, cq, cdir, calb, cidx, ccount, perm, ld));
  }
  if (field) {
    StageTimer tm(ctx, PF_STAGE_FIELD);
    // The number of valid samples is only known on the device; the field pass
    // reads it from there and covers the worst case n_slots.
    PF_TRY(pf_field_forward_impl(ctx, field, cq, n_slots, ccount, nullptr, cidx, calb, li));
  }
  {
    StageTimer tm(ctx, PF_STAGE_COMPOSE);
    k_compose<<<(unsigned)((n_pix + 127) / 128), 128, 0, ctx->stream>>>(ld, field ? li : nullptr, vmask, n_pix, spp,
                                                                        out_rgb_dev);
  }
  PF_CUDA(ctx, cudaGetLastError());
  return PF_OK;
}

// Ray marching with the field at every step: count the field queries of every
// camera sample, then render in chunks of whole pixels whose queries fit the
// query buffer (queries + weights, the field forward with the render
// epilogue, compose).
extern "C" pf_status pf_render_raymarched(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights,
                                          float g, const pf_camera* cam, int spp, float step_vox, uint64_t seed,
                                          const pf_field* field, float* out_rgb_dev) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, vol));
  PF_TRY(pf_check_lights(ctx, lights, n_lights));
  PF_TRY(check_cam(ctx, cam, spp));
  if (!out_rgb_dev) return pf_fail(ctx, PF_ERR_INVALID_ARG, "out_rgb_dev is NULL");
  if (!(step_vox >= 0.05f && step_vox <= 64.f) || !(g > -1.f && g < 1.f))
    return pf_fail(ctx, PF_ERR_INVALID_ARG, "need step_vox in [0.05, 64] voxels and |g| < 1");
  if (field && field->ctx != ctx) return pf_fail(ctx, PF_ERR_INVALID_ARG, "field belongs to another context");
  const int64_t n_pix = (int64_t)cam->width * cam->height;
  const int64_t n_rays = n_pix * spp;
  if (n_rays > (int64_t)0xFFFFFFFFll) return pf_fail(ctx, PF_ERR_INVALID_ARG, "width*height*spp must be < 2^32");
  const Vol V = pf_make_vol(vol, 0.f, nullptr);
  const DevLights L = pf_make_lights(lights, n_lights);
  const CamF C = make_cam(cam);
  const int nmax = std::max(vol->nx, std::max(vol->ny, vol->nz));
  const float h = step_vox / (float)nmax;
  float* direct;
  PF_TRY(pf_scratch(ctx, WS_SLOT_LD, (size_t)n_rays * 3 * sizeof(float), (void**)&direct));
#define RM_LAUNCH(EMIT, r0_, n_, ...)                                                                              \
  do {                                                                                                             \
    const unsigned gr_ = (unsigned)(((n_) + 127) / 128);                                                           \
    if (vol->dtype == PF_F32) k_raymarch<0, EMIT><<<gr_, 128, 0, ctx->stream>>>(V, L, C, g, spp, h, seed, r0_, n_, \
                                                                               __VA_ARGS__);                       \
    else if (vol->dtype == PF_F16) k_raymarch<1, EMIT><<<gr_, 128, 0, ctx->stream>>>(V, L, C, g, spp, h, seed, r0_, \
                                                                                    n_, __VA_ARGS__);              \
    else k_raymarch<2, EMIT><<<gr_, 128, 0, ctx->stream>>>(V, L, C, g, spp, h, seed, r0_, n_, __VA_ARGS__);        \
    PF_CUDA(ctx, cudaGetLastError());                                                                              \
  } while (0)
  if (!field) {
    StageTimer tm(ctx, PF_STAGE_CAMERA);
    RM_LAUNCH(true, (int64_t)0, n_rays, nullptr, nullptr, (uint64_t)0, nullptr, nullptr, direct);
    k_raymarch_compose<<<(unsigned)((n_pix + 127) / 128), 128, 0, ctx->stream>>>(direct, nullptr, nullptr, 0, 0, n_pix,
                                                                                spp, out_rgb_dev);
    PF_CUDA(ctx, cudaGetLastError());
    return PF_OK;
  }
  uint32_t* counts;
  uint64_t* off;
  PF_TRY(pf_scratch(ctx, WS_COMPACT_IDX, (size_t)n_rays * sizeof(uint32_t), (void**)&counts));
  PF_TRY(pf_scratch(ctx, WS_CELL_OFF, (size_t)(n_rays + 1) * sizeof(uint64_t), (void**)&off));
  {
    StageTimer tm(ctx, PF_STAGE_CAMERA);
    RM_LAUNCH(false, (int64_t)0, n_rays, counts, nullptr, (uint64_t)0, nullptr, nullptr, nullptr);
  }
  PF_TRY(pf_scan_u32(ctx, counts, off, n_rays));
  // the offsets at pixel boundaries plan the chunks on the host
  uint64_t* poff;
  PF_TRY(pf_scratch(ctx, WS_CELL_KEY, (size_t)(n_pix + 1) * sizeof(uint64_t), (void**)&poff));
  k_pixel_offsets<<<(unsigned)((n_pix + 1 + 255) / 256), 256, 0, ctx->stream>>>(off, spp, n_pix, poff);
  PF_CUDA(ctx, cudaGetLastError());
  std::vector<uint64_t> hoff((size_t)n_pix + 1);
  PF_CUDA(ctx, cudaMemcpyAsync(hoff.data(), poff, hoff.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // query buffer: 2^23 queries, or one pixel's worth if that is more
  uint64_t cap = 1ull << 23, most = 0;
  for (int64_t p = 0; p < n_pix; ++p) most = std::max(most, hoff[(size_t)p + 1] - hoff[(size_t)p]);
  cap = std::max(cap, most);
  cap = std::min<uint64_t>(cap, std::max<uint64_t>(hoff[(size_t)n_pix], 1));
  float *q, *wgt, *li;
  uint32_t* iota;
  PF_TRY(pf_scratch(ctx, WS_COMPACT_Q, (size_t)cap * 6 * sizeof(float), (void**)&q));
  PF_TRY(pf_scratch(ctx, WS_SLOT_ALB, (size_t)cap * 3 * sizeof(float), (void**)&wgt));
  PF_TRY(pf_scratch(ctx, WS_SLOT_LI, (size_t)cap * 3 * sizeof(float), (void**)&li));
  PF_TRY(pf_scratch(ctx, WS_CELL_PERM, (size_t)cap * sizeof(uint32_t), (void**)&iota));
  k_iota<<<(unsigned)((cap + 255) / 256), 256, 0, ctx->stream>>>(iota, (int64_t)cap);
  PF_CUDA(ctx, cudaGetLastError());
  for (int64_t p0 = 0; p0 < n_pix;) {
    // the most whole pixels from p0 whose queries fit the buffer
    int64_t lo = p0 + 1, hi = n_pix;
    const uint64_t base = hoff[(size_t)p0];
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (hoff[(size_t)mid] - base <= cap) lo = mid;
      else hi = mid - 1;
    }
    const int64_t p1 = lo;
    const int64_t nq = (int64_t)(hoff[(size_t)p1] - base);
    {
      StageTimer tm(ctx, PF_STAGE_CAMERA);
      RM_LAUNCH(true, p0 * spp, (p1 - p0) * spp, nullptr, off, base, q, wgt, direct);
    }
    if (nq > 0) {
      StageTimer tm(ctx, PF_STAGE_FIELD);
      PF_TRY(pf_field_forward_impl(ctx, field, q, nq, nullptr, nullptr, iota, wgt, li));
    }
    {
      StageTimer tm(ctx, PF_STAGE_COMPOSE);
      k_raymarch_compose<<<(unsigned)((p1 - p0 + 127) / 128), 128, 0, ctx->stream>>>(direct, nq > 0 ? li : nullptr,
                                                                                    off, base, p0, p1 - p0, spp,
                                                                                    out_rgb_dev);
      PF_CUDA(ctx, cudaGetLastError());
    }
    p0 = p1;
  }
#undef RM_LAUNCH
  return PF_OK;
}

extern "C" pf_status pf_render_pathtraced(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights,
                                          float g, const pf_camera* cam, int spp, int max_bounces, uint64_t seed,
                                          int use_rr, float* out_rgb_dev) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  PF_TRY(pf_check_volume(ctx, vol));
  PF_TRY(pf_check_lights(ctx, lights, n_lights));
  PF_TRY(check_cam(ctx, cam, spp));
  if (!out_rgb_dev) return pf_fail(ctx, PF_ERR_INVALID_ARG, "out_rgb_dev is NULL");
  if (max_bounces < 1 || max_bounces > 1024) return pf_fail(ctx, PF_ERR_INVALID_ARG, "max_bounces must be in [1, 1024]");
  if (!(g > -1.f && g < 1.f)) return pf_fail(ctx, PF_ERR_INVALID_ARG, "|g| must be < 1");
  const float* grid;
  PF_TRY(pf_grid_for(ctx, vol, &grid));
  int64_t n_pix = (int64_t)cam->width * cam->height;
  // samples per chunk: keep the per-sample scratch within 2^26 slots
  int64_t kc = std::max<int64_t>(1, std::min<int64_t>(spp, ((int64_t)1 << 26) / n_pix));
  float *rad, *acc;
  PF_TRY(pf_scratch(ctx, WS_SLOT_LD, (size_t)(n_pix * kc * 3) * sizeof(float), (void**)&rad));
  PF_TRY(pf_scratch(ctx, WS_SLOT_ALB, (size_t)(n_pix * 3) * sizeof(float), (void**)&acc));
  unsigned long long* next;   // the persistent kernel's sample counter
  PF_TRY(pf_scratch(ctx, WS_MISC, 256, (void**)&next));
  Vol V = pf_make_vol(vol, 0.f, grid);
  PF_TRY(pf_bordered_grid(ctx, grid, V.gx, V.gy, V.gz, WS_GRID_WALK, &V.mgw));
  DevLights L = pf_make_lights(lights, n_lights);
  CamF C = make_cam(cam);
  StageTimer tm(ctx, PF_STAGE_PATH);
  for (int k0 = 0; k0 < spp; k0 += (int)kc) {
    int kn = (int)std::min<int64_t>(kc, spp - k0);
    int64_t n_items = n_pix * kn;
    PF_CUDA(ctx, cudaMemsetAsync(next, 0, sizeof(unsigned long long), ctx->stream));
    const dim3 pg((unsigned)std::min<int64_t>((int64_t)ctx->num_sms * 8, (n_items + 127) / 128));
    if (vol->dtype == PF_F32)
      k_path_persistent<0><<<pg, 128, 0, ctx->stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad,
                                                        next, ctx->err_dev);
    else if (vol->dtype == PF_F16)
      k_path_persistent<1><<<pg, 128, 0, ctx->stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad,
                                                        next, ctx->err_dev);
    else
      k_path_persistent<2><<<pg, 128, 0, ctx->stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad,
                                                        next, ctx->err_dev);
    PF_CUDA(ctx, cudaGetLastError());
    k_path_accumulate<<<(unsigned)((n_pix + 127) / 128), 128, 0, ctx->stream>>>(rad, n_pix, kn, k0 == 0, k0 + kn >= spp,
                                                                                spp, acc, out_rgb_dev);
    PF_CUDA(ctx, cudaGetLastError());
  }
  return PF_OK;
}

// ---------------------------------------------------------------- allocation-free path tracer
// Scratch for pf_render_pathtraced_noalloc lives in this file-scope device
// array instead of the context arena: bytes [0, 256) hold the error word,
// then the per-pixel accumulator (12 B/pixel), then one chunk of per-sample
// slots (at least 12 B/pixel).  Every GPU that loads the library holds it
// until the process exits.
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)48 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

void put_msg(char* buf, int len, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
void put_msg(char* buf, int len, const char* fmt, ...) {
  if (!buf || len <= 0) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, (size_t)len, fmt, ap);
  va_end(ap);
}
}  // namespace

extern "C" pf_status pf_render_pathtraced_noalloc(const pf_volume* vol, const pf_light* lights, int n_lights, float g,
                                                  const pf_camera* cam, int spp, int max_bounces, uint64_t seed,
                                                  int use_rr, void* cuda_stream, float* out_rgb_dev, char* err_msg,
                                                  int err_len) {
  put_msg(err_msg, err_len, "%s", "");
  // argument checks: the same volume and light checks as the context entry
  // points (pf_check_volume / pf_check_lights), without a context
  if (pf_volume_problem(vol, err_msg, err_len > 0 ? (size_t)err_len : 0)) return PF_ERR_INVALID_ARG;
  if (!vol->brick_majorants_dev) {
    put_msg(err_msg, err_len, "volume->brick_majorants_dev must be set: this entry point does not compute it");
    return PF_ERR_INVALID_ARG;
  }
  if (pf_lights_problem(lights, n_lights, err_msg, err_len > 0 ? (size_t)err_len : 0)) return PF_ERR_INVALID_ARG;
  if (!cam || cam->width <= 0 || cam->height <= 0 || !(cam->fovy_deg > 0.f && cam->fovy_deg < 180.f) ||
      !cam_frame_ok(cam) || spp <= 0 ||
      spp > (1 << 24) || max_bounces < 1 || max_bounces > 1024 || !(g > -1.f && g < 1.f) || !out_rgb_dev) {
    put_msg(err_msg, err_len, "invalid camera, spp, max_bounces, g or output");
    return PF_ERR_INVALID_ARG;
  }
  const int64_t n_pix = (int64_t)cam->width * cam->height;
  const size_t acc_off = 256, per_pix = 3 * sizeof(float);
  const int64_t max_pix = (int64_t)((kNoAllocScratchBytes - 2 * acc_off) / (2 * per_pix));
  if (n_pix > max_pix) {
    put_msg(err_msg, err_len,
            "image of %lld pixels exceeds this entry point's static scratch (%zu bytes: at most %lld pixels)",
            (long long)n_pix, kNoAllocScratchBytes, (long long)max_pix);
    return PF_ERR_INVALID_ARG;
  }
  // once per device, with that device current: the array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    put_msg(err_msg, err_len, "no current CUDA device");
    return PF_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        put_msg(err_msg, err_len, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return PF_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    base = (unsigned char*)g_noalloc_addr[dev];
  }
  uint32_t* err_word = (uint32_t*)base;
  float* acc = (float*)(base + acc_off);
  size_t rad_off = (acc_off + (size_t)n_pix * per_pix + 255) / 256 * 256;
  float* rad = (float*)(base + rad_off);
  int64_t kc = (int64_t)((kNoAllocScratchBytes - rad_off) / ((size_t)n_pix * per_pix));
  kc = std::max<int64_t>(1, std::min<int64_t>(kc, spp));
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemsetAsync(err_word, 0, sizeof(uint32_t), stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    put_msg(err_msg, err_len, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  Vol V = pf_make_vol(vol, 0.f, vol->brick_majorants_dev);
  DevLights L = pf_make_lights(lights, n_lights);
  CamF C = make_cam(cam);
  for (int k0 = 0; k0 < spp; k0 += (int)kc) {
    int kn = (int)std::min<int64_t>(kc, spp - k0);
    int64_t n_items = n_pix * kn;
    dim3 grd((unsigned)((n_items + 127) / 128));
    if (vol->dtype == PF_F32)
      k_path_samples<0><<<grd, 128, 0, stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad, err_word, nullptr);
    else if (vol->dtype == PF_F16)
      k_path_samples<1><<<grd, 128, 0, stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad, err_word, nullptr);
    else
      k_path_samples<2><<<grd, 128, 0, stream>>>(V, L, C, g, spp, k0, kn, max_bounces, use_rr, seed, n_items, rad, err_word, nullptr);
    k_path_accumulate<<<(unsigned)((n_pix + 127) / 128), 128, 0, stream>>>(rad, n_pix, kn, k0 == 0, k0 + kn >= spp, spp,
                                                                           acc, out_rgb_dev);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    put_msg(err_msg, err_len, "launch: %s", cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  uint32_t w = 0;
  e = cudaMemcpyAsync(&w, err_word, sizeof(w), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    put_msg(err_msg, err_len, "%s", cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  if (w) {
    put_msg(err_msg, err_len, "a tracking loop hit its iteration limit (error word 0x%x)", w);
    return PF_ERR_TIMEOUT;
  }
  return PF_OK;
}
