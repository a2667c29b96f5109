// Device building blocks of the tracers: Philox4x32-10, the library's own
// float logarithm and sine/cosine, vector helpers, volume access, transfer
// function, Henyey-Greenstein phase function, delta and ratio tracking.
//
// Reproducibility contract.  Every translation unit that includes this file
// is compiled with -fmad=false and IEEE division and square root, so each
// float product and sum is a separately rounded IEEE operation.  Together
// with the own logarithm and sine/cosine below, the tracers compute the same
// float bits as any IEEE-754 implementation that evaluates the same
// expressions in the same order -- which is what lets photon bins, counts
// and path-tracer pixels be compared bit for bit with a reference.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cstring>
#include "../../include/pf.h"

namespace pfd {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11: ten rounds of the 4x32 S-box, multipliers 0xD2511F53 / 0xCD9E8D57,
// key bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
struct Rng {
  uint32_t k0, k1, c0, c1, c2, c3;
  __device__ __forceinline__ Rng(uint64_t seed, uint32_t tag, uint64_t item, uint32_t sub) {
    k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
    c0 = (uint32_t)item; c1 = (uint32_t)(item >> 32);
    c2 = (tag << 24) | (sub & 0xFFFFFFu); c3 = 0;
  }
  __device__ __forceinline__ void raw4(uint32_t o[4]) {
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, a = k0, b = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r > 0) { a += 0x9E3779B9u; b += 0xBB67AE85u; }
      uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
      uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
      uint32_t n0 = hi1 ^ x1 ^ a, n2 = hi0 ^ x3 ^ b;
      x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    o[0] = x0; o[1] = x1; o[2] = x2; o[3] = x3;
    c3 += 1;
  }
  // Four uniforms u = (x >> 8) * 2^-24 from the next block.
  __device__ __forceinline__ void uni4(float u[4]) {
    uint32_t o[4]; raw4(o);
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = (float)(o[i] >> 8) * 5.9604644775390625e-08f;
  }
};
enum { TAG_CAMERA = 1, TAG_PHOTON = 2, TAG_QUERY = 3, TAG_INIT = 4, TAG_SHADOW = 5 };
// Stream item of the shadow ray towards light l at interaction j of a camera
// sample (tag TAG_SHADOW, sub = sample index): every shadow ray draws from
// its own stream, so it can be traced apart from the sample's walk.
__device__ __forceinline__ uint64_t shadow_item(uint64_t pixel, int j, int l) {
  return pixel + ((uint64_t)(16 * (j - 1) + l) << 32);
}

// ------------------------------------------------------------------ own float math
// ln x: x = 2^e m, m folded into [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s) with
// s = (m-1)/(m+1) and the odd series to s^9; e ln2 added as a two-part
// (Cody-Waite) constant.  Valid for normal positive x.
__device__ __forceinline__ float own_lnf(float x) {
  uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  float p = 0.111111111f;
  p = p * s2 + 0.142857143f;
  p = p * s2 + 0.2f;
  p = p * s2 + 0.333333333f;
  p = p * s2;
  float r = s + s * p;
  r = r + r;
  float ef = (float)e;
  return ef * 0.693145752f + (ef * 1.42860677e-06f + r);
}

// sin(2 pi u), cos(2 pi u) for u in [0,1): exact octant reduction in turns,
// Taylor polynomials of sin (to a^9) and cos (to a^10) on [0, pi/4].
__device__ __forceinline__ void own_sincos2pif(float u, float* s_out, float* c_out) {
  float v = u * 8.0f;
  float fo = floorf(v);
  int o = (int)fo;
  float r = v - fo;
  int q = (o >> 1) & 3;
  float a = ((o & 1) ? (1.0f - r) : r) * 0.785398163f;
  float a2 = a * a;
  float ps = 2.75573192e-06f;
  ps = ps * a2 + -0.000198412698f;
  ps = ps * a2 + 0.00833333333f;
  ps = ps * a2 + -0.166666667f;
  float sa = a + (a * a2) * ps;
  float pc = -2.75573192e-07f;
  pc = pc * a2 + 2.48015873e-05f;
  pc = pc * a2 + -0.00138888889f;
  pc = pc * a2 + 0.0416666667f;
  pc = pc * a2 + -0.5f;
  float ca = 1.0f + a2 * pc;
  float sphi = (o & 1) ? ca : sa;
  float cphi = (o & 1) ? sa : ca;
  float s, c;
  if (q == 0) { s = sphi; c = cphi; }
  else if (q == 1) { s = cphi; c = -sphi; }
  else if (q == 2) { s = -sphi; c = -cphi; }
  else { s = -cphi; c = sphi; }
  *s_out = s; *c_out = c;
}

// atan2(y, x) in float32: the quotient t = min(|x|,|y|) / max(|x|,|y|) in
// [0, 1]; for t > tan(pi/8) the identity atan t = pi/4 + atan((t-1)/(t+1));
// one half-angle step atan t = 2 atan(t / (1 + sqrt(1 + t^2))) brings the
// argument below tan(pi/16); the odd Taylor series of atan to u^11
// (truncation < 1e-10); then the octant and quadrant fix-ups.  atan2(0, 0) = 0.
__device__ __forceinline__ float own_atan2f(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float hi = (ax < ay) ? ay : ax;
  const float lo = (ax < ay) ? ax : ay;
  if (!(hi > 0.0f)) return 0.0f;
  float t = lo / hi;
  const bool big = t > 0.414213562f;
  if (big) t = (t - 1.0f) / (t + 1.0f);
  const float u = t / (1.0f + sqrtf(1.0f + t * t));
  const float u2 = u * u;
  float p = -0.0909090909f;         // -1/11
  p = p * u2 + 0.111111111f;        // 1/9
  p = p * u2 + -0.142857143f;       // -1/7
  p = p * u2 + 0.2f;                // 1/5
  p = p * u2 + -0.333333333f;       // -1/3
  float r = u + u * (u2 * p);
  r = r + r;
  if (big) r = r + 0.785398163f;
  if (ax < ay) r = 1.57079633f - r;
  if (x < 0.0f) r = 3.14159265f - r;
  return (y < 0.0f) ? -r : r;
}

// The field's direction inputs (Sec. 3.1, normalised spherical coordinates)
// of an outgoing direction w: theta' = acos(w_z) / pi (acos as
// atan2(sqrt((1 - z)(1 + z)), z)), phi' = atan2(w_y, w_x) / 2pi mod 1.
__device__ __forceinline__ void query_angles(float wx, float wy, float wz, float* th, float* ph) {
  const float z = (wz < -1.0f) ? -1.0f : ((wz > 1.0f) ? 1.0f : wz);
  *th = own_atan2f(sqrtf((1.0f - z) * (1.0f + z)), z) * 0.318309886f;
  float p = own_atan2f(wy, wx) * 0.159154943f;
  if (p < 0.0f) p = p + 1.0f;
  *ph = p;
}

// min / max with the semantics of std::min / std::max (first argument on ties)
__device__ __forceinline__ float mn(float a, float b) { return (b < a) ? b : a; }
__device__ __forceinline__ float mx(float a, float b) { return (a < b) ? b : a; }

// ------------------------------------------------------------------ vectors
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float a, float b, float c) { V3 r; r.x = a; r.y = b; r.z = c; return r; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 normalize(V3 a) {
  float inv = 1.0f / sqrtf(dot(a, a));
  return v3(a.x * inv, a.y * inv, a.z * inv);
}
__device__ __forceinline__ V3 along(V3 o, V3 d, float t) { return v3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z); }

// Orthonormal basis around unit n (Duff et al., "Building an Orthonormal
// Basis, Revisited", JCGT 2017).
__device__ __forceinline__ void onb(V3 n, V3* b1, V3* b2) {
  float sign = copysignf(1.0f, n.z);
  float a = -1.0f / (sign + n.z);
  float b = n.x * n.y * a;
  *b1 = v3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *b2 = v3(b, sign + n.y * n.y * a, -n.y);
}

// ------------------------------------------------------------------ volume
struct Vol {
  const void* data;
  int nx, ny, nz, dtype;
  float sigma_scale, albedo, majorant;
  const float4* tf;   // RGBA rows
  int tf_n;
  const float* mg;    // brick majorants (x fastest)
  int gx, gy, gz, B;  // brick grid and brick edge (voxels)
  const float* mgw;   // the same majorants with a border of kBorder zero bricks on every side (the walks' copy)
  int pgx, pgy;       // its extent along x and y (gx + 2 kBorder, gy + 2 kBorder)
  float wx, wy, wz;   // brick edge in world units, B / n (IEEE division)
  const void* tiled;  // voxels in 4x4x4 tiles (same values), or null
  int tnx, tny;       // tiles along x and y
  int off32;          // element offsets of the layout in use fit 32 bits
};

// Element offset of voxel (i, j, k) = X(i) + Y(j) + Z(k) in either layout:
// x-fastest (X = i, Y = nx j, Z = nx ny k) or 4x4x4 tiles with z-slices of
// 16 consecutive elements (X = 64 (i>>2) + (i&3), Y = 64 tnx (j>>2) + 4 (j&3),
// Z = 64 tnx tny (k>>2) + 16 (k&3)).
__device__ __forceinline__ size_t offx(const Vol& V, int i) {
  return V.tiled ? (size_t)(i >> 2) * 64 + (size_t)(i & 3) : (size_t)i;
}
__device__ __forceinline__ size_t offy(const Vol& V, int j) {
  return V.tiled ? (size_t)(j >> 2) * (size_t)V.tnx * 64 + (size_t)((j & 3) * 4) : (size_t)j * (size_t)V.nx;
}
__device__ __forceinline__ size_t offz(const Vol& V, int k) {
  return V.tiled ? (size_t)(k >> 2) * (size_t)V.tnx * (size_t)V.tny * 64 + (size_t)((k & 3) * 16)
                 : (size_t)k * (size_t)V.nx * (size_t)V.ny;
}
__device__ __forceinline__ uint32_t offx32(const Vol& V, int i) {
  return V.tiled ? ((uint32_t)(i >> 2) << 6) + (uint32_t)(i & 3) : (uint32_t)i;
}
__device__ __forceinline__ uint32_t offy32(const Vol& V, int j) {
  return V.tiled ? (uint32_t)(j >> 2) * ((uint32_t)V.tnx << 6) + (uint32_t)((j & 3) * 4) : (uint32_t)j * (uint32_t)V.nx;
}
__device__ __forceinline__ uint32_t offz32(const Vol& V, int k) {
  return V.tiled ? (uint32_t)(k >> 2) * ((uint32_t)V.tnx * (uint32_t)V.tny << 6) + (uint32_t)((k & 3) * 16)
                 : (uint32_t)k * ((uint32_t)V.nx * (uint32_t)V.ny);
}
template <int DT> __device__ __forceinline__ float voxel_at(const void* base, size_t idx) {
  if (DT == 0) return __ldg((const float*)base + idx);
  if (DT == 1) return __half2float(__ldg((const __half*)base + idx));
  return (float)__ldg((const uint8_t*)base + idx) / 255.0f;
}
template <int DT> __device__ __forceinline__ float voxel(const Vol& V, int i, int j, int k) {
  return voxel_at<DT>(V.tiled ? V.tiled : V.data, offx(V, i) + offy(V, j) + offz(V, k));
}

// Trilinear density; x, then y, then z lerps, each a + t*(b - a).
template <int DT> __device__ __forceinline__ float density(const Vol& V, V3 p) {
  if (!(p.x >= 0.0f && p.x <= 1.0f && p.y >= 0.0f && p.y <= 1.0f && p.z >= 0.0f && p.z <= 1.0f)) return 0.0f;
  float fx = p.x * (float)V.nx - 0.5f, fy = p.y * (float)V.ny - 0.5f, fz = p.z * (float)V.nz - 0.5f;
  float ix = floorf(fx), iy = floorf(fy), iz = floorf(fz);
  float tx = fx - ix, ty = fy - iy, tz = fz - iz;
  int x0 = (int)ix, y0 = (int)iy, z0 = (int)iz;
  int x1 = min(x0 + 1, V.nx - 1), y1 = min(y0 + 1, V.ny - 1), z1 = min(z0 + 1, V.nz - 1);
  x0 = max(x0, 0); y0 = max(y0, 0); z0 = max(z0, 0);
  // the layout decided once per lookup; the eight loads then issue together
  const void* base = V.tiled ? V.tiled : V.data;
  float v000, v100, v010, v110, v001, v101, v011, v111;
  if (V.off32) {  // 32-bit offset arithmetic (volumes below 2^32 elements)
    const uint32_t ax0 = offx32(V, x0), ax1 = offx32(V, x1), ay0 = offy32(V, y0), ay1 = offy32(V, y1);
    const uint32_t az0 = offz32(V, z0), az1 = offz32(V, z1);
    v000 = voxel_at<DT>(base, ax0 + ay0 + az0); v100 = voxel_at<DT>(base, ax1 + ay0 + az0);
    v010 = voxel_at<DT>(base, ax0 + ay1 + az0); v110 = voxel_at<DT>(base, ax1 + ay1 + az0);
    v001 = voxel_at<DT>(base, ax0 + ay0 + az1); v101 = voxel_at<DT>(base, ax1 + ay0 + az1);
    v011 = voxel_at<DT>(base, ax0 + ay1 + az1); v111 = voxel_at<DT>(base, ax1 + ay1 + az1);
  } else {
    const size_t ax0 = offx(V, x0), ax1 = offx(V, x1), ay0 = offy(V, y0), ay1 = offy(V, y1);
    const size_t az0 = offz(V, z0), az1 = offz(V, z1);
    v000 = voxel_at<DT>(base, ax0 + ay0 + az0); v100 = voxel_at<DT>(base, ax1 + ay0 + az0);
    v010 = voxel_at<DT>(base, ax0 + ay1 + az0); v110 = voxel_at<DT>(base, ax1 + ay1 + az0);
    v001 = voxel_at<DT>(base, ax0 + ay0 + az1); v101 = voxel_at<DT>(base, ax1 + ay0 + az1);
    v011 = voxel_at<DT>(base, ax0 + ay1 + az1); v111 = voxel_at<DT>(base, ax1 + ay1 + az1);
  }
  float c00 = v000 + tx * (v100 - v000);
  float c10 = v010 + tx * (v110 - v010);
  float c01 = v001 + tx * (v101 - v001);
  float c11 = v011 + tx * (v111 - v011);
  float c0 = c00 + ty * (c10 - c00);
  float c1 = c01 + ty * (c11 - c01);
  return c0 + tz * (c1 - c0);
}

// Transfer-function row lookup: returns lerped RGBA at density d.
__device__ __forceinline__ void tf_pos(const Vol& V, float d, int* i_out, float* f_out) {
  if (d < 0.0f) d = 0.0f;
  if (d > 1.0f) d = 1.0f;
  float s = d * (float)(V.tf_n - 1);
  int i = (int)floorf(s);
  if (i > V.tf_n - 2) i = V.tf_n - 2;
  *i_out = i;
  *f_out = s - (float)i;
}
__device__ __forceinline__ float tf_alpha(const Vol& V, float d) {
  int i; float f; tf_pos(V, d, &i, &f);
  float a = __ldg(&V.tf[i].w), b = __ldg(&V.tf[i + 1].w);
  return a + f * (b - a);
}
template <int DT> __device__ __forceinline__ float sigma_at(const Vol& V, V3 p) {
  return V.sigma_scale * tf_alpha(V, density<DT>(V, p));
}
template <int DT> __device__ __forceinline__ void medium_at(const Vol& V, V3 p, float* sigma, V3* alb) {
  float d = density<DT>(V, p);
  int i; float f; tf_pos(V, d, &i, &f);
  float4 a = __ldg(&V.tf[i]), b = __ldg(&V.tf[i + 1]);
  *sigma = V.sigma_scale * (a.w + f * (b.w - a.w));
  *alb = v3(V.albedo * (a.x + f * (b.x - a.x)), V.albedo * (a.y + f * (b.y - a.y)), V.albedo * (a.z + f * (b.z - a.z)));
}

// Ray / unit-box slab test; t range clipped to t >= 0.
__device__ __forceinline__ bool box_hit(V3 o, V3 d, float* t0, float* t1) {
  float lo = 0.0f, hi = __int_as_float(0x7f800000);
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0f) {
      if (oo[a] < 0.0f || oo[a] > 1.0f) return false;
      continue;
    }
    float ta = (0.0f - oo[a]) / dd[a], tb = (1.0f - oo[a]) / dd[a];
    float tn = mn(ta, tb), tf = mx(ta, tb);
    lo = mx(lo, tn);
    hi = mn(hi, tf);
  }
  *t0 = lo; *t1 = hi;
  return lo < hi;
}

// ------------------------------------------------------------------ phase function
// Henyey-Greenstein; mu = cosine between incoming and outgoing travel
// directions (g > 0 forward).
__device__ __forceinline__ float hg_eval(float g, float mu) {
  float gg = g * g;
  float den = 1.0f + gg - 2.0f * g * mu;
  return 0.0795774715459476678f * (1.0f - gg) / (den * sqrtf(den));
}
// Inverse-CDF sampling of HG about the travel direction d.
__device__ __forceinline__ V3 hg_sample(float g, V3 d, float xi1, float xi2) {
  float mu;
  if (fabsf(g) < 1e-3f) mu = 1.0f - 2.0f * xi1;
  else {
    float gg = g * g;
    float tmp = (1.0f - gg) / (1.0f - g + 2.0f * g * xi1);
    mu = (1.0f + gg - tmp * tmp) / (2.0f * g);
  }
  if (mu < -1.0f) mu = -1.0f;
  if (mu > 1.0f) mu = 1.0f;
  float st = sqrtf(mx(0.0f, 1.0f - mu * mu));
  float sp, cp;
  own_sincos2pif(xi2, &sp, &cp);
  V3 e1, e2;
  onb(d, &e1, &e2);
  float a = st * cp, b = st * sp;
  V3 nd = v3(e1.x * a + e2.x * b + d.x * mu, e1.y * a + e2.y * b + d.y * mu, e1.z * a + e2.z * b + d.z * mu);
  return normalize(nd);
}

// ------------------------------------------------------------------ tracking
// Iteration limit of every tracking loop; exceeding it sets PFE_ITER_CAP.
constexpr int kMaxTrackSteps = 1 << 24;

// Walk over the bricks a ray crosses (Amanatides-Woo).  Per axis: brick
// width w = B / n, inverse direction inv = 1/d; the first plane parameter is
// (plane - o) * inv and each further plane adds w * |inv| (register-only,
// no division per crossing).  Plane rounding stays far below the half-voxel
// margin of the brick majorants.  The walk keeps the linear brick index and
// loads the majorant of the next brick one crossing ahead so that the load's
// latency overlaps the work in the current brick.
//
// G: the walk reads V.mgw, the majorants with a border of kBorder = 2 zero
// bricks.  A ray inside the box ends (t >= t_end, at most the box exit)
// within rounding of where it leaves the grid, far less than a brick's width
// in t, so past the grid it enters at most the first border layer (once per
// axis, near an edge or corner), whose majorant 0 holds no tentative
// collision and leaves the budget unchanged: no crossing counts are needed.
// The next brick's majorant is loaded one crossing ahead, from the second
// layer at most.  !G: the walk reads
// V.mg and counts the crossings left per axis, ending where the grid ends
// (for callers that cannot allocate the bordered copy).  Both take the same
// float steps and give the same results.
constexpr int kBorder = 2;   // zero bricks around the walks' copy of the brick grid
template <bool G>
struct Walk {
  float tx, ty, tz, dtx, dty, dtz;
  int lx, ly, lz;  // !G: crossings left along each axis before the ray leaves the grid
  int ox, oy, oz;  // linear-index offset of a crossing along each axis
  int idx, na;     // current brick, axis of the next crossing
  int noff;        // linear-index offset of the next crossing (axis na)
  bool more;       // !G: the next crossing stays inside the grid
  float m, m_next; // majorants of the current and the next brick
  float t_exit;    // plane parameter of the next crossing (the current brick's exit)
  __device__ __forceinline__ static float load(const Vol& V, int i) { return __ldg((G ? V.mgw : V.mg) + i); }
  __device__ __forceinline__ static void axis(float o, float d, float t, float w, int g, int stride, int& c, int& l,
                                              int& off, float& tn, float& dt) {
    const float p = o + t * d;
    const int ci = (int)floorf(p / w);
    c = min(max(ci, 0), g - 1);
    if (d > 0.0f) {
      const float inv = 1.0f / d;
      l = g - 1 - c; off = stride; tn = ((float)(c + 1) * w - o) * inv; dt = w * inv;
    } else if (d < 0.0f) {
      const float inv = 1.0f / d;
      l = c; off = -stride; tn = ((float)c * w - o) * inv; dt = -(w * inv);
    } else {
      l = 0; off = 0; tn = __int_as_float(0x7f800000); dt = tn;
    }
  }
  // the next crossing: its axis, exit parameter, offset and majorant, chosen
  // once per brick (the step and the caller's exit test reuse them)
  __device__ __forceinline__ void plan(const Vol& V) {
    const bool bx = tx <= ty && tx <= tz, by = !bx && ty <= tz;
    na = bx ? 0 : (by ? 1 : 2);
    noff = bx ? ox : (by ? oy : oz);
    t_exit = bx ? tx : (by ? ty : tz);
    if (G) {
      m_next = load(V, idx + noff);
    } else {
      const int left = bx ? lx : (by ? ly : lz);
      more = left > 0;
      m_next = more ? load(V, idx + noff) : 0.0f;
    }
  }
  __device__ __forceinline__ void init(const Vol& V, V3 o, V3 d, float t) {
    int cx, cy, cz;
    const int sy = G ? V.pgx : V.gx, sz = G ? V.pgx * V.pgy : V.gx * V.gy;
    axis(o.x, d.x, t, V.wx, V.gx, 1, cx, lx, ox, tx, dtx);
    axis(o.y, d.y, t, V.wy, V.gy, sy, cy, ly, oy, ty, dty);
    axis(o.z, d.z, t, V.wz, V.gz, sz, cz, lz, oz, tz, dtz);
    idx = G ? (cx + kBorder) + sy * (cy + kBorder) + sz * (cz + kBorder) : cx + sy * cy + sz * cz;
    m = load(V, idx);
    plan(V);
  }
  __device__ __forceinline__ float exit_t() const { return t_exit; }
  // step into the next brick (branch-free selects); false when the ray
  // leaves the grid (!G only)
  __device__ __forceinline__ bool step(const Vol& V) {
    if (!G && !more) return false;
    const bool ax = na == 0, ay = na == 1, az = na == 2;
    if (!G) { lx -= (int)ax; ly -= (int)ay; lz -= (int)az; }
    idx += noff;
    const float sx = tx + dtx, sy = ty + dty, sz = tz + dtz;
    tx = ax ? sx : tx; ty = ay ? sy : ty; tz = az ? sz : tz;
    m = m_next;
    plan(V);
    return true;
  }
};

// Uniforms of one tracking call, taken one at a time from the caller's
// stream, four per Philox block in lane order; the rest of the last block is
// discarded when the call returns.
struct Uniforms {
  float q0, q1, q2, q3;
  int n = 0;
  __device__ __forceinline__ float next(Rng& rng) {
    if (n == 0) {
      float u[4]; rng.uni4(u);
      q0 = u[0]; q1 = u[1]; q2 = u[2]; q3 = u[3]; n = 4;
    }
    const float v = q0;
    q0 = q1; q1 = q2; q2 = q3; --n;
    return v;
  }
};

// Delta (Woodcock) tracking in [t, t_end) over the brick majorants.
// Uniforms in order: the optical-depth budget tau = -ln(1-u) of the next
// tentative collision, spent brick by brick; at a tentative collision one
// uniform accepts it with probability sigma_t / majorant, then the next
// budget.  Returns true on a real collision.  `fetches` counts density
// lookups (the tracers' unit of memory work).
//
// The loop is nested: the inner loop crosses bricks until the budget runs
// out inside one, then the lookup follows.  Lanes of a warp thus reach their
// (expensive) lookups together instead of alternating lookups and
// (cheap) brick crossings.  Every lane performs the same float operations
// in the same order as a flat event loop would.
template <int DT, bool G = true>
__device__ __forceinline__ bool delta_track(const Vol& V, V3 o, V3 d, float t, float t_end, Rng& rng, float* t_hit,
                                            uint32_t* err, uint32_t& fetches) {
  Walk<G> W;
  W.init(V, o, d, t);
  Uniforms U;
  float tau = -own_lnf(1.0f - U.next(rng));
  float tc = mn(W.exit_t(), t_end);
  int it = 0;
  for (;;) {
    float seg = tc - t;
    if (seg < 0.0f) seg = 0.0f;
    while (!(tau < W.m * seg)) {          // tau >= 0: a brick of majorant 0 is crossed
      tau = tau - W.m * seg;
      t = tc;
      if (t >= t_end) return false;
      if (!W.step(V)) return false;
      tc = mn(W.exit_t(), t_end);
      seg = tc - t;
      if (seg < 0.0f) seg = 0.0f;
      if (++it >= kMaxTrackSteps) { atomicOr(err, 1u); return false; }
    }
    const float m = W.m;
    t = t + tau / m;
    ++fetches;
    const float ua = U.next(rng);
    if (ua * m < sigma_at<DT>(V, along(o, d, t))) { *t_hit = t; return true; }
    tau = -own_lnf(1.0f - U.next(rng));
    if (++it >= kMaxTrackSteps) { atomicOr(err, 1u); return false; }
  }
}

// Ratio-tracking transmittance over [0, t_end) with the brick majorants: at
// each tentative collision T *= max(0, 1 - sigma_t / majorant); one uniform
// per tentative collision (its budget).  Same nested loop as delta_track.
template <int DT, bool G = true>
__device__ __forceinline__ float ratio_track(const Vol& V, V3 o, V3 d, float t_end, Rng& rng, uint32_t* err,
                                             uint32_t& fetches) {
  Walk<G> W;
  W.init(V, o, d, 0.0f);
  Uniforms U;
  float T = 1.0f, t = 0.0f;
  float tau = -own_lnf(1.0f - U.next(rng));
  float tc = mn(W.exit_t(), t_end);
  int it = 0;
  for (;;) {
    float seg = tc - t;
    if (seg < 0.0f) seg = 0.0f;
    while (!(tau < W.m * seg)) {          // tau >= 0: a brick of majorant 0 is crossed
      tau = tau - W.m * seg;
      t = tc;
      if (t >= t_end) return T;
      if (!W.step(V)) return T;
      tc = mn(W.exit_t(), t_end);
      seg = tc - t;
      if (seg < 0.0f) seg = 0.0f;
      if (++it >= kMaxTrackSteps) { atomicOr(err, 1u); return T; }
    }
    const float m = W.m;
    t = t + tau / m;
    ++fetches;
    const float f = 1.0f - sigma_at<DT>(V, along(o, d, t)) / m;
    T = T * mx(0.0f, f);
    tau = -own_lnf(1.0f - U.next(rng));
    if (++it >= kMaxTrackSteps) { atomicOr(err, 1u); return T; }
  }
}

// Largest TF alpha over densities [dmin, dmax] (piecewise-linear table).
__device__ __forceinline__ float tf_alpha_max(const Vol& V, float dmin, float dmax) {
  if (dmin < 0.0f) dmin = 0.0f;
  if (dmax > 1.0f) dmax = 1.0f;
  float a = mx(tf_alpha(V, dmin), tf_alpha(V, dmax));
  for (int i = 0; i < V.tf_n; ++i) {
    const float nd = (float)i / (float)(V.tf_n - 1);
    const float ai = __ldg(&V.tf[i].w);
    if (nd >= dmin && nd <= dmax && ai > a) a = ai;
  }
  return a;
}

// ------------------------------------------------------------------ lights and camera
struct DevLight { int kind; float v[3]; float rgb[3]; };
struct DevLights { DevLight l[16]; int n; };

__device__ __forceinline__ void light_geom(const DevLight& L, V3 x, V3* wl, float* dist, V3* E) {
  if (L.kind == 0) {
    *wl = normalize(v3(L.v[0], L.v[1], L.v[2]));
    *dist = __int_as_float(0x7f800000);
    *E = v3(L.rgb[0], L.rgb[1], L.rgb[2]);
  } else {
    V3 dv = v3(L.v[0] - x.x, L.v[1] - x.y, L.v[2] - x.z);
    float d2 = dot(dv, dv);
    float dl = sqrtf(d2);
    float inv = 1.0f / dl;
    *wl = v3(dv.x * inv, dv.y * inv, dv.z * inv);
    *dist = dl;
    *E = v3(L.rgb[0] / d2, L.rgb[1] / d2, L.rgb[2] / d2);
  }
}

// Camera frame: rounded once from the host's double-precision frame.
struct CamF { float eye[3], f[3], r[3], u[3]; float sx, sy; int W, H; };

__device__ __forceinline__ void camera_ray(const CamF& c, int px, int py, float j1, float j2, V3* o, V3* d) {
  float a = (2.0f * ((float)px + j1) / (float)c.W - 1.0f) * c.sx;
  float b = (1.0f - 2.0f * ((float)py + j2) / (float)c.H) * c.sy;
  V3 dir = v3(c.f[0] + a * c.r[0] + b * c.u[0], c.f[1] + a * c.r[1] + b * c.u[1], c.f[2] + a * c.r[2] + b * c.u[2]);
  *d = normalize(dir);
  *o = v3(c.eye[0], c.eye[1], c.eye[2]);
}

}  // namespace pfd

// Host-side packing of the public scene structs into the kernels' views.
// brick_edge: edge of the bricks of `grid` (0: the volume's brick).
inline pfd::Vol pf_make_vol(const pf_volume* v, float majorant, const float* grid = nullptr, int brick_edge = 0) {
  const int B = brick_edge > 0 ? brick_edge : (v->brick > 0 ? v->brick : 8);
  pfd::Vol V;
  V.data = v->data_dev; V.nx = v->nx; V.ny = v->ny; V.nz = v->nz; V.dtype = v->dtype;
  V.sigma_scale = v->sigma_scale; V.albedo = v->albedo; V.majorant = majorant;
  V.tf = (const float4*)v->tf_lut_dev; V.tf_n = v->tf_n;
  V.mg = grid;
  V.mgw = nullptr;
  V.B = B;
  V.gx = (v->nx + B - 1) / B;
  V.gy = (v->ny + B - 1) / B;
  V.gz = (v->nz + B - 1) / B;
  V.pgx = V.gx + 2 * pfd::kBorder;
  V.pgy = V.gy + 2 * pfd::kBorder;
  V.wx = (float)B / (float)v->nx;
  V.wy = (float)B / (float)v->ny;
  V.wz = (float)B / (float)v->nz;
  V.tiled = v->tiled_dev;
  V.tnx = (v->nx + 3) / 4;
  V.tny = (v->ny + 3) / 4;
  const uint64_t elems = v->tiled_dev ? (uint64_t)V.tnx * (uint64_t)V.tny * (uint64_t)((v->nz + 3) / 4) * 64u
                                      : (uint64_t)v->nx * (uint64_t)v->ny * (uint64_t)v->nz;
  V.off32 = elems <= 0xffffffffull ? 1 : 0;
  return V;
}
inline pfd::DevLights pf_make_lights(const pf_light* lights, int n) {
  pfd::DevLights L;
  std::memset(&L, 0, sizeof(L));
  L.n = n;
  for (int i = 0; i < n; ++i) {
    L.l[i].kind = lights[i].kind;
    for (int c = 0; c < 3; ++c) { L.l[i].v[c] = lights[i].v[c]; L.l[i].rgb[c] = lights[i].rgb[c]; }
  }
  return L;
}
