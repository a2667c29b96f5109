// Photon Field Networks (arXiv 2304.07338) -- CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA path is checked against.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load it.  It shares no code with the CUDA
// library: every routine below is written from the paper and from the
// published definitions it names.
//
// Precision.  Every stochastic tracer is a template over the real type R.
//   R = double : the FP64 reference, pinned by the closed-form tests.
//   R = float  : the same steps in IEEE binary32 with no contraction
//                (compiled with -ffp-contract=off) and the project's own
//                logarithm and sine/cosine (below).  Delta tracking, Russian
//                roulette and photon binning take integer decisions from
//                floating-point comparisons; this instantiation takes them in
//                the kernel's precision, so bins and counts can be compared
//                bit for bit.
//
// Random numbers.  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11).  Key = (seed_lo, seed_hi); counter =
// (item_lo, item_hi, tag << 24 | sub, block).  One call yields four uniforms
// u = (x >> 8) * 2^-24 and advances `block` by one.
//   tag 1 CAMERA  item = pixel index, sub = sample index
//   tag 2 PHOTON  item = photon id,   sub = 0
//   tag 3 QUERY   item = query index, sub = training step
//   tag 4 INIT    item = layer,       sub = 0, block = element / 4
//
// Scene conventions (shared with the input generator): volume x-fastest,
// voxel centres at (i+1/2)/n, trilinear with clamp-to-edge inside [0,1]^3 and
// zero outside; transfer function = linear RGBA table over density [0,1];
// sigma_t = sigma_scale * alpha, albedo = A * rgb.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>
#include <type_traits>

namespace {

// ------------------------------------------------------------------ Philox
inline uint32_t mulhi32(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

void philox4x32_10(const uint32_t key_in[2], const uint32_t ctr_in[4], uint32_t out[4]) {
    // Ten rounds of the Philox-4x32 S-box with the published multipliers and
    // Weyl key increments.
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t lo0 = M0 * c0, hi0 = mulhi32(M0, c0);
        uint32_t lo1 = M1 * c2, hi1 = mulhi32(M1, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

struct Rng {
    uint32_t key[2];
    uint32_t ctr[4];
    Rng(uint64_t seed, uint32_t tag, uint64_t item, uint32_t sub) {
        key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
        ctr[0] = (uint32_t)item; ctr[1] = (uint32_t)(item >> 32);
        ctr[2] = (tag << 24) | (sub & 0xFFFFFFu); ctr[3] = 0;
    }
    // Four raw 32-bit words from the next block.
    void raw4(uint32_t o[4]) { philox4x32_10(key, ctr, o); ctr[3] += 1; }
    template <typename R> void uni4(R u[4]) {
        uint32_t o[4]; raw4(o);
        for (int i = 0; i < 4; ++i) u[i] = (R)(o[i] >> 8) * (R)(1.0 / 16777216.0);
    }
};

// ------------------------------------------------------------------ own FP32 math
// Natural logarithm, written from the textbook method: split x = 2^e * m with
// m in [sqrt(1/2), sqrt(2)), then ln m = 2 atanh(s), s = (m-1)/(m+1), summed
// as the odd series s + s^3/3 + ... + s^9/9 (truncation < 1e-9 for |s|<0.172),
// and e*ln2 added in two parts (Cody-Waite split of ln 2).
float own_lnf(float x) {
    uint32_t b; std::memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    float m; std::memcpy(&m, &mb, 4);
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 0.111111111f;           // 1/9
    p = p * s2 + 0.142857143f;        // 1/7
    p = p * s2 + 0.2f;                // 1/5
    p = p * s2 + 0.333333333f;        // 1/3
    p = p * s2;
    float r = s + s * p;
    r = r + r;
    float ef = (float)e;
    return ef * 0.693145752f + (ef * 1.42860677e-06f + r);
}

// sin and cos of 2*pi*u for u in [0,1): octant reduction done exactly in
// turns, then Taylor polynomials of sin (to a^9) and cos (to a^10) on
// [0, pi/4] (truncation below 2e-9).
void own_sincos2pif(float u, float* s_out, float* c_out) {
    float v = u * 8.0f;
    float fo = std::floor(v);
    int o = (int)fo;
    float r = v - fo;
    int q = (o >> 1) & 3;
    float a = ((o & 1) ? (1.0f - r) : r) * 0.785398163f;
    float a2 = a * a;
    float ps = 2.75573192e-06f;           // 1/9!
    ps = ps * a2 + -0.000198412698f;      // -1/7!
    ps = ps * a2 + 0.00833333333f;        // 1/5!
    ps = ps * a2 + -0.166666667f;         // -1/3!
    float sa = a + (a * a2) * ps;
    float pc = -2.75573192e-07f;          // -1/10!
    pc = pc * a2 + 2.48015873e-05f;       // 1/8!
    pc = pc * a2 + -0.00138888889f;       // -1/6!
    pc = pc * a2 + 0.0416666667f;         // 1/4!
    pc = pc * a2 + -0.5f;                 // -1/2!
    float ca = 1.0f + a2 * pc;
    float sphi, cphi;
    if (o & 1) { sphi = ca; cphi = sa; } else { sphi = sa; cphi = ca; }
    float s, c;
    switch (q) {
        case 0: s = sphi; c = cphi; break;
        case 1: s = cphi; c = -sphi; break;
        case 2: s = -sphi; c = -cphi; break;
        default: s = -cphi; c = sphi; break;
    }
    *s_out = s; *c_out = c;
}

// atan2(y, x) in float32, from the textbook reductions: t = min/max of |x|,
// |y| in [0, 1]; above tan(pi/8) use atan t = pi/4 + atan((t-1)/(t+1)); one
// half-angle step atan t = 2 atan(t / (1 + sqrt(1 + t^2))); the odd Taylor
// series of atan up to u^11; octant and quadrant fix-ups.  atan2(0, 0) = 0.
float own_atan2f(float y, float x) {
    const float ax = std::fabs(x), ay = std::fabs(y);
    const float hi = (ax < ay) ? ay : ax;
    const float lo = (ax < ay) ? ax : ay;
    if (!(hi > 0.0f)) return 0.0f;
    float t = lo / hi;
    const bool big = t > 0.414213562f;
    if (big) t = (t - 1.0f) / (t + 1.0f);
    const float u = t / (1.0f + std::sqrt(1.0f + t * t));
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

// The field's direction inputs in float32 (the renderer's precision):
// theta' = acos(w_z)/pi with acos z = atan2(sqrt((1-z)(1+z)), z), and
// phi' = atan2(w_y, w_x)/(2 pi), wrapped into [0, 1).
void query_angles_f32(float wx, float wy, float wz, float* th, float* ph) {
    const float z = (wz < -1.0f) ? -1.0f : ((wz > 1.0f) ? 1.0f : wz);
    *th = own_atan2f(std::sqrt((1.0f - z) * (1.0f + z)), z) * 0.318309886f;
    float p = own_atan2f(wy, wx) * 0.159154943f;
    if (p < 0.0f) p = p + 1.0f;
    *ph = p;
}

template <typename R> struct M;
template <> struct M<double> {
    static double ln(double x) { return std::log(x); }
    static void sincos2pi(double u, double* s, double* c) {
        double a = 2.0 * M_PI * u; *s = std::sin(a); *c = std::cos(a);
    }
    static double sqrt_(double x) { return std::sqrt(x); }
};
template <> struct M<float> {
    static float ln(float x) { return own_lnf(x); }
    static void sincos2pi(float u, float* s, float* c) { own_sincos2pif(u, s, c); }
    static float sqrt_(float x) { return std::sqrt(x); }
};

// ------------------------------------------------------------------ vectors
template <typename R> struct V3 { R x, y, z; };
template <typename R> inline V3<R> v3(R a, R b, R c) { return V3<R>{a, b, c}; }
template <typename R> inline V3<R> sub(V3<R> a, V3<R> b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename R> inline V3<R> scl(V3<R> a, R s) { return v3(a.x * s, a.y * s, a.z * s); }
template <typename R> inline R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> inline V3<R> normalize(V3<R> a) {
    R inv = (R)1 / M<R>::sqrt_(dot(a, a));
    return v3(a.x * inv, a.y * inv, a.z * inv);
}
// point along a ray: o + t*d, component-wise
template <typename R> inline V3<R> along(V3<R> o, V3<R> d, R t) { return v3(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z); }

// Orthonormal basis around unit n (Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin, "Building an Orthonormal Basis, Revisited", JCGT 2017).
template <typename R> void onb(V3<R> n, V3<R>* b1, V3<R>* b2) {
    R sign = std::copysign((R)1, n.z);
    R a = (R)-1 / (sign + n.z);
    R b = n.x * n.y * a;
    *b1 = v3((R)1 + sign * n.x * n.x * a, sign * b, -sign * n.x);
    *b2 = v3(b, sign + n.y * n.y * a, -n.y);
}

// ------------------------------------------------------------------ scene
struct Volume {
    int nx, ny, nz, dtype;          // dtype 0 f32, 1 f16 bits, 2 u8
    const void* data;
    double sigma_scale, albedo;
    const float* tf; int tf_n;      // RGBA rows
};

struct Light { int kind; double v[3]; double rgb[3]; };

double half_bits_to_double(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = std::ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = std::ldexp((double)(m + 1024), e - 25);
    return s ? -v : v;
}

template <typename R> R voxel(const Volume& V, int i, int j, int k) {
    size_t idx = (size_t)i + (size_t)V.nx * ((size_t)j + (size_t)V.ny * (size_t)k);
    if (V.dtype == 0) return (R)((const float*)V.data)[idx];
    if (V.dtype == 1) return (R)half_bits_to_double(((const uint16_t*)V.data)[idx]);
    return (R)((const uint8_t*)V.data)[idx] / (R)255;
}

// Trilinear density at p; x, then y, then z lerps, each a + t*(b - a).
template <typename R> R density(const Volume& V, V3<R> p) {
    if (!(p.x >= (R)0 && p.x <= (R)1 && p.y >= (R)0 && p.y <= (R)1 && p.z >= (R)0 && p.z <= (R)1)) return (R)0;
    R fx = p.x * (R)V.nx - (R)0.5, fy = p.y * (R)V.ny - (R)0.5, fz = p.z * (R)V.nz - (R)0.5;
    R ix = std::floor(fx), iy = std::floor(fy), iz = std::floor(fz);
    R tx = fx - ix, ty = fy - iy, tz = fz - iz;
    int x0 = (int)ix, y0 = (int)iy, z0 = (int)iz;
    int x1 = std::min(x0 + 1, V.nx - 1), y1 = std::min(y0 + 1, V.ny - 1), z1 = std::min(z0 + 1, V.nz - 1);
    x0 = std::max(x0, 0); y0 = std::max(y0, 0); z0 = std::max(z0, 0);
    R v000 = voxel<R>(V, x0, y0, z0), v100 = voxel<R>(V, x1, y0, z0);
    R v010 = voxel<R>(V, x0, y1, z0), v110 = voxel<R>(V, x1, y1, z0);
    R v001 = voxel<R>(V, x0, y0, z1), v101 = voxel<R>(V, x1, y0, z1);
    R v011 = voxel<R>(V, x0, y1, z1), v111 = voxel<R>(V, x1, y1, z1);
    R c00 = v000 + tx * (v100 - v000);
    R c10 = v010 + tx * (v110 - v010);
    R c01 = v001 + tx * (v101 - v001);
    R c11 = v011 + tx * (v111 - v011);
    R c0 = c00 + ty * (c10 - c00);
    R c1 = c01 + ty * (c11 - c01);
    return c0 + tz * (c1 - c0);
}

// Transfer function entry c (0..3) at density d (clamped to [0,1]).
template <typename R> R tf_at(const Volume& V, R d, int c) {
    if (d < (R)0) d = (R)0;
    if (d > (R)1) d = (R)1;
    R s = d * (R)(V.tf_n - 1);
    int i = (int)std::floor(s);
    if (i > V.tf_n - 2) i = V.tf_n - 2;
    R f = s - (R)i;
    R a = (R)V.tf[4 * i + c], b = (R)V.tf[4 * (i + 1) + c];
    return a + f * (b - a);
}

template <typename R> struct Medium { R sigma; V3<R> albedo; };

template <typename R> R sigma_at(const Volume& V, V3<R> p) {
    R d = density<R>(V, p);
    return (R)V.sigma_scale * tf_at<R>(V, d, 3);
}
template <typename R> Medium<R> medium_at(const Volume& V, V3<R> p) {
    R d = density<R>(V, p);
    Medium<R> m;
    m.sigma = (R)V.sigma_scale * tf_at<R>(V, d, 3);
    m.albedo = v3((R)V.albedo * tf_at<R>(V, d, 0), (R)V.albedo * tf_at<R>(V, d, 1), (R)V.albedo * tf_at<R>(V, d, 2));
    return m;
}

// Global majorant: sigma_scale * (max of TF alpha over [0, d_max]) with a
// relative safety margin of 2^-10, so that rounding inside the trilinear and
// table lerps can never lift sigma_t above it.
template <typename R> R majorant(const Volume& V) {
    R dmax = (R)0;
    for (int z = 0; z < V.nz; ++z)
        for (int y = 0; y < V.ny; ++y)
            for (int x = 0; x < V.nx; ++x) {
                R d = voxel<R>(V, x, y, z);
                if (d > dmax) dmax = d;
            }
    if (dmax > (R)1) dmax = (R)1;
    R amax = tf_at<R>(V, dmax, 3);
    for (int i = 0; i < V.tf_n; ++i) {
        R node_d = (R)i / (R)(V.tf_n - 1);
        if (node_d <= dmax && (R)V.tf[4 * i + 3] > amax) amax = (R)V.tf[4 * i + 3];
    }
    return (R)V.sigma_scale * amax * (R)1.0009765625;
}

// Ray / unit-box slab test.  Returns false on a miss; t range clipped to t>=0.
template <typename R> bool box_hit(V3<R> o, V3<R> d, R* t0, R* t1) {
    R lo = (R)0, hi = (R)INFINITY;
    const R oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == (R)0) {
            if (oo[a] < (R)0 || oo[a] > (R)1) return false;
            continue;
        }
        R ta = ((R)0 - oo[a]) / dd[a], tb = ((R)1 - oo[a]) / dd[a];
        R tn = std::min(ta, tb), tf = std::max(ta, tb);
        lo = std::max(lo, tn);
        hi = std::min(hi, tf);
    }
    *t0 = lo; *t1 = hi;
    return lo < hi;
}

// Henyey-Greenstein phase function; mu = cosine between the incoming and the
// outgoing travel directions, so g > 0 is forward scattering (Fig. hg_plot).
template <typename R> R hg_eval(R g, R mu) {
    R gg = g * g;
    R den = (R)1 + gg - (R)2 * g * mu;
    return (R)0.0795774715459476678 * ((R)1 - gg) / (den * M<R>::sqrt_(den));
}

// Importance sampling of HG by inverting its CDF in mu; azimuth uniform.
template <typename R> V3<R> hg_sample(R g, V3<R> d, R xi1, R xi2) {
    R mu;
    if (std::fabs(g) < (R)1e-3) mu = (R)1 - (R)2 * xi1;
    else {
        R gg = g * g;
        R tmp = ((R)1 - gg) / ((R)1 - g + (R)2 * g * xi1);
        mu = ((R)1 + gg - tmp * tmp) / ((R)2 * g);
    }
    if (mu < (R)-1) mu = (R)-1;
    if (mu > (R)1) mu = (R)1;
    R st = M<R>::sqrt_(std::max((R)0, (R)1 - mu * mu));
    R sp, cp;
    M<R>::sincos2pi(xi2, &sp, &cp);
    V3<R> e1, e2;
    onb(d, &e1, &e2);
    R a = st * cp, b = st * sp;
    V3<R> nd = v3(e1.x * a + e2.x * b + d.x * mu, e1.y * a + e2.y * b + d.y * mu, e1.z * a + e2.z * b + d.z * mu);
    return normalize(nd);
}

// Brick majorant grid.  Brick (i,j,k) covers voxels [B i, B i + B) per axis
// (B = brick edge in voxels, a power of two) and the region between the
// planes x = B i / nx and B (i+1) / nx (same for y, z; the last brick is cut
// by the box).  Its majorant bounds sigma_t anywhere in that region, extended
// by half a voxel: sigma_scale times the largest TF alpha over the density
// range [dmin, dmax] of the voxels trilinear interpolation can reach there
// (the brick plus a one-voxel apron; bricks on the box boundary also include
// density 0, the value outside the box), times (1 + 2^-10).
template <typename R> struct Grid {
    int gx, gy, gz, nx, ny, nz, B;
    std::vector<R> m;
    R at(int i, int j, int k) const { return m[(size_t)i + (size_t)gx * ((size_t)j + (size_t)gy * k)]; }
};

template <typename R> R tf_alpha_max(const Volume& V, R dmin, R dmax) {
    if (dmin < (R)0) dmin = (R)0;
    if (dmax > (R)1) dmax = (R)1;
    R a = std::max(tf_at<R>(V, dmin, 3), tf_at<R>(V, dmax, 3));
    for (int i = 0; i < V.tf_n; ++i) {
        R nd = (R)i / (R)(V.tf_n - 1);
        if (nd >= dmin && nd <= dmax && (R)V.tf[4 * i + 3] > a) a = (R)V.tf[4 * i + 3];
    }
    return a;
}

template <typename R> Grid<R> build_grid(const Volume& V, int B) {
    Grid<R> G;
    G.nx = V.nx; G.ny = V.ny; G.nz = V.nz; G.B = B;
    G.gx = (V.nx + B - 1) / B; G.gy = (V.ny + B - 1) / B; G.gz = (V.nz + B - 1) / B;
    G.m.assign((size_t)G.gx * G.gy * G.gz, (R)0);
    for (int bz = 0; bz < G.gz; ++bz)
        for (int by = 0; by < G.gy; ++by)
            for (int bx = 0; bx < G.gx; ++bx) {
                R dmin = (R)INFINITY, dmax = (R)-INFINITY;
                for (int k = std::max(B * bz - 1, 0); k <= std::min(B * bz + B, V.nz - 1); ++k)
                    for (int j = std::max(B * by - 1, 0); j <= std::min(B * by + B, V.ny - 1); ++j)
                        for (int i = std::max(B * bx - 1, 0); i <= std::min(B * bx + B, V.nx - 1); ++i) {
                            R d = voxel<R>(V, i, j, k);
                            if (d < dmin) dmin = d;
                            if (d > dmax) dmax = d;
                        }
                if (bx == 0 || by == 0 || bz == 0 || bx == G.gx - 1 || by == G.gy - 1 || bz == G.gz - 1)
                    if ((R)0 < dmin) dmin = (R)0;
                G.m[(size_t)bx + (size_t)G.gx * ((size_t)by + (size_t)G.gy * bz)] =
                    (R)V.sigma_scale * tf_alpha_max<R>(V, dmin, dmax) * (R)1.0009765625;
            }
    return G;
}

// Coarser majorant grid for f x f x f groups of bricks (brick edge f B):
// the largest of the group's brick majorants (exact; it bounds sigma_t over
// the group because each brick majorant bounds it over its brick).
template <typename R> Grid<R> pool_grid(const Grid<R>& G, int f) {
    if (f <= 1) return G;
    Grid<R> P;
    P.nx = G.nx; P.ny = G.ny; P.nz = G.nz; P.B = G.B * f;
    P.gx = (G.gx + f - 1) / f; P.gy = (G.gy + f - 1) / f; P.gz = (G.gz + f - 1) / f;
    P.m.assign((size_t)P.gx * P.gy * P.gz, (R)0);
    for (int k = 0; k < G.gz; ++k)
        for (int j = 0; j < G.gy; ++j)
            for (int i = 0; i < G.gx; ++i) {
                R& c = P.m[(size_t)(i / f) + (size_t)P.gx * ((size_t)(j / f) + (size_t)P.gy * (k / f))];
                c = std::max(c, G.at(i, j, k));
            }
    return P;
}

// Walk over the bricks a ray crosses (Amanatides-Woo).  Per axis: brick
// width w = B / n, inverse direction inv = 1/d; the first plane parameter is
// (plane - o) * inv and each further plane adds w * |inv|.  The rounding of
// the plane parameters stays far below the half-voxel margin of the brick
// majorants.
template <typename R> struct Walk {
    int c[3], s[3], g[3];
    R tn[3], dt[3];
    void init(const Grid<R>& G, V3<R> o, V3<R> d, R t) {
        const R oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
        const int n[3] = {G.nx, G.ny, G.nz};
        g[0] = G.gx; g[1] = G.gy; g[2] = G.gz;
        for (int a = 0; a < 3; ++a) {
            R w = (R)G.B / (R)n[a];
            R p = oo[a] + t * dd[a];
            int ci = (int)std::floor(p / w);
            c[a] = std::min(std::max(ci, 0), g[a] - 1);
            if (dd[a] > (R)0) {
                R inv = (R)1 / dd[a];
                s[a] = 1; tn[a] = ((R)(c[a] + 1) * w - oo[a]) * inv; dt[a] = w * inv;
            } else if (dd[a] < (R)0) {
                R inv = (R)1 / dd[a];
                s[a] = -1; tn[a] = ((R)c[a] * w - oo[a]) * inv; dt[a] = -(w * inv);
            } else {
                s[a] = 0; tn[a] = (R)INFINITY; dt[a] = (R)INFINITY;
            }
        }
    }
    R exit_t() const { return std::min(tn[0], std::min(tn[1], tn[2])); }
    // step into the next brick; false when the ray leaves the grid
    bool step() {
        int a = (tn[0] <= tn[1] && tn[0] <= tn[2]) ? 0 : (tn[1] <= tn[2] ? 1 : 2);
        c[a] += s[a];
        if (c[a] < 0 || c[a] >= g[a]) return false;
        tn[a] = tn[a] + dt[a];
        return true;
    }
};

// Uniforms of one tracking call, taken one at a time from the caller's
// stream, four per Philox block in lane order; the rest of the last block is
// discarded when the call returns.
template <typename R> struct Uniforms {
    Rng& rng;
    R u[4] = {0, 0, 0, 0};
    int k = 4;
    explicit Uniforms(Rng& r) : rng(r) {}
    R next() {
        if (k == 4) { rng.uni4<R>(u); k = 0; }
        return u[k++];
    }
};

// Delta (Woodcock) tracking over the brick majorants from o along d inside
// [t, t_end).  Uniforms in order: the optical-depth budget tau = -ln(1-u) of
// the next tentative collision, spent brick by brick; at a tentative
// collision one uniform accepts it with probability sigma_t / majorant, then
// the next budget.  Returns true and the distance on a real collision.
template <typename R> bool delta_track(const Volume& V, const Grid<R>& G, V3<R> o, V3<R> d, R t, R t_end, Rng& rng,
                                       R* t_hit, long* steps) {
    Walk<R> W; W.init(G, o, d, t);
    Uniforms<R> U(rng);
    R tau = -M<R>::ln((R)1 - U.next());
    for (long it = 0; it < (1L << 24); ++it) {
        R m = G.at(W.c[0], W.c[1], W.c[2]);
        R tc = std::min(W.exit_t(), t_end);
        R seg = tc - t;
        if (seg < (R)0) seg = (R)0;
        if (m > (R)0 && tau < m * seg) {
            t = t + tau / m;
            if (steps) ++*steps;
            R ua = U.next();
            if (ua * m < sigma_at<R>(V, along(o, d, t))) { *t_hit = t; return true; }
            tau = -M<R>::ln((R)1 - U.next());
            continue;
        }
        tau = tau - m * seg;
        t = tc;
        if (t >= t_end) return false;
        if (!W.step()) return false;
    }
    return false;
}

// Ratio-tracking transmittance over [0, t_end) with the brick majorants: at
// each tentative collision T *= max(0, 1 - sigma_t / majorant); one uniform
// per tentative collision (its budget).
template <typename R> R ratio_track(const Volume& V, const Grid<R>& G, V3<R> o, V3<R> d, R t_end, Rng& rng) {
    Walk<R> W; W.init(G, o, d, (R)0);
    Uniforms<R> U(rng);
    R T = (R)1, t = (R)0;
    R tau = -M<R>::ln((R)1 - U.next());
    for (long it = 0; it < (1L << 24); ++it) {
        R m = G.at(W.c[0], W.c[1], W.c[2]);
        R tc = std::min(W.exit_t(), t_end);
        R seg = tc - t;
        if (seg < (R)0) seg = (R)0;
        if (m > (R)0 && tau < m * seg) {
            t = t + tau / m;
            R f = (R)1 - sigma_at<R>(V, along(o, d, t)) / m;
            T = T * std::max((R)0, f);
            tau = -M<R>::ln((R)1 - U.next());
            continue;
        }
        tau = tau - m * seg;
        t = tc;
        if (t >= t_end) break;
        if (!W.step()) break;
    }
    return T;
}

// Ratio tracking as above whose tentative collisions come from a coarser
// walk: the rays cross the bricks of Gw (edge f B, each the largest of its
// f^3 bricks of G) and a tentative collision of that process at x is kept
// with probability m_G(x) / m_Gw (one more uniform, after the collision's
// budget), which thins it to a Poisson process of rate m_G: the estimator is
// ratio tracking with the tight majorant of G, T *= max(0, 1 - sigma_t /
// m_G(x)) at kept collisions, at the cost of a walk over the coarse bricks.
// m_G(x) is the majorant of the brick of G holding x, its index clamped into
// the current brick of Gw.  Gw = G is plain ratio tracking.
template <typename R> R ratio_track_thinned(const Volume& V, const Grid<R>& G, const Grid<R>& Gw, V3<R> o, V3<R> d,
                                            R t_end, Rng& rng) {
    if (Gw.B == G.B) return ratio_track<R>(V, G, o, d, t_end, rng);
    const int f = Gw.B / G.B;
    Walk<R> W; W.init(Gw, o, d, (R)0);
    Uniforms<R> U(rng);
    R T = (R)1, t = (R)0;
    R tau = -M<R>::ln((R)1 - U.next());
    for (long it = 0; it < (1L << 24); ++it) {
        R m = Gw.at(W.c[0], W.c[1], W.c[2]);
        R tc = std::min(W.exit_t(), t_end);
        R seg = tc - t;
        if (seg < (R)0) seg = (R)0;
        if (m > (R)0 && tau < m * seg) {
            t = t + tau / m;
            R ut = U.next();
            V3<R> x = along(o, d, t);
            const R p[3] = {x.x, x.y, x.z};
            const int n[3] = {G.nx, G.ny, G.nz}, g[3] = {G.gx, G.gy, G.gz};
            int c[3];
            for (int a = 0; a < 3; ++a) {
                R w = (R)G.B / (R)n[a];
                int ci = (int)std::floor(p[a] / w);
                int lo = W.c[a] * f, hi = std::min(W.c[a] * f + f, g[a]) - 1;
                c[a] = std::min(std::max(ci, lo), hi);
            }
            R mf = G.at(c[0], c[1], c[2]);
            if (ut * m < mf) {
                R fr = (R)1 - sigma_at<R>(V, x) / mf;
                T = T * std::max((R)0, fr);
            }
            tau = -M<R>::ln((R)1 - U.next());
            continue;
        }
        tau = tau - m * seg;
        t = tc;
        if (t >= t_end) break;
        if (!W.step()) break;
    }
    return T;
}

// Direction to light l from x, distance limit and irradiance at x.
template <typename R> void light_geom(const Light& L, V3<R> x, V3<R>* wl, R* dist, V3<R>* E) {
    if (L.kind == 0) {
        *wl = normalize(v3((R)L.v[0], (R)L.v[1], (R)L.v[2]));
        *dist = (R)INFINITY;
        *E = v3((R)L.rgb[0], (R)L.rgb[1], (R)L.rgb[2]);
    } else {
        V3<R> dv = sub(v3((R)L.v[0], (R)L.v[1], (R)L.v[2]), x);
        R d2 = dot(dv, dv);
        R dl = M<R>::sqrt_(d2);
        *wl = scl(dv, (R)1 / dl);
        *dist = dl;
        *E = v3((R)L.rgb[0] / d2, (R)L.rgb[1] / d2, (R)L.rgb[2] / d2);
    }
}

// Pinhole camera frame, computed in double on the host and rounded once.
struct CamFrame { double eye[3], f[3], r[3], u[3]; double sx, sy; int W, H; };
CamFrame cam_frame(const double eye[3], const double at[3], const double up[3], double fovy_deg, int W, int H) {
    CamFrame c;
    double f[3] = {at[0] - eye[0], at[1] - eye[1], at[2] - eye[2]};
    double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int i = 0; i < 3; ++i) f[i] /= fn;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int i = 0; i < 3; ++i) r[i] /= rn;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    double th = std::tan(0.5 * fovy_deg * M_PI / 180.0);
    for (int i = 0; i < 3; ++i) { c.eye[i] = eye[i]; c.f[i] = f[i]; c.r[i] = r[i]; c.u[i] = u[i]; }
    c.sy = th; c.sx = th * (double)W / (double)H; c.W = W; c.H = H;
    return c;
}

// Camera ray through pixel (px, py) with jitter (j1, j2); row 0 at the top.
template <typename R> void camera_ray(const CamFrame& c, int px, int py, R j1, R j2, V3<R>* o, V3<R>* d) {
    R a = ((R)2 * ((R)px + j1) / (R)c.W - (R)1) * (R)c.sx;
    R b = ((R)1 - (R)2 * ((R)py + j2) / (R)c.H) * (R)c.sy;
    V3<R> dir = v3((R)c.f[0] + a * (R)c.r[0] + b * (R)c.u[0],
                   (R)c.f[1] + a * (R)c.r[1] + b * (R)c.u[1],
                   (R)c.f[2] + a * (R)c.r[2] + b * (R)c.u[2]);
    *d = normalize(dir);
    *o = v3((R)c.eye[0], (R)c.eye[1], (R)c.eye[2]);
}

// ------------------------------------------------------------------ photon tracing (Algorithm 1)
// Photon p: light l = p / (n_g*N), phase index gi = (p / N) % n_g.
// Emission (Philox block 0):
//   directional: start on the square of side sqrt(3) perpendicular to the
//     light direction, centred one unit upstream of the box centre; power
//     E * 3 / N (the square's area is 3);
//   point: isotropic direction (z = 1 - 2u0, azimuth 2*pi*u1); power I*4*pi/N.
// Transport: delta tracking against the global majorant; at real collision j
//   (i) j >= 2: record (bin(x), incoming direction, power before albedo);
//   (ii) power *= albedo(x);  (iii) j == max_bounces: stop;
//   (iv) new direction from HG(g) [block u0,u1];
//   (v) Russian roulette for j >= 3 [u2]: q = min(1, max_c P_c / max_c P_emit,c).
struct Tally { double emitted[3], escaped[3], absorbed[3], truncated[3], rr[3]; };

template <typename R>
void trace_photon(const Volume& V, const Grid<R>& G, const Light* lights, int n_lights, const float* gset, int n_g,
                  uint64_t N, int max_bounces, int res, uint64_t seed, int use_rr, uint64_t p,
                  // outputs: per-photon slots (max_bounces-1 of them)
                  uint32_t* keys, float* dirs, float* phis, float* poss, int* nrec, Tally* T) {
    int l = (int)(p / ((uint64_t)n_g * N));
    int gi = (int)((p / N) % (uint64_t)n_g);
    const Light& L = lights[l];
    R g = (R)gset[gi];
    Rng rng(seed, 2, p, 0);
    R u[4]; rng.uni4<R>(u);
    V3<R> o, d; R P[3], Pe[3];
    if (L.kind == 0) {
        V3<R> v = normalize(v3((R)L.v[0], (R)L.v[1], (R)L.v[2]));
        V3<R> e1, e2; onb(v, &e1, &e2);
        R side = (R)1.7320508075688772;
        R a = (u[0] - (R)0.5) * side, b = (u[1] - (R)0.5) * side;
        o = v3((R)0.5 + v.x + a * e1.x + b * e2.x, (R)0.5 + v.y + a * e1.y + b * e2.y, (R)0.5 + v.z + a * e1.z + b * e2.z);
        d = v3(-v.x, -v.y, -v.z);
        for (int c = 0; c < 3; ++c) P[c] = (R)L.rgb[c] * (R)3 / (R)N;
    } else {
        R z = (R)1 - (R)2 * u[0];
        R r = M<R>::sqrt_(std::max((R)0, (R)1 - z * z));
        R sp, cp; M<R>::sincos2pi(u[1], &sp, &cp);
        d = v3(r * cp, r * sp, z);
        o = v3((R)L.v[0], (R)L.v[1], (R)L.v[2]);
        for (int c = 0; c < 3; ++c) P[c] = (R)L.rgb[c] * (R)12.566370614359172 / (R)N;
    }
    for (int c = 0; c < 3; ++c) { Pe[c] = P[c]; T->emitted[c] += (double)P[c]; }
    R pe_max = std::max(Pe[0], std::max(Pe[1], Pe[2]));
    int n = 0, j = 0;
    R t0 = (R)0, t1 = (R)0;
    bool alive = true;                     // photons that miss the box escape at once
    bool inside = box_hit(o, d, &t0, &t1);
    R t = t0;
    while (alive && inside) {
        R th;
        if (!delta_track<R>(V, G, o, d, t, t1, rng, &th, nullptr)) break;
        V3<R> x = along(o, d, th);
        j = j + 1;
        Medium<R> m = medium_at<R>(V, x);
        if (j >= 2) {
            int bx = (int)std::floor(x.x * (R)res), by = (int)std::floor(x.y * (R)res), bz = (int)std::floor(x.z * (R)res);
            bx = std::min(std::max(bx, 0), res - 1); by = std::min(std::max(by, 0), res - 1); bz = std::min(std::max(bz, 0), res - 1);
            uint32_t bin = (uint32_t)bx + (uint32_t)res * ((uint32_t)by + (uint32_t)res * (uint32_t)bz);
            uint32_t key = (uint32_t)(l * n_g + gi) * (uint32_t)(res * res * res) + bin;
            keys[n] = key;
            dirs[3 * n + 0] = (float)d.x; dirs[3 * n + 1] = (float)d.y; dirs[3 * n + 2] = (float)d.z;
            phis[3 * n + 0] = (float)P[0]; phis[3 * n + 1] = (float)P[1]; phis[3 * n + 2] = (float)P[2];
            poss[3 * n + 0] = (float)x.x; poss[3 * n + 1] = (float)x.y; poss[3 * n + 2] = (float)x.z;
            n = n + 1;
        }
        R Pa[3] = {P[0] * m.albedo.x, P[1] * m.albedo.y, P[2] * m.albedo.z};
        for (int c = 0; c < 3; ++c) { T->absorbed[c] += (double)P[c] - (double)Pa[c]; P[c] = Pa[c]; }
        if (j == max_bounces) {
            for (int c = 0; c < 3; ++c) T->truncated[c] += (double)P[c];
            alive = false; break;
        }
        R w[4]; rng.uni4<R>(w);
        V3<R> nd = hg_sample<R>(g, d, w[0], w[1]);
        if (use_rr && j >= 3) {
            R q = std::max(P[0], std::max(P[1], P[2])) / pe_max;
            if (q > (R)1) q = (R)1;
            if (!(w[2] < q)) {
                for (int c = 0; c < 3; ++c) T->rr[c] += (double)P[c];
                alive = false; break;
            }
            for (int c = 0; c < 3; ++c) { R np = P[c] / q; T->rr[c] -= (double)np - (double)P[c]; P[c] = np; }
        }
        o = x; d = nd;
        R a0, a1;
        if (!box_hit(o, d, &a0, &a1)) { break; }
        t = (R)0; t1 = a1;
    }
    if (alive) for (int c = 0; c < 3; ++c) T->escaped[c] += (double)P[c];
    *nrec = n;
}

// ------------------------------------------------------------------ camera samples (Algorithm 2)
// March mode (step > 0): ray-marched inverse-CDF free flight and marched
// shadow rays.  Segment k covers [t0+k*h, min(t0+(k+1)*h, t1)), sigma taken at
// seg_start + u*len.  Interaction where the accumulated optical depth reaches
// tau* = -ln(1-u3).  Philox block 0: (j1, j2, u_march, u_tau); blocks 1..:
// one jitter per light (light l uses lane l%4 of block 1 + l/4).
// Delta mode (step == 0): block 0 (j1, j2, -, -), then delta tracking for the
// free flight on the same stream; the shadow ray towards light l is ratio
// tracked on a stream of its own (shadow_item, bounce 1), summed in light
// order.
// Stream of the shadow ray towards light l at interaction j of a camera
// sample: tag 5, sub = sample index, item = pixel + (16 (j-1) + l) 2^32.
inline uint64_t shadow_item(uint64_t pixel, int j, int l) {
    return pixel + ((uint64_t)(16 * (j - 1) + l) << 32);
}

template <typename R>
R march_tau(const Volume& V, V3<R> o, V3<R> d, R t0, R t1, R h, R jit) {
    R tau = (R)0;
    if (!(t1 > t0)) return tau;
    long nseg = (long)std::ceil((double)((t1 - t0) / h));
    for (long k = 0; k < nseg; ++k) {
        R s0 = t0 + (R)k * h;
        R s1 = std::min(t0 + (R)(k + 1) * h, t1);
        R len = s1 - s0;
        if (!(len > (R)0)) continue;
        tau = tau + sigma_at<R>(V, along(o, d, s0 + jit * len)) * len;
    }
    return tau;
}

// Marched free flight and shadow-ray optical depth in the kernel's float32
// precision contract.  The segments, their sample points and sigma are the
// float32 steps above; the running optical depth is a compensated (Kahan)
// float32 sum; the target tau* = -ln(1 - u) and the remainder at the
// interaction, (tau* - tau) / sigma, are evaluated in FP64 (where sigma is
// small one float ulp of tau* or tau would move the interaction by ulp/sigma).
// Real arithmetic gives the plain sums of march_tau and camera_sample.
bool march_flight_f32(const Volume& V, V3<float> o, V3<float> d, float t0, float t1, float h, float u_seg, float u_tau,
                      float* th) {
    const double tau_star_d = -std::log1p(-(double)u_tau);
    const float tau_star = (float)tau_star_d;
    float tau = 0.0f, comp = 0.0f;
    const int nseg = (int)std::ceil((t1 - t0) / h);
    for (int s = 0; s < nseg; ++s) {
        const float s0 = t0 + (float)s * h;
        const float s1 = std::min(t0 + (float)(s + 1) * h, t1);
        const float len = s1 - s0;
        if (!(len > 0.0f)) continue;
        const float sg = sigma_at<float>(V, along(o, d, s0 + u_seg * len));
        const float dtau = sg * len;
        if (sg > 0.0f && (tau - comp) + dtau >= tau_star) {
            const double rem = tau_star_d - ((double)tau - (double)comp);
            const float dl = (float)(rem / (double)sg);
            *th = s0 + std::min(std::max(dl, 0.0f), len);
            return true;
        }
        const float y = dtau - comp;
        const float t = tau + y;
        comp = (t - tau) - y;
        tau = t;
    }
    return false;
}

float march_tau_f32(const Volume& V, V3<float> o, V3<float> d, float tend, float h, float jit) {
    float tau = 0.0f, comp = 0.0f;
    if (!(tend > 0.0f)) return 0.0f;
    const int nseg = (int)std::ceil(tend / h);
    for (int s = 0; s < nseg; ++s) {
        const float s0 = (float)s * h;
        const float s1 = std::min((float)(s + 1) * h, tend);
        const float len = s1 - s0;
        if (!(len > 0.0f)) continue;
        const float y = sigma_at<float>(V, along(o, d, s0 + jit * len)) * len - comp;
        const float t = tau + y;
        comp = (t - tau) - y;
        tau = t;
    }
    return tau - comp;
}

template <typename R>
void camera_sample(const Volume& V, const Grid<R>& G, const Grid<R>& Gp, const Grid<R>& Gs, const Light* lights,
                   int n_lights, R g, const CamFrame& cf,
                   int px, int py, int k, R step_vox, uint64_t seed,
                   int* valid, V3<R>* xo, V3<R>* wo, V3<R>* alb, V3<R>* Ld) {
    Rng rng(seed, 1, (uint64_t)py * (uint64_t)cf.W + (uint64_t)px, (uint32_t)k);
    R b0[4]; rng.uni4<R>(b0);
    V3<R> o, d;
    camera_ray<R>(cf, px, py, b0[0], b0[1], &o, &d);
    *valid = 0; *Ld = v3((R)0, (R)0, (R)0); *alb = *Ld; *xo = *Ld;
    *wo = v3(-d.x, -d.y, -d.z);
    R t0, t1;
    if (!box_hit(o, d, &t0, &t1)) return;
    int nmax = std::max(V.nx, std::max(V.ny, V.nz));
    R th = (R)0;
    bool hit = false;
    R jl[16];
    if (step_vox > (R)0) {
        R h = step_vox / (R)nmax;
        for (int b = 0; b < (n_lights + 3) / 4; ++b) { R w[4]; rng.uni4<R>(w); for (int i = 0; i < 4; ++i) if (4 * b + i < 16) jl[4 * b + i] = w[i]; }
        if constexpr (std::is_same<R, float>::value) {
            hit = march_flight_f32(V, o, d, t0, t1, h, b0[2], b0[3], &th);
        } else {
            R tau_star = -M<R>::ln((R)1 - b0[3]);
            R tau = (R)0;
            long nseg = (long)std::ceil((double)((t1 - t0) / h));
            for (long s = 0; s < nseg; ++s) {
                R s0 = t0 + (R)s * h;
                R s1 = std::min(t0 + (R)(s + 1) * h, t1);
                R len = s1 - s0;
                if (!(len > (R)0)) continue;
                R sg = sigma_at<R>(V, along(o, d, s0 + b0[2] * len));
                if (sg > (R)0 && tau + sg * len >= tau_star) {
                    th = s0 + (tau_star - tau) / sg;
                    hit = true; break;
                }
                tau = tau + sg * len;
            }
        }
    } else {
        hit = delta_track<R>(V, Gp, o, d, t0, t1, rng, &th, nullptr);
    }
    if (!hit) return;
    V3<R> x = along(o, d, th);
    Medium<R> m = medium_at<R>(V, x);
    V3<R> L = v3((R)0, (R)0, (R)0);
    for (int l = 0; l < n_lights; ++l) {
        V3<R> wl, E; R dist;
        light_geom<R>(lights[l], x, &wl, &dist, &E);
        R a0, a1;
        R tend = (R)0;
        if (box_hit(x, wl, &a0, &a1)) tend = std::min(a1, dist);
        R T;
        if (step_vox > (R)0) {
            R h = step_vox / (R)nmax;
            if constexpr (std::is_same<R, float>::value)
                T = (float)std::exp(-(double)march_tau_f32(V, x, wl, tend, h, jl[l]));
            else
                T = std::exp(-march_tau<R>(V, x, wl, (R)0, tend, h, jl[l]));
        } else {
            Rng rs(seed, 5, shadow_item((uint64_t)py * (uint64_t)cf.W + (uint64_t)px, 1, l), (uint32_t)k);
            T = ratio_track_thinned<R>(V, G, Gs, x, wl, tend, rs);
        }
        R ph = hg_eval<R>(g, dot(d, wl));
        L = v3(L.x + ph * T * E.x, L.y + ph * T * E.y, L.z + ph * T * E.z);
    }
    *valid = 1; *xo = x; *alb = m.albedo; *Ld = L;
}

// ------------------------------------------------------------------ ray marching with the field at every step
// Sec. 3.6: the field replaces the multiple-scattering term in ray marching
// as well as in path tracing.  Camera sample k of pixel p: the ray from Philox
// block 0 of (seed, tag 1, p, k) (lanes 0, 1: pixel jitter; lane 2: march
// offset u).  Segment s covers [t0 + s h, min(t0 + (s+1) h, t1)) with its
// sample point at fraction u of it and sigma_s = sigma_t there; tau_s is the
// optical depth of the segments before it.  Weight
//   a_s = exp(-tau_s) (1 - exp(-sigma_s len_s))
// (the segment's exact share of the ray's extinction for constant sigma, so
// the weights of a ray add up to 1 - exp(-tau) of the whole ray), and
//   L = sum_s a_s albedo(x_s) (L_d(x_s) + L_i(x_s, -d, g)),
// L_d towards every light by a marched shadow ray (march_tau) whose jitter is
// lane l % 4 of block 4 s + l / 4 of the stream (seed, tag 6, p, k).  A
// segment with sigma_s = 0 adds nothing and asks no field query.
// D: the ray's direct part; returns the number of field queries; q, w (each
// nullable) receive the queries (x, theta', phi', g) and weights a_s albedo_s.
long raymarch_ray(const Volume& V, const Light* lights, int n_lights, double g, const CamFrame& cf, int px, int py,
                  int k, double h, uint64_t seed, double D[3], double* q, double* w) {
    const uint64_t pix = (uint64_t)py * (uint64_t)cf.W + (uint64_t)px;
    Rng rng(seed, 1, pix, (uint32_t)k);
    double b0[4]; rng.uni4<double>(b0);
    V3<double> o, d;
    camera_ray<double>(cf, px, py, b0[0], b0[1], &o, &d);
    D[0] = D[1] = D[2] = 0.0;
    long n = 0;
    double t0, t1;
    if (!box_hit(o, d, &t0, &t1)) return 0;
    const double th = std::acos(std::min(1.0, std::max(-1.0, -d.z))) / M_PI;
    double ph = std::atan2(-d.y, -d.x) / (2.0 * M_PI);
    if (ph < 0.0) ph += 1.0;
    const long nseg = (long)std::ceil((t1 - t0) / h);
    double tau = 0.0;
    for (long s = 0; s < nseg; ++s) {
        const double s0 = t0 + (double)s * h;
        const double s1 = std::min(t0 + (double)(s + 1) * h, t1);
        const double len = s1 - s0;
        if (!(len > 0.0)) continue;
        const V3<double> x = along(o, d, s0 + b0[2] * len);
        const Medium<double> m = medium_at<double>(V, x);
        if (m.sigma > 0.0) {
            const double a = std::exp(-tau) * -std::expm1(-m.sigma * len);
            double Ld[3] = {0.0, 0.0, 0.0};
            Rng rs(seed, 6, pix, (uint32_t)k);
            for (int gq = 0; 4 * gq < n_lights; ++gq) {
                rs.ctr[3] = (uint32_t)(4 * s + gq);
                double jit[4]; rs.uni4<double>(jit);
                for (int i = 0; i < 4 && 4 * gq + i < n_lights; ++i) {
                    V3<double> wl, E; double dist;
                    light_geom<double>(lights[4 * gq + i], x, &wl, &dist, &E);
                    double a0, a1, tend = 0.0;
                    if (box_hit(x, wl, &a0, &a1)) tend = std::min(a1, dist);
                    const double T = std::exp(-march_tau<double>(V, x, wl, 0.0, tend, h, jit[i]));
                    const double p = hg_eval<double>(g, dot(d, wl));
                    Ld[0] += p * T * E.x; Ld[1] += p * T * E.y; Ld[2] += p * T * E.z;
                }
            }
            const double wr[3] = {a * m.albedo.x, a * m.albedo.y, a * m.albedo.z};
            for (int c = 0; c < 3; ++c) D[c] += wr[c] * Ld[c];
            if (q) {
                q[6 * n + 0] = x.x; q[6 * n + 1] = x.y; q[6 * n + 2] = x.z;
                q[6 * n + 3] = th; q[6 * n + 4] = ph; q[6 * n + 5] = g;
            }
            if (w) for (int c = 0; c < 3; ++c) w[3 * n + c] = wr[c];
            ++n;
        }
        tau += m.sigma * len;
    }
    return n;
}

// ------------------------------------------------------------------ path tracer
// Delta tracking; at every real collision j: next-event estimation towards
// every light with ratio-tracking transmittance (each shadow ray on its own
// stream, shadow_item(pixel, j, l)), weighted by throughput and
// albedo; then throughput *= albedo; stop at j == max_bounces; HG continuation
// and Russian roulette (j >= 3, q = min(1, max_c beta_c)) from one block.
template <typename R>
V3<R> path_sample(const Volume& V, const Grid<R>& G, const Light* lights, int n_lights, R g, const CamFrame& cf,
                  int px, int py, int k, int max_bounces, uint64_t seed, int use_rr) {
    Rng rng(seed, 1, (uint64_t)py * (uint64_t)cf.W + (uint64_t)px, (uint32_t)k);
    R b0[4]; rng.uni4<R>(b0);
    V3<R> o, d;
    camera_ray<R>(cf, px, py, b0[0], b0[1], &o, &d);
    V3<R> rad = v3((R)0, (R)0, (R)0);
    R beta[3] = {(R)1, (R)1, (R)1};
    R t0, t1;
    if (!box_hit(o, d, &t0, &t1)) return rad;
    R t = t0;
    for (int j = 1; j <= max_bounces; ++j) {
        R th;
        if (!delta_track<R>(V, G, o, d, t, t1, rng, &th, nullptr)) break;
        V3<R> x = along(o, d, th);
        Medium<R> m = medium_at<R>(V, x);
        V3<R> L = v3((R)0, (R)0, (R)0);
        for (int l = 0; l < n_lights; ++l) {
            V3<R> wl, E; R dist;
            light_geom<R>(lights[l], x, &wl, &dist, &E);
            R a0, a1, tend = (R)0;
            if (box_hit(x, wl, &a0, &a1)) tend = std::min(a1, dist);
            Rng rs(seed, 5, shadow_item((uint64_t)py * (uint64_t)cf.W + (uint64_t)px, j, l), (uint32_t)k);
            R T = ratio_track<R>(V, G, x, wl, tend, rs);
            R ph = hg_eval<R>(g, dot(d, wl));
            L = v3(L.x + ph * T * E.x, L.y + ph * T * E.y, L.z + ph * T * E.z);
        }
        R ca[3] = {beta[0] * m.albedo.x, beta[1] * m.albedo.y, beta[2] * m.albedo.z};
        rad = v3(rad.x + ca[0] * L.x, rad.y + ca[1] * L.y, rad.z + ca[2] * L.z);
        beta[0] = ca[0]; beta[1] = ca[1]; beta[2] = ca[2];
        if (j == max_bounces) break;
        R w[4]; rng.uni4<R>(w);
        V3<R> nd = hg_sample<R>(g, d, w[0], w[1]);
        if (use_rr && j >= 3) {
            R q = std::max(beta[0], std::max(beta[1], beta[2]));
            if (q > (R)1) q = (R)1;
            if (!(w[2] < q)) break;
            for (int c = 0; c < 3; ++c) beta[c] = beta[c] / q;
        }
        o = x; d = nd;
        R a0, a1;
        if (!box_hit(o, d, &a0, &a1)) break;
        t = (R)0; t1 = a1;
    }
    return rad;
}

Volume mkvol(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb, const float* tf, int tf_n) {
    Volume V; V.nx = nx; V.ny = ny; V.nz = nz; V.dtype = dtype; V.data = data;
    V.sigma_scale = ss; V.albedo = alb; V.tf = tf; V.tf_n = tf_n; return V;
}
std::vector<Light> mklights(const int* kinds, const double* v, const double* rgb, int n) {
    std::vector<Light> L(n);
    for (int i = 0; i < n; ++i) {
        L[i].kind = kinds[i];
        for (int c = 0; c < 3; ++c) { L[i].v[c] = v[3 * i + c]; L[i].rgb[c] = rgb[3 * i + c]; }
    }
    return L;
}

}  // namespace

// ================================================================== C ABI for the Python wrapper
extern "C" {

void orc_philox(uint64_t seed, const uint32_t* ctr4, uint32_t* out4) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox4x32_10(key, ctr4, out4);
}

// n blocks of four raw words for items [0, n_items), blocks [0, n_blocks)
void orc_philox_stream(uint64_t seed, uint32_t tag, uint32_t sub, int64_t n_items, int n_blocks, uint32_t* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_items; ++i) {
        Rng r(seed, tag, (uint64_t)i, sub);
        for (int b = 0; b < n_blocks; ++b) r.raw4(out + ((size_t)i * n_blocks + b) * 4);
    }
}

// Raw words [block][4] of one item of the stream (seed, tag, sub).
void orc_philox_item(uint64_t seed, uint32_t tag, uint32_t sub, uint64_t item, int64_t n_blocks, uint32_t* out) {
    Rng r(seed, tag, item, sub);
    for (int64_t b = 0; b < n_blocks; ++b) r.raw4(out + (size_t)b * 4);
}

void orc_lnf(const float* x, float* y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = own_lnf(x[i]); }
void orc_sincos2pif(const float* u, float* s, float* c, int64_t n) {
    for (int64_t i = 0; i < n; ++i) own_sincos2pif(u[i], s + i, c + i);
}

// Frequency encoding (Sec. 3.4) of n queries of 6 inputs, F frequencies,
// features [input][k][sin, cos], in the float32 steps of the tensor-core
// fields: sin / cos (2^k pi v) at k = 0, 4, 8, ... from the own turn-based
// sine / cosine of frac(2^(k-1) v); in between by the double-angle formulas
// sin 2a = 2 sin a cos a, cos 2a = 1 - 2 sin^2 a.
void orc_encode_f32(const float* q, int64_t n, int F, float* out) {
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 6; ++d) {
            const float v = q[6 * i + d];
            float s = 0.0f, c = 1.0f;
            for (int k = 0; k < F; ++k) {
                if ((k & 3) == 0) {
                    const float t = v * std::ldexp(1.0f, k - 1);
                    own_sincos2pif(t - std::floor(t), &s, &c);
                } else {
                    const float s2 = (s * c) * 2.0f;
                    c = 1.0f - 2.0f * (s * s);
                    s = s2;
                }
                out[(i * 6 + d) * 2 * F + 2 * k] = s;
                out[(i * 6 + d) * 2 * F + 2 * k + 1] = c;
            }
        }
}

void orc_atan2f(const float* y, const float* x, float* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) out[i] = own_atan2f(y[i], x[i]);
}

// Field queries (x, theta', phi', g) of camera samples in float32, as the
// renderer forms them from its float32 interaction point and direction.
void orc_query_f32(const float* x, const float* wo, float g, int64_t n, float* q) {
    for (int64_t i = 0; i < n; ++i) {
        float th, ph;
        query_angles_f32(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2], &th, &ph);
        q[6 * i + 0] = x[3 * i]; q[6 * i + 1] = x[3 * i + 1]; q[6 * i + 2] = x[3 * i + 2];
        q[6 * i + 3] = th; q[6 * i + 4] = ph; q[6 * i + 5] = g;
    }
}

double orc_hg_eval(double g, double mu) { return hg_eval<double>(g, mu); }
void orc_hg_sample(double g, const double* d, const double* xi, int64_t n, double* out, int fp32) {
    for (int64_t i = 0; i < n; ++i) {
        if (fp32) {
            V3<float> r = hg_sample<float>((float)g, v3((float)d[0], (float)d[1], (float)d[2]), (float)xi[2 * i], (float)xi[2 * i + 1]);
            out[3 * i] = r.x; out[3 * i + 1] = r.y; out[3 * i + 2] = r.z;
        } else {
            V3<double> r = hg_sample<double>(g, v3(d[0], d[1], d[2]), xi[2 * i], xi[2 * i + 1]);
            out[3 * i] = r.x; out[3 * i + 1] = r.y; out[3 * i + 2] = r.z;
        }
    }
}

void orc_density(int nx, int ny, int nz, int dtype, const void* data, const double* p, int64_t n, double* out, int fp32) {
    Volume V = mkvol(nx, ny, nz, dtype, data, 1.0, 1.0, nullptr, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (fp32) out[i] = density<float>(V, v3((float)p[3 * i], (float)p[3 * i + 1], (float)p[3 * i + 2]));
        else out[i] = density<double>(V, v3(p[3 * i], p[3 * i + 1], p[3 * i + 2]));
    }
}

double orc_majorant(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb,
                    const float* tf, int tf_n, int fp32) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, alb, tf, tf_n);
    return fp32 ? (double)majorant<float>(V) : majorant<double>(V);
}

// Brick majorant grid (gx*gy*gz values, x fastest).
void orc_brick_majorants(int nx, int ny, int nz, int dtype, const void* data, double ss, const float* tf, int tf_n, int brick,
                         int fp32, double* out) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, 1.0, tf, tf_n);
    if (fp32) { Grid<float> G = build_grid<float>(V, brick); for (size_t i = 0; i < G.m.size(); ++i) out[i] = G.m[i]; }
    else { Grid<double> G = build_grid<double>(V, brick); for (size_t i = 0; i < G.m.size(); ++i) out[i] = G.m[i]; }
}

// Mean ratio-tracking transmittance from o along d over [0, t_end) (n walks).
double orc_ratio_mean(int nx, int ny, int nz, int dtype, const void* data, double ss, const float* tf, int tf_n, int brick,
                      int brick_shadow, const double* o, const double* d, double t_end, int64_t n, uint64_t seed,
                      double* var) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, 1.0, tf, tf_n);
    Grid<double> G = build_grid<double>(V, brick);
    Grid<double> Gw = pool_grid(G, brick_shadow > brick ? brick_shadow / brick : 1);
    double s = 0, s2 = 0;
    for (int64_t i = 0; i < n; ++i) {
        Rng r(seed, 2, (uint64_t)i, 0);
        double T = ratio_track_thinned<double>(V, G, Gw, v3(o[0], o[1], o[2]), v3(d[0], d[1], d[2]), t_end, r);
        s += T; s2 += T * T;
    }
    *var = s2 / n - (s / n) * (s / n);
    return s / n;
}

// Free-flight distances by delta tracking from o along d (one item per
// sample, Philox tag PHOTON, item i); -1 where the ray leaves the box.
void orc_free_flight(int nx, int ny, int nz, int dtype, const void* data, double ss, const float* tf, int tf_n, int brick,
                     const double* o, const double* d, int64_t n, uint64_t seed, double* out, int64_t* steps) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, 1.0, tf, tf_n);
    Grid<double> G = build_grid<double>(V, brick);
    long st = 0;
    for (int64_t i = 0; i < n; ++i) {
        Rng r(seed, 2, (uint64_t)i, 0);
        V3<double> oo = v3(o[0], o[1], o[2]), dd = v3(d[0], d[1], d[2]);
        double t0, t1, th;
        out[i] = -1.0;
        if (box_hit(oo, dd, &t0, &t1) && delta_track<double>(V, G, oo, dd, t0, t1, r, &th, &st)) out[i] = th - t0;
    }
    *steps = st;
}

// Photon tracing into per-photon slots.  keys[p*S + n] etc. with S =
// max_bounces - 1 (dirs, phis, poss: three floats per slot; poss = the
// interaction position); nrec[p] = records of photon p.  tally[15] = emitted,
// escaped, absorbed, truncated, rr (3 channels each).
void orc_trace_photons(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb,
                       const float* tf, int tf_n, int brick,
                       const int* lkind, const double* lv, const double* lrgb, int n_lights,
                       const float* gset, int n_g, uint64_t N, int max_bounces, int res, uint64_t seed,
                       int use_rr, int fp32, uint64_t p_begin, uint64_t p_end,
                       uint32_t* keys, float* dirs, float* phis, float* poss, int* nrec, double* tally) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, alb, tf, tf_n);
    std::vector<Light> L = mklights(lkind, lv, lrgb, n_lights);
    int S = max_bounces - 1 > 0 ? max_bounces - 1 : 1;
    Grid<double> G64 = fp32 ? Grid<double>() : build_grid<double>(V, brick);
    Grid<float> G32 = fp32 ? build_grid<float>(V, brick) : Grid<float>();
    Tally tot; std::memset(&tot, 0, sizeof(tot));
    #pragma omp parallel
    {
        Tally loc; std::memset(&loc, 0, sizeof(loc));
        #pragma omp for schedule(dynamic, 256)
        for (int64_t q = (int64_t)p_begin; q < (int64_t)p_end; ++q) {
            size_t s = (size_t)(q - (int64_t)p_begin);
            if (fp32) trace_photon<float>(V, G32, L.data(), n_lights, gset, n_g, N, max_bounces, res, seed, use_rr,
                                         (uint64_t)q, keys + s * S, dirs + s * S * 3, phis + s * S * 3, poss + s * S * 3,
                                         nrec + s, &loc);
            else trace_photon<double>(V, G64, L.data(), n_lights, gset, n_g, N, max_bounces, res, seed, use_rr,
                                      (uint64_t)q, keys + s * S, dirs + s * S * 3, phis + s * S * 3, poss + s * S * 3,
                                         nrec + s, &loc);
        }
        #pragma omp critical
        {
            for (int c = 0; c < 3; ++c) {
                tot.emitted[c] += loc.emitted[c]; tot.escaped[c] += loc.escaped[c];
                tot.absorbed[c] += loc.absorbed[c]; tot.truncated[c] += loc.truncated[c]; tot.rr[c] += loc.rr[c];
            }
        }
    }
    for (int c = 0; c < 3; ++c) {
        tally[c] = tot.emitted[c]; tally[3 + c] = tot.escaped[c]; tally[6 + c] = tot.absorbed[c];
        tally[9 + c] = tot.truncated[c]; tally[12 + c] = tot.rr[c];
    }
}

// Camera samples of the neural renderer (Algorithm 2: RayGeneration,
// VolumeSampling, DirectIllumination) of the pixels in rows [y_begin, y_end)
// and columns [x_begin, x_end).  Arrays are [rows][columns][spp].  The free
// flight of the camera rays uses the brick grid pooled to bricks of edge
// brick_primary (0: brick); shadow rays walk the grid pooled to brick_shadow
// (0: brick) thinned to the brick grid.
void orc_camera_samples(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb,
                        const float* tf, int tf_n, int brick, int brick_primary, int brick_shadow,
                        const int* lkind, const double* lv, const double* lrgb, int n_lights, double g,
                        const double* eye, const double* at, const double* up, double fovy, int W, int H,
                        int spp, double step_vox, uint64_t seed, int fp32, int y_begin, int y_end,
                        int x_begin, int x_end,
                        uint8_t* valid, double* x, double* wo, double* albedo, double* Ld) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, alb, tf, tf_n);
    const int NW = x_end - x_begin;
    std::vector<Light> L = mklights(lkind, lv, lrgb, n_lights);
    CamFrame cf = cam_frame(eye, at, up, fovy, W, H);
    Grid<double> G64 = fp32 ? Grid<double>() : build_grid<double>(V, brick);
    Grid<float> G32 = fp32 ? build_grid<float>(V, brick) : Grid<float>();
    const int f = brick_primary > brick ? brick_primary / brick : 1;
    Grid<double> P64 = pool_grid(G64, f);
    Grid<float> P32 = pool_grid(G32, f);
    const int fs = brick_shadow > brick ? brick_shadow / brick : 1;
    Grid<double> S64 = pool_grid(G64, fs);
    Grid<float> S32 = pool_grid(G32, fs);
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int py = y_begin; py < y_end; ++py)
        for (int px = x_begin; px < x_end; ++px)
            for (int k = 0; k < spp; ++k) {
                size_t idx = (((size_t)(py - y_begin) * NW + (px - x_begin)) * spp + k);
                int vld;
                if (fp32) {
                    V3<float> a, b, c, e;
                    camera_sample<float>(V, G32, P32, S32, L.data(), n_lights, (float)g, cf, px, py, k, (float)step_vox, seed, &vld, &a, &b, &c, &e);
                    x[3 * idx] = a.x; x[3 * idx + 1] = a.y; x[3 * idx + 2] = a.z;
                    wo[3 * idx] = b.x; wo[3 * idx + 1] = b.y; wo[3 * idx + 2] = b.z;
                    albedo[3 * idx] = c.x; albedo[3 * idx + 1] = c.y; albedo[3 * idx + 2] = c.z;
                    Ld[3 * idx] = e.x; Ld[3 * idx + 1] = e.y; Ld[3 * idx + 2] = e.z;
                } else {
                    V3<double> a, b, c, e;
                    camera_sample<double>(V, G64, P64, S64, L.data(), n_lights, g, cf, px, py, k, step_vox, seed, &vld, &a, &b, &c, &e);
                    x[3 * idx] = a.x; x[3 * idx + 1] = a.y; x[3 * idx + 2] = a.z;
                    wo[3 * idx] = b.x; wo[3 * idx + 1] = b.y; wo[3 * idx + 2] = b.z;
                    albedo[3 * idx] = c.x; albedo[3 * idx + 1] = c.y; albedo[3 * idx + 2] = c.z;
                    Ld[3 * idx] = e.x; Ld[3 * idx + 1] = e.y; Ld[3 * idx + 2] = e.z;
                }
                valid[idx] = (uint8_t)vld;
            }
}

// Path-traced image rows [y_begin, y_end): out[(y-y_begin)][x][3], the
// per-pixel mean over spp samples accumulated in sample order; or an explicit
// list of (x, y) pixels.
void orc_path_trace(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb,
                    const float* tf, int tf_n, int brick,
                    const int* lkind, const double* lv, const double* lrgb, int n_lights, double g,
                    const double* eye, const double* at, const double* up, double fovy, int W, int H,
                    int spp, int max_bounces, uint64_t seed, int use_rr, int fp32, int y_begin, int y_end,
                    const int32_t* px_list, int64_t n_px, double* out) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, alb, tf, tf_n);
    std::vector<Light> L = mklights(lkind, lv, lrgb, n_lights);
    CamFrame cf = cam_frame(eye, at, up, fovy, W, H);
    Grid<double> G64 = fp32 ? Grid<double>() : build_grid<double>(V, brick);
    Grid<float> G32 = fp32 ? build_grid<float>(V, brick) : Grid<float>();
    int64_t n_items = px_list ? n_px : (int64_t)(y_end - y_begin) * W;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t it = 0; it < n_items; ++it) {
        int px, py;
        if (px_list) { px = px_list[2 * it]; py = px_list[2 * it + 1]; }
        else { py = y_begin + (int)(it / W); px = (int)(it % W); }
        if (fp32) {
            float acc[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < spp; ++k) {
                V3<float> r = path_sample<float>(V, G32, L.data(), n_lights, (float)g, cf, px, py, k, max_bounces, seed, use_rr);
                acc[0] = acc[0] + r.x; acc[1] = acc[1] + r.y; acc[2] = acc[2] + r.z;
            }
            for (int c = 0; c < 3; ++c) out[3 * it + c] = (double)(acc[c] / (float)spp);
        } else {
            double acc[3] = {0, 0, 0};
            for (int k = 0; k < spp; ++k) {
                V3<double> r = path_sample<double>(V, G64, L.data(), n_lights, g, cf, px, py, k, max_bounces, seed, use_rr);
                acc[0] += r.x; acc[1] += r.y; acc[2] += r.z;
            }
            for (int c = 0; c < 3; ++c) out[3 * it + c] = acc[c] / spp;
        }
    }
}

// Mean sigma_t over the fine voxel centres inside each cache cell (cells
// without a voxel centre take sigma_t at the cell centre).
void orc_cell_sigma(int nx, int ny, int nz, int dtype, const void* data, double ss, const float* tf, int tf_n,
                    int res, double* out) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, 1.0, tf, tf_n);
    size_t nc = (size_t)res * res * res;
    std::vector<double> sum(nc, 0.0);
    std::vector<int64_t> cnt(nc, 0);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                // cell holding the voxel centre (i+1/2)/n: floor((2i+1)*res / 2n)
                int cx = (int)(((int64_t)(2 * i + 1) * res) / (2 * (int64_t)nx));
                int cy = (int)(((int64_t)(2 * j + 1) * res) / (2 * (int64_t)ny));
                int cz = (int)(((int64_t)(2 * k + 1) * res) / (2 * (int64_t)nz));
                size_t c = (size_t)cx + (size_t)res * ((size_t)cy + (size_t)res * cz);
                sum[c] += ss * tf_at<double>(V, voxel<double>(V, i, j, k), 3);
                cnt[c] += 1;
            }
    for (size_t c = 0; c < nc; ++c) {
        if (cnt[c] > 0) out[c] = sum[c] / (double)cnt[c];
        else {
            int cx = (int)(c % res), cy = (int)((c / res) % res), cz = (int)(c / ((size_t)res * res));
            out[c] = sigma_at<double>(V, v3((cx + 0.5) / res, (cy + 0.5) / res, (cz + 0.5) / res));
        }
    }
}

// Grid-cell radiance estimate (the paper's KNN estimator with the cache cell
// as the gather region): for query b with position x, outgoing direction w
// and phase index gi,
//   L_s = sum_l sum_{records n in (l, gi, bin(x))} p_g(dir_n . w) Phi_n / (V_cell * sigma_cell)
// Records are given as CSR over keys (l*n_g + gi)*res^3 + bin.
void orc_estimate(const double* x, const double* w, const int* gi, int64_t B,
                  const int64_t* offsets, const float* rdir, const float* rphi,
                  const double* cell_sigma, const float* gset, int n_g, int n_lights, int res, double* out) {
    int64_t nc = (int64_t)res * res * res;
    double vcell = 1.0 / (double)nc;
    #pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; ++b) {
        // bin of the float32 query position, decided in float32 as the kernel does
        int bx = std::min(std::max((int)std::floor((float)x[3 * b] * (float)res), 0), res - 1);
        int by = std::min(std::max((int)std::floor((float)x[3 * b + 1] * (float)res), 0), res - 1);
        int bz = std::min(std::max((int)std::floor((float)x[3 * b + 2] * (float)res), 0), res - 1);
        int64_t cell = bx + (int64_t)res * (by + (int64_t)res * bz);
        double g = gset[gi[b]];
        double acc[3] = {0, 0, 0};
        for (int l = 0; l < n_lights; ++l) {
            int64_t key = (int64_t)(l * n_g + gi[b]) * nc + cell;
            for (int64_t n = offsets[key]; n < offsets[key + 1]; ++n) {
                double mu = rdir[3 * n] * w[3 * b] + rdir[3 * n + 1] * w[3 * b + 1] + rdir[3 * n + 2] * w[3 * b + 2];
                double p = hg_eval<double>(g, mu);
                for (int c = 0; c < 3; ++c) acc[c] += p * (double)rphi[3 * n + c];
            }
        }
        double s = cell_sigma[cell];
        for (int c = 0; c < 3; ++c) out[3 * b + c] = s > 0 ? acc[c] / (vcell * s) : 0.0;
    }
}


// Phase-selective k-nearest-neighbour radiance estimate (Sec. 3.3.1: the
// adaptive-radius estimator of Jensen and Christensen over the photons of the
// query's phase only, K nearest, search radius capped at r_max).
// For query b at float32 position x, outgoing direction w and phase index gi:
//   candidates: every record n of phase gi (any light) with
//     d2_n = ((x_n - x)^2 + (y_n - y)^2) + (z_n - z)^2 <= r_max^2,
//     each difference, square and sum a float32 operation;
//   ordered by (d2_n, record id); the first k = min(K, #candidates) are used;
//   r = sqrt(d2) of the K-th if #candidates >= K (the K nearest lie inside
//     the cap), else r_max (fewer than K photons: the estimate covers the
//     whole ball searched);
//   L_s = sum_{used n} p_g(dir_n . w) Phi_n / ((4/3) pi r^3 sigma_cell(x)),
//     sigma_cell(x) = mean sigma_t of the cache cell holding x (the same
//     normaliser as the cache-cell estimate), and L_s = 0 if r or sigma is 0.
// Brute force over all records: no spatial index.  k_out, r_out nullable.
void orc_estimate_knn(const float* xq, const double* w, const int* gi, int64_t B,
                      const float* rpos, const uint32_t* rid, const int* rphase, const float* rdir,
                      const float* rphi, int64_t n_rec, int K, float r_max, const double* cell_sigma,
                      const float* gset, int res, double* out, int* k_out, float* r_out) {
    const double pi = 3.14159265358979323846;
    float r2max = r_max * r_max;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < B; ++b) {
        float qx = xq[3 * b], qy = xq[3 * b + 1], qz = xq[3 * b + 2];
        struct Cand { float d2; uint32_t id; int64_t n; };
        std::vector<Cand> cand;
        for (int64_t n = 0; n < n_rec; ++n) {
            if (rphase[n] != gi[b]) continue;
            float dx = rpos[3 * n] - qx, dy = rpos[3 * n + 1] - qy, dz = rpos[3 * n + 2] - qz;
            float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 <= r2max) cand.push_back(Cand{d2, rid[n], n});
        }
        std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& c) {
            return a.d2 < c.d2 || (a.d2 == c.d2 && a.id < c.id);
        });
        int64_t k = std::min<int64_t>((int64_t)K, (int64_t)cand.size());
        float r = (int64_t)cand.size() >= (int64_t)K && K > 0 ? std::sqrt(cand[(size_t)K - 1].d2) : r_max;
        double g = gset[gi[b]];
        double acc[3] = {0, 0, 0};
        for (int64_t i = 0; i < k; ++i) {
            int64_t n = cand[(size_t)i].n;
            double mu = (double)rdir[3 * n] * w[3 * b] + (double)rdir[3 * n + 1] * w[3 * b + 1] +
                        (double)rdir[3 * n + 2] * w[3 * b + 2];
            double p = hg_eval<double>(g, mu);
            for (int c = 0; c < 3; ++c) acc[c] += p * (double)rphi[3 * n + c];
        }
        int bx = std::min(std::max((int)std::floor(qx * (float)res), 0), res - 1);
        int by = std::min(std::max((int)std::floor(qy * (float)res), 0), res - 1);
        int bz = std::min(std::max((int)std::floor(qz * (float)res), 0), res - 1);
        double s = cell_sigma[bx + (int64_t)res * (by + (int64_t)res * bz)];
        double vol = 4.0 / 3.0 * pi * (double)r * (double)r * (double)r;
        for (int c = 0; c < 3; ++c) out[3 * b + c] = (s > 0 && r > 0) ? acc[c] / (vol * s) : 0.0;
        if (k_out) k_out[b] = (int)k;
        if (r_out) r_out[b] = r;
    }
}


// Ray-marched render of rows [y_begin, y_end): per camera sample (ray r =
// ((py - y_begin) W + px) spp + k) the direct part D[r] and the number of
// field queries count[r]; with offsets (exclusive sums of count, nullable)
// also the queries q [..][6] and weights w [..][3] at offsets[r].
void orc_raymarch(int nx, int ny, int nz, int dtype, const void* data, double ss, double alb,
                  const float* tf, int tf_n, const int* lkind, const double* lv, const double* lrgb, int n_lights,
                  double g, const double* eye, const double* at, const double* up, double fovy, int W, int H,
                  int spp, double step_vox, uint64_t seed, int y_begin, int y_end,
                  double* D, int64_t* count, const int64_t* offsets, double* q, double* w) {
    Volume V = mkvol(nx, ny, nz, dtype, data, ss, alb, tf, tf_n);
    std::vector<Light> L = mklights(lkind, lv, lrgb, n_lights);
    CamFrame cf = cam_frame(eye, at, up, fovy, W, H);
    const double h = step_vox / (double)std::max(nx, std::max(ny, nz));
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int py = y_begin; py < y_end; ++py)
        for (int px = 0; px < W; ++px)
            for (int k = 0; k < spp; ++k) {
                const size_t r = ((size_t)(py - y_begin) * W + px) * spp + k;
                double* qq = offsets ? q + 6 * offsets[r] : nullptr;
                double* ww = offsets ? w + 3 * offsets[r] : nullptr;
                count[r] = raymarch_ray(V, L.data(), n_lights, g, cf, px, py, k, h, seed, D + 3 * r, qq, ww);
            }
}
}  // extern "C"
