// Device code of the residual path integral estimator (arXiv 2406.16302).
//
// One thread owns one root of one technique in one frame: it samples the
// root (a point x_D on the edited object, Sec. 4.1, or a camera ray for path
// tracing, Sec. 4.3), performs the random walks with next-event estimation
// and sensor connections, and for every base path it produces: evaluates its
// contribution f (Eq. pathcontribution), the balance-heuristic denominator
// over all techniques (Sec. 4.3, forward/backward pdf tables), maps it into
// the other frame (Sec. 5) and splats the two-way mapped contribution into
// an FP64 image.  BVH traversal (two-level: static BVH, dynamic BVH under a
// per-frame rigid transform) uses a shared-memory stack and the watertight
// ray/triangle test of Woop, Benthin and Wald (JCGT 2013).
//
// Geometry and shading are FP32; the image accumulates in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rp_internal.h"

#ifndef RP_WALK_FP64
#define RP_WALK_FP64 0
#endif
#ifndef RP_REFINE_FP64
#define RP_REFINE_FP64 1
#endif
#ifndef RP_TRACE_MINBLOCKS
#define RP_TRACE_MINBLOCKS 8
#endif

namespace rp {

// ---------------------------------------------------------------------------
// vectors
// ---------------------------------------------------------------------------

static __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
static __device__ __forceinline__ float3 operator+(float3 a, float3 b) {
    return f3(a.x + b.x, a.y + b.y, a.z + b.z);
}
static __device__ __forceinline__ float3 operator-(float3 a, float3 b) {
    return f3(a.x - b.x, a.y - b.y, a.z - b.z);
}
static __device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
static __device__ __forceinline__ float3 mul3(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
static __device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static __device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
static __device__ __forceinline__ float3 unit3(float3 a) { return a * (1.0f / sqrtf(dot3(a, a))); }
static __device__ __forceinline__ bool zero3(float3 a) { return a.x == 0.f && a.y == 0.f && a.z == 0.f; }
static __device__ __forceinline__ bool same3(float3 a, float3 b) {
    return a.x == b.x && a.y == b.y && a.z == b.z;
}
static __device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
static __device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }

static __device__ __forceinline__ float3 affine(const float *M, float3 p) {
    return f3(M[0] * p.x + M[1] * p.y + M[2] * p.z + M[3],
              M[4] * p.x + M[5] * p.y + M[6] * p.z + M[7],
              M[8] * p.x + M[9] * p.y + M[10] * p.z + M[11]);
}
static __device__ __forceinline__ float3 linear(const float *M, float3 p) {
    return f3(M[0] * p.x + M[1] * p.y + M[2] * p.z, M[4] * p.x + M[5] * p.y + M[6] * p.z,
              M[8] * p.x + M[9] * p.y + M[10] * p.z);
}

constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;

// double-precision vectors: path vertices and sampled directions are
// constructed in FP64 and rounded to FP32 once
static __device__ __forceinline__ double3 d3(double x, double y, double z) { return make_double3(x, y, z); }
static __device__ __forceinline__ double3 d3(float3 v) { return make_double3(v.x, v.y, v.z); }
static __device__ __forceinline__ double3 d3(float4 v) { return make_double3(v.x, v.y, v.z); }
static __device__ __forceinline__ double3 dadd(double3 a, double3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
static __device__ __forceinline__ double3 dsub(double3 a, double3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
static __device__ __forceinline__ double3 dscale(double3 a, double s) { return d3(a.x * s, a.y * s, a.z * s); }
static __device__ __forceinline__ double ddot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static __device__ __forceinline__ double3 dcross(double3 a, double3 b) {
    return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static __device__ __forceinline__ double3 dunit(double3 a) { return dscale(a, 1.0 / sqrt(ddot(a, a))); }
static __device__ __forceinline__ float3 tof(double3 a) { return make_float3((float)a.x, (float)a.y, (float)a.z); }
static __device__ __forceinline__ double3 daffine(const float *M, double3 p) {
    return d3(M[0] * p.x + M[1] * p.y + M[2] * p.z + M[3], M[4] * p.x + M[5] * p.y + M[6] * p.z + M[7],
              M[8] * p.x + M[9] * p.y + M[10] * p.z + M[11]);
}
static __device__ __forceinline__ double3 dlinear(const float *M, double3 p) {
    return d3(M[0] * p.x + M[1] * p.y + M[2] * p.z, M[4] * p.x + M[5] * p.y + M[6] * p.z,
              M[8] * p.x + M[9] * p.y + M[10] * p.z);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11)
// ---------------------------------------------------------------------------

static __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

enum { T_PT = 0, T_1 = 1, T_2 = 2, T_3 = 3, T_4 = 4, T_5 = 5, T_6 = 6, T_7 = 7 };
enum { SD_ROOT = 0, SD_EYE = 1, SD_LIGHT = 2, SD_NEE = 3 };

// four uniforms in [0, 1) on a 2^-24 grid, keyed by what they are used for
// the launch's seed (batched launches read it from device memory so that a
// captured graph can be replayed with new seeds)
static __device__ __forceinline__ uint64_t lseed(const LaunchArgs &a) {
    return a.seed_dev ? (uint64_t)*a.seed_dev : a.seed;
}

static __device__ __forceinline__ float4 draw(uint64_t seed, uint32_t root, int tech, int frame, int side,
                                       int step) {
    uint4 c = make_uint4(root, ((uint32_t)tech << 24) | ((uint32_t)frame << 20) |
                                   ((uint32_t)side << 16) | (uint32_t)step, 0u, 0u);
    uint4 r = philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float s = 1.0f / 16777216.0f;
    return make_float4((float)(r.x >> 8) * s, (float)(r.y >> 8) * s, (float)(r.z >> 8) * s,
                       (float)(r.w >> 8) * s);
}

// ---------------------------------------------------------------------------
// materials
// ---------------------------------------------------------------------------

constexpr int kMatCamera = -1;
constexpr int kMatDynamic = -2;      // object k of the edit's dynamic set: kMatDynamic - k

struct Mat {
    int type;
    float3 alb;
    float alpha;
    float3 f0;
    float3 em;
};

static __device__ __forceinline__ Mat load_mat(const float *r) {
    Mat m;
    m.type = (int)r[0];
    m.alb = f3(r[1], r[2], r[3]);
    m.alpha = r[4];
    m.f0 = f3(r[5], r[6], r[7]);
    m.em = f3(r[8], r[9], r[10]);
    return m;
}

struct Ctx;
static __device__ Mat get_mat(const Ctx &c, int frame, int mat);

static __device__ __forceinline__ bool mat_black(const Mat &m) {
    return m.type == 0 ? zero3(m.alb) : zero3(m.f0);
}
static __device__ __forceinline__ float mat_rough(const Mat &m) {
    return m.type == 0 ? __int_as_float(0x7f800000) : m.alpha;
}

// ---------------------------------------------------------------------------
// tangent frame: branchless orthonormal basis (Duff et al., JCGT 2017) built
// in a fixed generic rotation, so axis-aligned normals never sit on its seam
// ---------------------------------------------------------------------------

static __device__ __forceinline__ void tangent_frame(float3 n, float3 &t, float3 &b) {
    const float q00 = 0.727128712871287f, q01 = -0.16910891089108918f, q02 = 0.6653465346534656f;
    const float q10 = 0.44356435643564374f, q11 = 0.85544554455445543f, q12 = -0.26732673267326734f;
    const float q20 = -0.52396039603960409f, q21 = 0.48950495049504961f, q22 = 0.69702970297029698f;
    float3 m = f3(q00 * n.x + q01 * n.y + q02 * n.z, q10 * n.x + q11 * n.y + q12 * n.z,
                  q20 * n.x + q21 * n.y + q22 * n.z);
    float sg = m.z >= 0.0f ? 1.0f : -1.0f;
    float a = -1.0f / (sg + m.z);
    float c = m.x * m.y * a;
    float3 tl = f3(1.0f + sg * m.x * m.x * a, sg * c, -sg * m.x);
    float3 bl = f3(c, sg + m.y * m.y * a, -m.y);
    t = f3(q00 * tl.x + q10 * tl.y + q20 * tl.z, q01 * tl.x + q11 * tl.y + q21 * tl.z,
           q02 * tl.x + q12 * tl.y + q22 * tl.z);
    b = f3(q00 * bl.x + q10 * bl.y + q20 * bl.z, q01 * bl.x + q11 * bl.y + q21 * bl.z,
           q02 * bl.x + q12 * bl.y + q22 * bl.z);
}

// ---------------------------------------------------------------------------
// BSDFs: Lambert; GGX reflection (Walter et al. 2007), separable Smith,
// Schlick Fresnel.  Directions are unit vectors leaving the surface.
// ---------------------------------------------------------------------------

static __device__ __forceinline__ float ggx_D(float a2, float ch) {
    float k = ch * ch * (a2 - 1.0f) + 1.0f;
    return a2 / (kPi * k * k);
}
static __device__ __forceinline__ float ggx_G1(float a2, float c) {
    return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

static __device__ float3 bsdf_eval(const Mat &m, float3 n, float3 wi, float3 wo) {
    float ci = dot3(n, wi), co = dot3(n, wo);
    if (ci <= 0.f || co <= 0.f) return f3(0, 0, 0);
    if (m.type == 0) return m.alb * (1.0f / kPi);
    float a2 = m.alpha * m.alpha;
    float3 h = unit3(wi + wo);
    float ch = dot3(n, h), ih = dot3(wi, h);
    if (ch <= 0.f || ih <= 0.f) return f3(0, 0, 0);
    float x = 1.0f - ih;
    float x2 = x * x;
    float fw = x2 * x2 * x;
    float3 F = f3(m.f0.x + (1.f - m.f0.x) * fw, m.f0.y + (1.f - m.f0.y) * fw,
                  m.f0.z + (1.f - m.f0.z) * fw);
    float s = ggx_D(a2, ch) * ggx_G1(a2, ci) * ggx_G1(a2, co) / (4.0f * ci * co);
    return F * s;
}

// solid-angle density of sampling wo with conditioning direction wc
static __device__ float bsdf_pdf(const Mat &m, float3 n, float3 wc, float3 wo) {
    float cc = dot3(n, wc), co = dot3(n, wo);
    if (cc <= 0.f || co <= 0.f) return 0.f;
    if (m.type == 0) return co * (1.0f / kPi);
    float a2 = m.alpha * m.alpha;
    float3 h = unit3(wc + wo);
    float ch = dot3(n, h), oh = dot3(wo, h);
    if (ch <= 0.f || oh <= 0.f) return 0.f;
    return ggx_D(a2, ch) * ch / (4.0f * oh);
}

static __device__ __forceinline__ float cosine_pdf(float3 n, float3 w) {
    float c = dot3(n, w);
    return c > 0.f ? c * (1.0f / kPi) : 0.f;
}

// tangent frame in double precision (same construction as tangent_frame)
static __device__ __forceinline__ void tangent_frame_d(double3 n, double3 &t, double3 &b) {
    const double q00 = 0.727128712871287, q01 = -0.16910891089108918, q02 = 0.6653465346534656;
    const double q10 = 0.44356435643564374, q11 = 0.85544554455445543, q12 = -0.26732673267326734;
    const double q20 = -0.52396039603960409, q21 = 0.48950495049504961, q22 = 0.69702970297029698;
    double3 m = d3(q00 * n.x + q01 * n.y + q02 * n.z, q10 * n.x + q11 * n.y + q12 * n.z,
                   q20 * n.x + q21 * n.y + q22 * n.z);
    double sg = m.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + m.z);
    double c = m.x * m.y * a;
    double3 tl = d3(1.0 + sg * m.x * m.x * a, sg * c, -sg * m.x);
    double3 bl = d3(c, sg + m.y * m.y * a, -m.y);
    t = d3(q00 * tl.x + q10 * tl.y + q20 * tl.z, q01 * tl.x + q11 * tl.y + q21 * tl.z,
           q02 * tl.x + q12 * tl.y + q22 * tl.z);
    b = d3(q00 * bl.x + q10 * bl.y + q20 * bl.z, q01 * bl.x + q11 * bl.y + q21 * bl.z,
           q02 * bl.x + q12 * bl.y + q22 * bl.z);
}

// cos and sin of 2 pi u in double precision: uniforms on the 2^-24 grid use
// the angle-addition tables of the scene, other angles sincospi
static __device__ __forceinline__ void sincos2pi(const DevScene &S, double u, double &s, double &c) {
    const double k = u * 16777216.0;
    if (k == floor(k) && k >= 0.0 && k < 16777216.0 && S.cs_hi) {
        const uint32_t ki = (uint32_t)k;
        const double2 a = __ldg(&S.cs_hi[ki >> 12]), b = __ldg(&S.cs_lo[ki & 4095u]);
        c = a.x * b.x - a.y * b.y;
        s = a.y * b.x + a.x * b.y;
        return;
    }
    sincospi(2.0 * u, &s, &c);
}

// cosine-distributed direction about n for (u1, u2), in double precision
static __device__ double3 cosine_dir_d(const DevScene &S, double3 n, double u1, double u2) {
    double3 t, b;
    tangent_frame_d(n, t, b);
    double r = sqrt(u1), sp, cp;
    sincos2pi(S, u2, sp, cp);
    double z = sqrt(fmax(0.0, 1.0 - u1));
    return dadd(dadd(dscale(t, r * cp), dscale(b, r * sp)), dscale(n, z));
}

static __device__ float3 cosine_dir(const DevScene &S, float3 n, double u1, double u2) {
    return tof(cosine_dir_d(S, d3(n), u1, u2));
}

static __device__ void cosine_inverse(float3 n, float3 w, double &u1, double &u2) {
    double3 t, b;
    tangent_frame_d(d3(n), t, b);
    double3 wd = d3(w);
    double x = ddot(wd, t), y = ddot(wd, b);
    u1 = x * x + y * y;
    double a = atan2(y, x) / (2.0 * kPiD);
    u2 = a < 0.0 ? a + 1.0 : a;
}

// sample wo at a surface with conditioning direction wc; false on failure
static __device__ bool bsdf_sample(const DevScene &S, const Mat &m, float3 n, float3 wc, double u1,
                                   double u2, float3 &wo) {
    const double3 nd = d3(n), wcd = d3(wc);
    if (ddot(nd, wcd) <= 0.0) return false;
    if (m.type == 0) {
        double3 w = cosine_dir_d(S, nd, u1, u2);
        if (ddot(nd, w) <= 0.0) return false;
        wo = tof(w);
        return true;
    }
    double a2 = (double)m.alpha * (double)m.alpha;
    double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
    double ct = sqrt(c2), st = sqrt(fmax(0.0, 1.0 - c2)), sp, cp;
    sincos2pi(S, u2, sp, cp);
    double3 t, b;
    tangent_frame_d(nd, t, b);
    double3 h = dadd(dadd(dscale(t, st * cp), dscale(b, st * sp)), dscale(nd, ct));
    double d = ddot(wcd, h);
    if (d <= 0.0) return false;
    double3 w = dsub(dscale(h, 2.0 * d), wcd);
    if (ddot(nd, w) <= 0.0) return false;
    wo = tof(w);
    return true;
}

// the same sampler in single precision, for the random walks (uniforms on
// the 2^-24 grid, trigonometry by sincospif)
static __device__ bool bsdf_sample_walk(const DevScene &S, const Mat &m, float3 n, float3 wc, float u1,
                                        float u2, float3 &wo) {
#if RP_WALK_FP64
    return bsdf_sample(S, m, n, wc, u1, u2, wo);
#else
    (void)S;
    if (dot3(n, wc) <= 0.f) return false;
    float3 t, b;
    tangent_frame(n, t, b);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    if (m.type == 0) {
        float r = sqrtf(u1), z = sqrtf(fmaxf(0.f, 1.0f - u1));
        wo = t * (r * cp) + b * (r * sp) + n * z;
        return dot3(n, wo) > 0.f;
    }
    float a2 = m.alpha * m.alpha;
    float c2 = (1.0f - u1) / (1.0f + (a2 - 1.0f) * u1);
    float ct = sqrtf(c2), st = sqrtf(fmaxf(0.f, 1.0f - c2));
    float3 h = t * (st * cp) + b * (st * sp) + n * ct;
    float d = dot3(wc, h);
    if (d <= 0.f) return false;
    wo = h * (2.0f * d) - wc;
    return dot3(n, wo) > 0.f;
#endif
}

static __device__ float3 cosine_dir_walk(const DevScene &S, float3 n, float u1, float u2) {
#if RP_WALK_FP64
    return cosine_dir(S, n, u1, u2);
#else
    (void)S;
    float3 t, b;
    tangent_frame(n, t, b);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    float r = sqrtf(u1), z = sqrtf(fmaxf(0.f, 1.0f - u1));
    return t * (r * cp) + b * (r * sp) + n * z;
#endif
}

// the numbers (u1, u2) for which bsdf_sample produces wo
static __device__ void bsdf_inverse(const Mat &m, float3 n, float3 wc, float3 wo, double &u1, double &u2) {
    if (m.type == 0) {
        cosine_inverse(n, wo, u1, u2);
        return;
    }
    double a2 = (double)m.alpha * (double)m.alpha;
    double3 h = dunit(dadd(d3(wc), d3(wo)));
    double3 t, b;
    tangent_frame_d(d3(n), t, b);
    double hx = ddot(h, t), hy = ddot(h, b), hz = ddot(h, d3(n));
    double c2 = hz * hz;
    u1 = (1.0 - c2) / (1.0 + c2 * (a2 - 1.0));
    double a = atan2(hy, hx) / (2.0 * kPiD);
    u2 = a < 0.0 ? a + 1.0 : a;
}

// ---------------------------------------------------------------------------
// traversal
// ---------------------------------------------------------------------------

struct Hit {
    float t, b1, b2;
    int prim;
    float3 p;      // closest hits: the intersection point recomputed in double
};

struct Counters {
    unsigned int nodes, tris, rays_closest, rays_shadow;
};

struct WtRay {
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

static __device__ __forceinline__ WtRay wt_setup(float3 d) {
    WtRay w;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    w.kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    w.kx = w.kz == 2 ? 0 : w.kz + 1;
    w.ky = w.kx == 2 ? 0 : w.kx + 1;
    float dz = comp(d, w.kz);
    if (dz < 0.f) {
        int tmp = w.kx;
        w.kx = w.ky;
        w.ky = tmp;
    }
    w.Sx = comp(d, w.kx) / dz;
    w.Sy = comp(d, w.ky) / dz;
    w.Sz = 1.0f / dz;
    return w;
}

// watertight ray/triangle test; t in (tmin, tmax); both faces
static __device__ __forceinline__ bool tri_hit(const WtRay &w, float3 o, float3 v0, float3 v1, float3 v2,
                                        float tmin, float tmax, float &t, float &b1, float &b2) {
    float3 A = v0 - o, B = v1 - o, C = v2 - o;
    float Az = comp(A, w.kz), Bz = comp(B, w.kz), Cz = comp(C, w.kz);
    float Ax = comp(A, w.kx) - w.Sx * Az, Ay = comp(A, w.ky) - w.Sy * Az;
    float Bx = comp(B, w.kx) - w.Sx * Bz, By = comp(B, w.ky) - w.Sy * Bz;
    float Cx = comp(C, w.kx) - w.Sx * Cz, Cy = comp(C, w.ky) - w.Sy * Cz;
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.f || V == 0.f || W == 0.f) {
        // edge or vertex hit: the 2D edge functions in double precision
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    float det = U + V + W;
    if (det == 0.f) return false;
    float T = U * (w.Sz * Az) + V * (w.Sz * Bz) + W * (w.Sz * Cz);
    float rcp = 1.0f / det;
    float tt = T * rcp;
    if (!(tt > tmin && tt < tmax)) return false;
    t = tt;
    b1 = V * rcp;
    b2 = W * rcp;
    return true;
}

static __device__ __forceinline__ bool box_hit(float lox, float hix, float loy, float hiy, float loz,
                                        float hiz, float3 id, float3 oid, float tmin, float tmax,
                                        float &tn) {
    float x0 = fmaf(lox, id.x, -oid.x), x1 = fmaf(hix, id.x, -oid.x);
    float y0 = fmaf(loy, id.y, -oid.y), y1 = fmaf(hiy, id.y, -oid.y);
    float z0 = fmaf(loz, id.z, -oid.z), z1 = fmaf(hiz, id.z, -oid.z);
    float a = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
    float b = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
    tn = a;
    return a <= b * 1.00000024f;
}

static __device__ __forceinline__ float safe_rcp(float x) {
    return 1.0f / (fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x);
}

// The path-level routines below that trace rays or walk a whole path
// (trace_next, segment_clear, ghost_prims, ghost_geom, path_throughput,
// mis_denominator, map_step) are kept out of line: the mapping kernel calls
// each from several places, and inlined copies of the traversal loop in
// every caller overflow the instruction cache when its lanes diverge.

// closest (any = false) or first found (any = true) hit in one BVH; leaf
// ids plus id_add are the global triangle ids.  Triangles with ids in
// [skip_lo, skip_lo + skip_n) (and, if skip_bits is set, whose bit
// id - skip_lo is set) are not there: the moved objects' base poses inside
// the static BVH
static __device__ bool traverse(const DevBVH &B, float3 o, float3 d, float tmin, float &tmax, int ex0,
                         int ex1, bool any, Hit &h, int *stack, Counters &cnt,
                         int *overflow, int id_add = 0, int skip_lo = 0, int skip_n = 0,
                         const uint32_t *skip_bits = nullptr) {
    if (B.n_nodes == 0) return false;
    // a ray with a non-finite component (the direction of two coincident
    // vertices) hits no triangle, but fminf/fmaxf drop its NaN slabs, so its
    // box tests would pass and it would walk most of the tree: stop here
    if (!(isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) &&
          isfinite(d.z)))
        return false;
    const WtRay w = wt_setup(d);
    const float3 id = f3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oid = f3(o.x * id.x, o.y * id.y, o.z * id.z);
    int sp = 0;
    int node = 0;
    bool found = false;
    for (;;) {
        ++cnt.nodes;
        const float4 na = __ldg(&B.nodes[4 * node + 0]);
        const float4 nb = __ldg(&B.nodes[4 * node + 1]);
        const float4 nc = __ldg(&B.nodes[4 * node + 2]);
        const float4 nd = __ldg(&B.nodes[4 * node + 3]);
        const int c0 = __float_as_int(nd.x), c1 = __float_as_int(nd.y);
        float t0, t1;
        bool h0 = box_hit(na.x, na.y, na.z, na.w, nc.x, nc.y, id, oid, tmin, tmax, t0);
        bool h1 = box_hit(nb.x, nb.y, nb.z, nb.w, nc.z, nc.w, id, oid, tmin, tmax, t1);
        for (int side = 0; side < 2; ++side) {
            const bool hs = side ? h1 : h0;
            const int cs = side ? c1 : c0;
            if (!hs || cs >= 0) continue;
            const int first = ~cs;
            const int count = __float_as_int(side ? nd.w : nd.z);
            for (int i = first; i < first + count; ++i) {
                ++cnt.tris;
                const float4 v0 = __ldg(&B.tris[3 * i + 0]);
                const int gid = __float_as_int(v0.w) + id_add;
                if (gid == ex0 || gid == ex1) continue;
                if ((unsigned)(gid - skip_lo) < (unsigned)skip_n &&
                    (!skip_bits ||
                     ((__ldg(&skip_bits[(unsigned)(gid - skip_lo) >> 5]) >> ((gid - skip_lo) & 31)) & 1u)))
                    continue;
                const float4 v1 = __ldg(&B.tris[3 * i + 1]);
                const float4 v2 = __ldg(&B.tris[3 * i + 2]);
                float tt, bb1, bb2;
                if (tri_hit(w, o, xyz(v0), xyz(v1), xyz(v2), tmin, tmax, tt, bb1, bb2)) {
                    tmax = tt;
                    h.t = tt;
                    h.b1 = bb1;
                    h.b2 = bb2;
                    h.prim = gid;
                    found = true;
                    if (any) return true;
                }
            }
        }
        const bool g0 = h0 && c0 >= 0, g1 = h1 && c1 >= 0;
        if (g0 && g1) {
            int nearc = c0, farc = c1;
            if (t1 < t0) {
                nearc = c1;
                farc = c0;
            }
            if (sp < kStackDepth) {
                stack[sp * kBlock] = farc;
                ++sp;
            } else {
                *overflow = 1;
            }
            node = nearc;
        } else if (g0) {
            node = c0;
        } else if (g1) {
            node = c1;
        } else {
            if (sp == 0) break;
            --sp;
            node = stack[sp * kBlock];
        }
    }
    return found;
}

// one out-of-line copy of the traversal loop for the path-level routines
static __device__ __noinline__ bool traverse_ol(const DevBVH &B, float3 o, float3 d, float tmin,
                                                float &tmax, int ex0, int ex1, bool any, Hit &h,
                                                int *stack, Counters &cnt, int *overflow, int id_add,
                                                int skip_lo, int skip_n, const uint32_t *skip_bits) {
    return traverse(B, o, d, tmin, tmax, ex0, ex1, any, h, stack, cnt, overflow, id_add, skip_lo,
                    skip_n, skip_bits);
}

// ---------------------------------------------------------------------------
// per-thread context
// ---------------------------------------------------------------------------

struct Ctx {
    const LaunchArgs &A;
    int *stack;
    Counters cnt;
    int overflow;
    __device__ Ctx(const LaunchArgs &a, int *s) : A(a), stack(s), cnt{0, 0, 0, 0}, overflow(0) {}
};

// the instance of a dynamic triangle id, and its object-space triangle
static __device__ __forceinline__ int inst_of(const DevScene &S, int prim) {
    const int l = prim - S.n_static;
    int k = 0;
#pragma unroll 1
    while (k + 1 < S.n_inst && l >= S.inst[k + 1].base) ++k;
    return k;
}

static __device__ __forceinline__ const float4 *dyn_tri_of(const DevScene &S, int prim, int &k) {
    k = inst_of(S, prim);
    return S.inst[k].tri + 3 * (prim - S.n_static - S.inst[k].base);
}

static __device__ __forceinline__ Mat get_mat(const Ctx &c, int frame, int mat) {
    if (mat <= kMatDynamic) return load_mat(c.A.E.mat(kMatDynamic - mat, frame));
    return load_mat(c.A.S.mats + 12 * mat);
}

// the closest hit recomputed in double: Moller-Trumbore on the hit triangle
// (in object space for the dynamic object), position rounded once
static __device__ void refine_hit(const Ctx &c, int g, float3 o, float3 d, Hit &h) {
    const DevScene &S = c.A.S;
#if !RP_REFINE_FP64
    {   // single precision: the point of the watertight barycentrics
        const bool dynp = h.prim >= S.n_static;
        int k = 0;
        const float4 *tr = dynp ? dyn_tri_of(S, h.prim, k) : S.stat_tri + 3 * h.prim;
        const float3 v0 = xyz(tr[0]);
        float3 p = v0 + (xyz(tr[1]) - v0) * h.b1 + (xyz(tr[2]) - v0) * h.b2;
        if (dynp) p = affine(c.A.E.M(k, g), p);
        h.p = p;
        return;
    }
#endif
    const bool dyn = h.prim >= S.n_static;
    int k = 0;
    const float4 *tri = dyn ? dyn_tri_of(S, h.prim, k) : S.stat_tri + 3 * h.prim;
    double3 od = d3(o), dd = d3(d);
    if (dyn) {
        od = daffine(c.A.E.Minv(k, g), od);
        dd = dlinear(c.A.E.Minv(k, g), dd);
    }
    const double3 v0 = d3(tri[0]), e1 = dsub(d3(tri[1]), v0), e2 = dsub(d3(tri[2]), v0);
    const double3 pv = dcross(dd, e2);
    const double det = ddot(e1, pv);
    if (det == 0.0) {
        h.p = o + d * h.t;
        return;
    }
    const double inv = 1.0 / det;
    const double3 sv = dsub(od, v0);
    const double u = ddot(sv, pv) * inv;
    const double3 qv = dcross(sv, e1);
    const double v = ddot(dd, qv) * inv;
    double3 p = dadd(dadd(v0, dscale(e1, u)), dscale(e2, v));
    if (dyn) p = daffine(c.A.E.M(k, g), p);
    h.p = tof(p);
    h.b1 = (float)u;
    h.b2 = (float)v;
}

// the segment o + t d, t in [tmin, tmax], passes within the radius of the
// bounding sphere bs (object space)
static __device__ __forceinline__ bool near_sphere(float4 bs, float3 o, float3 d, float tmin,
                                                   float tmax) {
    const float3 co = f3(bs.x, bs.y, bs.z) - o;
    const float tc = fminf(fmaxf(dot3(co, d), tmin), tmax);
    const float3 q = co - d * tc;
    return dot3(q, q) <= bs.w * bs.w;
}

// query of the scene in frame g: the static BVH, then each object of the
// dynamic set under its frame-g transform (a segment that misses an
// object's bounding sphere skips its BVH)
static __device__ bool scene_trace(Ctx &c, int g, float3 o, float3 d, float tmin, float tmax, int ex0,
                            int ex1, bool any, bool dyn_only, Hit &h) {
    const DevScene &S = c.A.S;
    bool found = false;
    if (!dyn_only) {
        found = traverse(S.stat, o, d, tmin, tmax, ex0, ex1, any, h, c.stack, c.cnt, &c.overflow,
                         0, c.A.E.skip_lo, c.A.E.skip_n, c.A.E.skip_bits);
        if (found && any) return true;
    }
    if (S.n_inst == 1) {
        // one object (the common edit): constant indexes keep its BVH
        // pointers and transform in the kernel's parameter bank
        const float *Mi = c.A.E.Minv(0, g);
        const float3 oo = affine(Mi, o), dd = linear(Mi, d);
        if (near_sphere(S.inst[0].bs, oo, dd, tmin, tmax) &&
            traverse(S.inst[0].bvh, oo, dd, tmin, tmax, ex0, ex1, any, h, c.stack, c.cnt,
                     &c.overflow))
            found = true;
    } else {
        for (int k = 0; k < S.n_inst; ++k) {
            const DevInst &I = S.inst[k];
            const float *Mi = c.A.E.Minv(k, g);
            const float3 oo = affine(Mi, o), dd = linear(Mi, d);
            if (near_sphere(I.bs, oo, dd, tmin, tmax) &&
                traverse(I.bvh, oo, dd, tmin, tmax, ex0, ex1, any, h, c.stack, c.cnt, &c.overflow,
                         I.base)) {
                found = true;
                if (any) return true;
            }
        }
    }
    if (found && !any) refine_hit(c, g, o, d, h);
    return found;
}

// scene_trace for the path-level routines: out of line, with one copy of
// the traversal loop for the static BVH and every object
static __device__ __noinline__ bool scene_trace_ol(Ctx &c, int g, float3 o, float3 d, float tmin,
                                                   float tmax, int ex0, int ex1, bool any,
                                                   bool dyn_only, Hit &h) {
    const DevScene &S = c.A.S;
    bool found = false;
    if (!dyn_only) {
        found = traverse_ol(S.stat, o, d, tmin, tmax, ex0, ex1, any, h, c.stack, c.cnt, &c.overflow,
                            0, c.A.E.skip_lo, c.A.E.skip_n, c.A.E.skip_bits);
        if (found && any) return true;
    }
    for (int k = 0; k < S.n_inst; ++k) {
        const DevInst &I = S.inst[k];
        const float *Mi = c.A.E.Minv(k, g);
        const float3 oo = affine(Mi, o), dd = linear(Mi, d);
        if (near_sphere(I.bs, oo, dd, tmin, tmax) &&
            traverse_ol(I.bvh, oo, dd, tmin, tmax, ex0, ex1, any, h, c.stack, c.cnt, &c.overflow,
                        I.base, 0, 0, nullptr)) {
            found = true;
            if (any) return true;
        }
    }
    if (found && !any) refine_hit(c, g, o, d, h);
    return found;
}

// every hit of a ray with t in (tmin, tmax) in one BVH, up to maxh (the
// ghost crossings of an edge); returns the number found
static __device__ int traverse_all(const DevBVH &B, float3 o, float3 d, float tmin, float tmax,
                                   float *ts, int *prims, int maxh, int *stack, Counters &cnt,
                                   int *overflow, int id_add) {
    if (B.n_nodes == 0) return 0;
    if (!(isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) &&
          isfinite(d.z)))
        return 0;                 // no crossings (see traverse)
    const WtRay w = wt_setup(d);
    const float3 id = f3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oid = f3(o.x * id.x, o.y * id.y, o.z * id.z);
    int sp = 0, node = 0, n = 0;
    for (;;) {
        ++cnt.nodes;
        const float4 na = __ldg(&B.nodes[4 * node + 0]);
        const float4 nb = __ldg(&B.nodes[4 * node + 1]);
        const float4 nc = __ldg(&B.nodes[4 * node + 2]);
        const float4 nd = __ldg(&B.nodes[4 * node + 3]);
        const int c0 = __float_as_int(nd.x), c1 = __float_as_int(nd.y);
        float t0, t1;
        const bool h0 = box_hit(na.x, na.y, na.z, na.w, nc.x, nc.y, id, oid, tmin, tmax, t0);
        const bool h1 = box_hit(nb.x, nb.y, nb.z, nb.w, nc.z, nc.w, id, oid, tmin, tmax, t1);
        for (int side = 0; side < 2; ++side) {
            const bool hs = side ? h1 : h0;
            const int cs = side ? c1 : c0;
            if (!hs || cs >= 0) continue;
            const int first = ~cs;
            const int count = __float_as_int(side ? nd.w : nd.z);
            for (int i = first; i < first + count; ++i) {
                ++cnt.tris;
                const float4 v0 = __ldg(&B.tris[3 * i + 0]);
                const float4 v1 = __ldg(&B.tris[3 * i + 1]);
                const float4 v2 = __ldg(&B.tris[3 * i + 2]);
                float tmx = tmax, tt, bb1, bb2;
                if (tri_hit(w, o, xyz(v0), xyz(v1), xyz(v2), tmin, tmx, tt, bb1, bb2) && n < maxh) {
                    ts[n] = tt;
                    prims[n] = __float_as_int(v0.w) + id_add;
                    ++n;
                }
            }
        }
        const bool g0 = h0 && c0 >= 0, g1 = h1 && c1 >= 0;
        if (g0 && g1) {
            if (sp < kStackDepth) {
                stack[sp * kBlock] = c1;
                ++sp;
            } else {
                *overflow = 1;
            }
            node = c0;
        } else if (g0) {
            node = c0;
        } else if (g1) {
            node = c1;
        } else {
            if (sp == 0) break;
            --sp;
            node = stack[sp * kBlock];
        }
    }
    return n;
}

constexpr int kMaxCross = 8;        // ghost crossings kept per edge

// ghost_prims: the triangles of the ghost (the edited objects at their pose
// of the other frame, Sec. 3.3) that the open segment a-b of frame g
// crosses, up to kMaxCross, with their distances.
static __device__ __noinline__ int ghost_prims(Ctx &c, int g, float3 a, float3 b, float *ts, int *prims) {
    const DevScene &S = c.A.S;
    if (!c.A.E.motion) return 0;
    const int go = 3 - g;
    const float3 e = b - a;
    const float dist = len3(e);
    const float3 d = e * (1.0f / dist);
    const float tmin = S.eps, tmax = dist - S.eps;
    int n = 0;
    for (int k = 0; k < S.n_inst && n < kMaxCross; ++k) {
        const DevInst &I = S.inst[k];
        const float *Mi = c.A.E.Minv(k, go);
        const float3 oo = affine(Mi, a), dd = linear(Mi, d);
        if (!near_sphere(I.bs, oo, dd, tmin, tmax)) continue;
        n += traverse_all(I.bvh, oo, dd, tmin, tmax, ts + n, prims + n, kMaxCross - n, c.stack,
                          c.cnt, &c.overflow, I.base);
    }
    return n;
}

// the crossing of the segment from da along unit dw with ghost triangle
// prim (frame-go pose), re-solved in double on the triangle's plane
// (tfall: the distance to use if the segment lies in the plane)
static __device__ __forceinline__ void ghost_resolve(const Ctx &c, int go, double3 da, double3 dw,
                                                     int prim, double tfall, double3 &cp,
                                                     double3 &cn) {
    int k;
    const float4 *tr = dyn_tri_of(c.A.S, prim, k);
    const float *M = c.A.E.M(k, go);
    const double3 v0 = daffine(M, d3(tr[0])), v1 = daffine(M, d3(tr[1])), v2 = daffine(M, d3(tr[2]));
    const double3 nn = dcross(dsub(v1, v0), dsub(v2, v0));
    const double den = ddot(nn, dw);
    const double t = den != 0.0 ? ddot(nn, dsub(v0, da)) / den : tfall;
    cp = dadd(da, dscale(dw, t));
    cn = dunit(nn);
}

// ---------------------------------------------------------------------------
// path vertices
// ---------------------------------------------------------------------------

struct Vtx {
    float3 p, n;
    int prim;      // -1: the pinhole
    int mat;       // material index, kMatCamera, or kMatDynamic - k on object k of the edit
    float b1, b2;
};

static __device__ __forceinline__ bool is_dyn(const Ctx &c, const Vtx &v) {
    return v.prim >= c.A.S.n_static;
}

// the surface point with barycentrics (b1, b2) on triangle `prim` in frame
// g, combined in double and rounded once; unit normals come from the scene
// tables (computed in double on the host, stored in the .w slots)
static __device__ Vtx make_vertex_d(const Ctx &c, int g, int prim, double b1, double b2) {
    const DevScene &S = c.A.S;
    Vtx v;
    if (prim < S.n_static) {
        const float4 a = S.stat_tri[3 * prim], b = S.stat_tri[3 * prim + 1],
                     d = S.stat_tri[3 * prim + 2];
        double3 v0 = d3(a);
        v.p = tof(dadd(dadd(v0, dscale(dsub(d3(b), v0), b1)), dscale(dsub(d3(d), v0), b2)));
        v.n = f3(a.w, b.w, d.w);
        v.mat = (int)S.stat_mat[prim];
    } else {
        int k;
        const float4 *tr = dyn_tri_of(S, prim, k);
        const float4 a = tr[0], b = tr[1], d = tr[2];
        double3 v0 = d3(a);
        double3 po = dadd(dadd(v0, dscale(dsub(d3(b), v0), b1)), dscale(dsub(d3(d), v0), b2));
        const float *M = c.A.E.M(k, g);
        v.p = tof(daffine(M, po));
        v.n = tof(dlinear(M, d3(a.w, b.w, d.w)));
        v.mat = kMatDynamic - k;
    }
    v.prim = prim;
    v.b1 = (float)b1;
    v.b2 = (float)b2;
    return v;
}

static __device__ __forceinline__ Vtx make_vertex(const Ctx &c, int g, int prim, float b1, float b2) {
    return make_vertex_d(c, g, prim, (double)b1, (double)b2);
}

// a vertex at a known (refined) position p on triangle `prim`
static __device__ Vtx make_vertex_at(const Ctx &c, int g, int prim, float b1, float b2, float3 p) {
    const DevScene &S = c.A.S;
    Vtx v;
    if (prim < S.n_static) {
        v.n = f3(S.stat_tri[3 * prim].w, S.stat_tri[3 * prim + 1].w, S.stat_tri[3 * prim + 2].w);
        v.mat = (int)S.stat_mat[prim];
    } else {
        int k;
        const float4 *tr = dyn_tri_of(S, prim, k);
        v.n = tof(dlinear(c.A.E.M(k, g), d3(tr[0].w, tr[1].w, tr[2].w)));
        v.mat = kMatDynamic - k;
    }
    v.p = p;
    v.prim = prim;
    v.b1 = b1;
    v.b2 = b2;
    return v;
}

static __device__ __forceinline__ Vtx camera_vertex(const Ctx &c) {
    Vtx v;
    v.p = c.A.S.cam_pos;
    v.n = f3(0, 0, 0);
    v.prim = -1;
    v.mat = kMatCamera;
    v.b1 = v.b2 = 0.f;
    return v;
}

// ---------------------------------------------------------------------------
// camera: pinhole, film at distance 1, box pixel filter
// ---------------------------------------------------------------------------

static __device__ __forceinline__ float3 camera_dir(const DevScene &S, int px, int py, float jx, float jy) {
    double sx = (2.0 * ((double)px + jx) / (double)S.W - 1.0) * (double)S.hw;
    double sy = (1.0 - 2.0 * ((double)py + jy) / (double)S.H) * (double)S.hh;
    return tof(dunit(dadd(dadd(d3(S.cam_fwd), dscale(d3(S.cam_right), sx)), dscale(d3(S.cam_up), sy))));
}

static __device__ __forceinline__ int camera_project(const DevScene &S, float3 p, float &cosc) {
    float3 v = p - S.cam_pos;
    float z = dot3(v, S.cam_fwd);
    if (z <= 0.f) return -1;
    float sx = dot3(v, S.cam_right) / z, sy = dot3(v, S.cam_up) / z;
    float fx = (sx / S.hw + 1.0f) * 0.5f * (float)S.W;
    float fy = (1.0f - sy / S.hh) * 0.5f * (float)S.H;
    if (!(fx >= 0.f && fx < (float)S.W && fy >= 0.f && fy < (float)S.H)) return -1;
    int px = min((int)floorf(fx), S.W - 1), py = min((int)floorf(fy), S.H - 1);
    cosc = z / len3(v);
    return py * S.W + px;
}

// ---------------------------------------------------------------------------
// path contribution (Eq. pathcontribution, pinhole importance), no visibility
// ---------------------------------------------------------------------------

// A single-precision value with its own power-of-two exponent.  Walks
// through near-coincident vertices (corners, crevices) make geometric terms
// and area densities of 1e8 and more per edge, so path products overflow
// plain single precision; the exponent is renormalised after each product.
struct SF {
    float m;
    int e;
};

static __device__ __forceinline__ void sf_fix(float &m, int &e) {
    const float a = fabsf(m);
    if (a > 0x1p40f || (a < 0x1p-40f && a > 0.f)) {
        int k;
        m = frexpf(m, &k);
        e += k;
    }
}

static __device__ __forceinline__ SF sf_mul(SF a, float x) {
    a.m *= x;
    sf_fix(a.m, a.e);
    return a;
}

// product with a double factor of any magnitude
static __device__ __forceinline__ SF sf_mul_d(SF a, double x) {
    int k;
    a.m *= (float)frexp(x, &k);
    a.e += k;
    sf_fix(a.m, a.e);
    return a;
}

static __device__ __forceinline__ SF sf_add(SF a, SF b) {
    if (a.m == 0.f) return b;
    if (b.m == 0.f) return a;
    SF r = a.e >= b.e ? SF{a.m + ldexpf(b.m, b.e - a.e), a.e} : SF{b.m + ldexpf(a.m, a.e - b.e), b.e};
    sf_fix(r.m, r.e);
    return r;
}

static __device__ __forceinline__ float sf_val(SF a) { return ldexpf(a.m, a.e); }

// path throughput f(x) (Eq. pathcontribution) as f * 2^e
static __device__ __noinline__ float3 path_throughput(const Ctx &c, int g, const Vtx *x, int k, int &pix, int &e) {
    const DevScene &S = c.A.S;
    e = 0;
    float cc;
    pix = camera_project(S, x[1].p, cc);
    if (pix < 0) return f3(0, 0, 0);
    float3 d01 = x[0].p - x[1].p;
    float r2 = dot3(d01, d01);
    float c1 = dot3(x[1].n, d01) / sqrtf(r2);
    if (c1 <= 0.f) return f3(0, 0, 0);
    float We = 1.0f / (S.pix_area * cc * cc * cc);
    float s0 = We * c1 / r2;
    float3 f = f3(s0, s0, s0);
    for (int j = 1; j <= k - 2; ++j) {
        float3 wi = unit3(x[j - 1].p - x[j].p);
        float3 ed = x[j + 1].p - x[j].p;
        float r2e = dot3(ed, ed);
        float3 wo = ed * (1.0f / sqrtf(r2e));
        Mat m = get_mat(c, g, x[j].mat);
        float3 rho = bsdf_eval(m, x[j].n, wi, wo);
        if (zero3(rho)) return f3(0, 0, 0);
        float ca = dot3(x[j].n, wo), cb = -dot3(x[j + 1].n, wo);
        if (ca <= 0.f || cb <= 0.f) return f3(0, 0, 0);
        f = mul3(f, rho) * (ca * cb);
        f = f * (1.0f / r2e);
        float mx = fmaxf(f.x, fmaxf(f.y, f.z));
        if (mx > 0x1p40f || (mx < 0x1p-40f && mx > 0.f)) {
            int kx;
            frexpf(mx, &kx);
            f = f * ldexpf(1.f, -kx);
            e += kx;
        }
    }
    Mat em = get_mat(c, g, x[k - 1].mat);
    return mul3(f, em.em);
}


// ---------------------------------------------------------------------------
// technique densities (Sec. 4.1, 4.3): pE = forward (camera-to-light walk)
// area pdfs, pL = backward (light-to-camera walk) area pdfs
// ---------------------------------------------------------------------------

static __device__ __forceinline__ float area_from_dir(float pw, float3 from, const Vtx &to) {
    float3 e = to.p - from;
    float r2 = dot3(e, e);
    float cs = -dot3(to.n, e) / sqrtf(r2);
    if (cs <= 0.f) return 0.f;
    return pw * cs / r2;
}

static __device__ float pdf_camera_area(const DevScene &S, const Vtx &x1) {
    float cc;
    if (camera_project(S, x1.p, cc) < 0) return 0.f;
    float3 d = S.cam_pos - x1.p;
    float r2 = dot3(d, d);
    float c1 = dot3(x1.n, d) / sqrtf(r2);
    if (c1 <= 0.f) return 0.f;
    return c1 / r2 / (S.film_area * cc * cc * cc);
}

static __device__ float step_pdf(const Ctx &c, int g, const Vtx *x, int cond, int at, int to) {
    float3 wc = unit3(x[cond].p - x[at].p);
    float3 wo = unit3(x[to].p - x[at].p);
    Mat m = get_mat(c, g, x[at].mat);
    return area_from_dir(bsdf_pdf(m, x[at].n, wc, wo), x[at].p, x[to]);
}

// The geometric factor of the term of ghost technique `kind` (4: last
// edge, 5: first edge, 6: in between) for the crossing of edge j of x with
// ghost triangle prim (the edited object at its frame 3 - g pose): the area
// density of the vertex behind a ghost point sampled by area (Eq.
// vertex1pdf) without p_D, or for (6) the two-ends geometric term with the
// uniform direction density 1 / 4 pi.  Single precision, except where the
// edge grazes the triangle (|cos| < 0.05): there the factor's 1 / |cos| and
// the crossing's place on the edge amplify rounding, and the crossing is
// re-solved and the factor taken in double.  0 when the edge lies in the
// triangle's plane.
static __device__ __noinline__ double ghost_geom(const Ctx &c, int g, const Vtx *x, int k, int j,
                                                 int kind, int prim, float tfall) {
    int kk;
    const float4 *tr = dyn_tri_of(c.A.S, prim, kk);
    const float *M = c.A.E.M(kk, 3 - g);
    const float3 a = x[j].p, e = x[j + 1].p - a;
    const float el2 = dot3(e, e);
    const float3 w = e * (1.0f / sqrtf(el2));
    const float3 v0 = affine(M, xyz(tr[0])), v1 = affine(M, xyz(tr[1])), v2 = affine(M, xyz(tr[2]));
    const float3 nn = cross3(v1 - v0, v2 - v0);
    const float nl = len3(nn);
    const float den = dot3(nn, w);
    if (fabsf(den) >= 0.05f * nl) {
        if (kind == 6)
            return (double)(fabsf(dot3(x[j].n, w)) * fabsf(dot3(x[j + 1].n, w))) /
                   ((double)(fabsf(den) / nl) * 4.0 * kPiD * (double)el2);
        const float3 cp = a + w * (dot3(nn, v0 - a) / den);
        const float3 o = (kind == 4) ? x[k - 1].p : x[0].p;
        const Vtx &x1 = (kind == 4) ? x[k - 2] : x[1];
        const float3 o1 = x1.p - o, og = cp - o;
        const float3 wo = o1 * (1.0f / len3(o1));
        const float cg = fabsf(dot3(nn, wo)) / nl, c1 = fabsf(dot3(x1.n, wo));
        if (!(cg > 0.f)) return 0.0;
        return (double)dot3(og, og) * (double)c1 / ((double)cg * (double)dot3(o1, o1));
    }
    const double3 da = d3(a), dw = dunit(dsub(d3(x[j + 1].p), da));
    double3 cp, cn;
    ghost_resolve(c, 3 - g, da, dw, prim, (double)tfall, cp, cn);
    if (kind == 6) {
        const double cg = fabs(ddot(cn, dw));
        if (!(cg > 0.0)) return 0.0;
        const double3 ed = dsub(d3(x[j + 1].p), da);
        return fabs(ddot(d3(x[j].n), dw)) * fabs(ddot(d3(x[j + 1].n), dw)) / (cg * 4.0 * kPiD * ddot(ed, ed));
    }
    const double3 o = d3((kind == 4) ? x[k - 1].p : x[0].p);
    const Vtx &x1 = (kind == 4) ? x[k - 2] : x[1];
    const double3 o1 = dsub(d3(x1.p), o), wo = dunit(o1);
    const double cg = fabs(ddot(cn, wo)), c1 = fabs(ddot(d3(x1.n), wo));
    if (!(cg > 0.0)) return 0.0;
    const double3 og = dsub(cp, o);
    return ddot(og, og) * c1 / (cg * ddot(o1, o1));
}

// the balance-heuristic denominator of a path: the sum over the enabled
// techniques that can produce it of their area densities (Sec. 4.3), each a
// product of single-precision factors kept as SF
// The ghost terms search each edge j of the path for crossings with the
// object at its other-frame pose: *searched gets bit j for every edge
// searched and *crossed bit j when one was found; edges in known_clear are
// not searched (they are known to cross nothing).
static __device__ __noinline__ SF mis_denominator(Ctx &c, int g, const Vtx *x, int k,
                                                  uint32_t *searched = nullptr,
                                                  uint32_t *crossed = nullptr,
                                                  uint32_t known_clear = 0u) {
    const DevScene &S = c.A.S;
    const int tm = c.A.tech_mask;
    const bool t1 = tm & 1, t2 = tm & 2, t3 = tm & 4, t7 = tm & 8;
    if (k == 2) return SF{t7 ? pdf_camera_area(S, x[1]) : 0.f, 0};
    float pE[kMaxVerts], pL[kMaxVerts];
    const float pD = 1.0f / S.dyn_area, pLi = 1.0f / S.emit_area;
    pE[1] = pdf_camera_area(S, x[1]);
    for (int j = 2; j <= k - 2; ++j) pE[j] = step_pdf(c, g, x, j - 2, j - 1, j);
    for (int j = 1; j <= k - 3; ++j) pL[j] = step_pdf(c, g, x, j + 2, j + 1, j);
    SF sum{0.f, 0};
    if (t7) {
        SF p{pLi, 0};
        for (int j = 1; j <= k - 2; ++j) p = sf_mul(p, pE[j]);
        sum = sf_add(sum, p);
    }
    for (int i = 1; i <= k - 2; ++i) {
        if (!is_dyn(c, x[i])) continue;
        if (i == k - 2) {                    // (1) dynamic from emitter
            if (!t1) continue;
            SF p{pD * pLi, 0};
            for (int j = 1; j <= k - 3; ++j) p = sf_mul(p, pL[j]);
            sum = sf_add(sum, p);
        } else if (i == 1) {                 // (2) dynamic from sensor
            if (!t2) continue;
            SF p{pD * pLi, 0};
            for (int j = 2; j <= k - 2; ++j) p = sf_mul(p, pE[j]);
            sum = sf_add(sum, p);
        } else {                             // (3) dynamic two ends
            if (!t3) continue;
            float3 w = unit3(x[i + 1].p - x[i].p);
            SF p{pD * pLi, 0};
            p = sf_mul(p, area_from_dir(cosine_pdf(x[i].n, w), x[i].p, x[i + 1]));
            for (int j = i + 2; j <= k - 2; ++j) p = sf_mul(p, pE[j]);
            for (int j = 1; j <= i - 1; ++j) p = sf_mul(p, pL[j]);
            sum = sf_add(sum, p);
        }
    }
    // (4)-(6): one term per ghost crossing of an edge, (5) on the first
    // edge, (4) on the last, (6) in between (Sec. 4.2: the area density of
    // the vertex behind a ghost point sampled by area, Eq. vertex1pdf, and
    // the two-ends geometric term with a uniform direction density 1 / 4 pi)
    if ((tm & 0x70) && c.A.E.motion && k >= 3) {
        for (int j = 0; j <= k - 2; ++j) {
            const int kind = (j == 0) ? 5 : (j == k - 2) ? 4 : 6;
            if (!(tm & (1 << kind)) || ((known_clear >> j) & 1u)) continue;
            float ts[kMaxCross];
            int prims[kMaxCross];
            const int nc = ghost_prims(c, g, x[j].p, x[j + 1].p, ts, prims);
            if (searched) *searched |= 1u << j;
            if (crossed && nc > 0) *crossed |= 1u << j;
            if (nc == 0) continue;
            // the walk densities the technique shares for every crossing of
            // this edge
            SF base{pD * pLi, 0};
            if (kind == 4) {
                for (int m = 1; m <= k - 3; ++m) base = sf_mul(base, pL[m]);
            } else if (kind == 5) {
                for (int m = 2; m <= k - 2; ++m) base = sf_mul(base, pE[m]);
            } else {
                for (int m = 1; m <= j - 1; ++m) base = sf_mul(base, pL[m]);
                for (int m = j + 2; m <= k - 2; ++m) base = sf_mul(base, pE[m]);
            }
            for (int q = 0; q < nc; ++q) {
                const double gf = ghost_geom(c, g, x, k, j, kind, prims[q], ts[q]);
                if (gf > 0.0) sum = sf_add(sum, sf_mul_d(base, gf));
            }
        }
    }
    return sum;
}

// ---------------------------------------------------------------------------
// visibility
// ---------------------------------------------------------------------------

static __device__ __noinline__ bool segment_clear(Ctx &c, int g, const Vtx &a, const Vtx &b, bool dyn_only) {
    float3 e = b.p - a.p;
    float dist = len3(e);
    float3 d = e * (1.0f / dist);
    Hit h;
    ++c.cnt.rays_shadow;
    return !scene_trace_ol(c, g, a.p, d, c.A.S.eps, dist - c.A.S.eps, a.prim, b.prim, true, dyn_only,
                        h);
}

static __device__ __noinline__ bool trace_next(Ctx &c, int g, const Vtx &a, float3 d, Vtx &out) {
    Hit h;
    ++c.cnt.rays_closest;
    if (!scene_trace_ol(c, g, a.p, d, c.A.S.eps, __int_as_float(0x7f800000), a.prim, -1, false, false,
                     h))
        return false;
    out = make_vertex_at(c, g, h.prim, h.b1, h.b2, h.p);
    return true;
}

// static: no dynamic vertex and no edge through the object's other-frame pose
static __device__ bool path_is_static(Ctx &c, int g, const Vtx *x, int k) {
    for (int i = 0; i < k; ++i)
        if (is_dyn(c, x[i])) return false;
    if (!c.A.E.motion) return true;
    for (int j = 0; j + 1 < k; ++j)
        if (!segment_clear(c, 3 - g, x[j], x[j + 1], true)) return false;
    return true;
}

// ---------------------------------------------------------------------------
// path mapping (Sec. 5)
// ---------------------------------------------------------------------------

enum {
    MAP_ACCEPT = 0,
    MAP_INVALID = 1,
    MAP_REJECT_NODYN = 2,
    MAP_REJECT_MULTI = 3,
    MAP_REJECT_INVERT = 4,
    MAP_REJECT_JAC = 5,
    MAP_OFF = 6                 // path mapping switched off
};

static __device__ bool reconnect_ok(const Ctx &c, int ga, const Vtx &a, int gap, const Vtx &ap, int gb,
                             const Vtx &b) {
    if (is_dyn(c, b)) return false;
    float r = fminf(fminf(mat_rough(get_mat(c, ga, a.mat)), mat_rough(get_mat(c, gap, ap.mat))),
                    mat_rough(get_mat(c, gb, b.mat)));
    if (!(r >= c.A.S.alpha_min)) return false;
    float d = fminf(len3(ap.p - b.p), len3(a.p - b.p));
    return d >= c.A.S.d_min;
}

struct MapInfo {
    int status;
    float J;
    unsigned replayed;   // bit j: y[j] produced by replay
};

// one walk step: x[b] was reached from x[a], sampled with conditioning x[cc]
// (cc < 0: cosine step); fills y[b]
static __device__ __noinline__ int map_step(Ctx &c, int g, int g2, const Vtx *x, Vtx *y, int a, int b, int cc,
                        MapInfo &mi) {
    if (same3(y[a].p, x[a].p)) {               // predecessor unchanged
        y[b] = x[b];
        return MAP_ACCEPT;
    }
    if (reconnect_ok(c, g, x[a], g2, y[a], g, x[b])) {    // keep vertex the same
        y[b] = x[b];
        return MAP_ACCEPT;
    }
    // random-seed replay through the inverse of the step's sampling routine
    float3 wo = unit3(x[b].p - x[a].p);
    double u1, u2;
    float3 w2;
    Mat ma = get_mat(c, g, x[a].mat), mya = get_mat(c, g2, y[a].mat);
    if (cc < 0) {
        cosine_inverse(x[a].n, wo, u1, u2);
        w2 = cosine_dir(c.A.S, y[a].n, u1, u2);
        if (dot3(y[a].n, w2) <= 0.f) return MAP_INVALID;
    } else {
        float3 wc = unit3(x[cc].p - x[a].p);
        bsdf_inverse(ma, x[a].n, wc, wo, u1, u2);
        float3 wc2 = unit3(y[cc].p - y[a].p);
        if (!bsdf_sample(c.A.S, mya, y[a].n, wc2, u1, u2, w2)) return MAP_INVALID;
    }
    Vtx nb;
    if (!trace_next(c, g2, y[a], w2, nb)) return MAP_INVALID;
    if (dot3(nb.n, w2) >= 0.f) return MAP_INVALID;
    if (is_dyn(c, nb)) return MAP_REJECT_MULTI;
    if (reconnect_ok(c, g2, y[a], g, x[a], g2, nb)) return MAP_REJECT_INVERT;
    y[b] = nb;
    mi.replayed |= 1u << b;
    float px, py;
    if (cc < 0) {
        px = area_from_dir(cosine_pdf(x[a].n, wo), x[a].p, x[b]);
        py = area_from_dir(cosine_pdf(y[a].n, w2), y[a].p, y[b]);
    } else {
        px = step_pdf(c, g, x, cc, a, b);
        py = step_pdf(c, g2, y, cc, a, b);
    }
    if (!(px > 0.f) || !(py > 0.f)) return MAP_INVALID;
    mi.J *= px / py;
    return MAP_ACCEPT;
}

// the first edge of a frame-g path is dynamic: x_1 lies on the object or the
// camera ray to x_1 crosses the ghost (the object at its other-frame pose)
static __device__ bool first_edge_dynamic(Ctx &c, int g, const Vtx *x, int k) {
    if (k < 2 || !c.A.E.motion) return false;
    if (is_dyn(c, x[1])) return true;
    return !segment_clear(c, 3 - g, x[0], x[1], true);
}

// camera replay (Sec. 5, "Mapping between the dynamic and ghost pair": the
// same camera direction in both frames): y_1 is the first hit of the camera
// ray through x_1 in frame g2 (area Jacobian: ratio of the camera
// densities), then the light side walks as for technique (2); the class of
// paths with a dynamic first edge is closed under this map
static __device__ void map_camera(Ctx &c, int g, int g2, const Vtx *x, int k, Vtx *y, MapInfo &mi) {
    for (int j = 2; j <= k - 2; ++j)
        if (is_dyn(c, x[j])) {
            mi.status = MAP_REJECT_MULTI;
            return;
        }
    const float3 w = unit3(x[1].p - x[0].p);
    Vtx y1;
    if (!trace_next(c, g2, y[0], w, y1) || dot3(y1.n, w) >= 0.f) {
        mi.status = MAP_INVALID;
        return;
    }
    y[1] = y1;
    mi.replayed |= 2u;
    const float px = pdf_camera_area(c.A.S, x[1]), py = pdf_camera_area(c.A.S, y[1]);
    if (!(px > 0.f) || !(py > 0.f)) {
        mi.status = MAP_INVALID;
        return;
    }
    mi.J *= px / py;
    for (int b = 2; b <= k - 2; ++b) {
        const int st = map_step(c, g, g2, x, y, b - 1, b, b - 2, mi);
        if (st != MAP_ACCEPT) {
            mi.status = st;
            return;
        }
    }
    if (!first_edge_dynamic(c, g2, y, k)) {
        mi.status = MAP_REJECT_INVERT;
        return;
    }
    const float jm = c.A.S.jac_max;
    if (!(mi.J <= jm && 1.0f / mi.J <= jm)) {
        mi.status = MAP_REJECT_JAC;
        return;
    }
    mi.status = MAP_ACCEPT;
}

static __device__ void map_path(Ctx &c, int g, int g2, const Vtx *x, int k, Vtx *y, MapInfo &mi) {
    mi.J = 1.0f;
    mi.replayed = 0u;
    for (int j = 0; j < k; ++j) y[j] = x[j];
    if (c.A.map_mode == 2 && first_edge_dynamic(c, g, x, k)) {
        map_camera(c, g, g2, x, k, y, mi);
        return;
    }
    int nd = 0, i = -1;
    for (int j = 1; j <= k - 2; ++j)
        if (is_dyn(c, x[j])) {
            ++nd;
            i = j;
        }
    if (nd == 0) {
        mi.status = MAP_REJECT_NODYN;
        return;
    }
    if (nd > 1) {
        mi.status = MAP_REJECT_MULTI;
        return;
    }
    y[i] = make_vertex(c, g2, x[i].prim, x[i].b1, x[i].b2);   // object transform
    int st;
    if (i == k - 2) {              // (1): eye side from x_D, first step conditioned on x_L
        for (int b = i - 1; b >= 1; --b) {
            int cc = (b == i - 1) ? k - 1 : b + 2;
            st = map_step(c, g, g2, x, y, b + 1, b, cc, mi);
            if (st != MAP_ACCEPT) { mi.status = st; return; }
        }
    } else if (i == 1) {           // (2): light side, first step conditioned on the camera
        for (int b = 2; b <= k - 2; ++b) {
            st = map_step(c, g, g2, x, y, b - 1, b, b - 2, mi);
            if (st != MAP_ACCEPT) { mi.status = st; return; }
        }
    } else {                       // (3): light side (cosine first), then eye side
        for (int b = i + 1; b <= k - 2; ++b) {
            int cc = (b == i + 1) ? -1 : b - 2;
            st = map_step(c, g, g2, x, y, b - 1, b, cc, mi);
            if (st != MAP_ACCEPT) { mi.status = st; return; }
        }
        for (int b = i - 1; b >= 1; --b) {
            st = map_step(c, g, g2, x, y, b + 1, b, b + 2, mi);
            if (st != MAP_ACCEPT) { mi.status = st; return; }
        }
    }
    const float jm = c.A.S.jac_max;
    if (!(mi.J <= jm && 1.0f / mi.J <= jm)) {
        mi.status = MAP_REJECT_JAC;
        return;
    }
    // the image must stay outside the camera-replay class (else the inverse
    // map would differ)
    if (c.A.map_mode == 2 && first_edge_dynamic(c, g2, y, k)) {
        mi.status = MAP_REJECT_INVERT;
        return;
    }
    mi.status = MAP_ACCEPT;
}

// replayed edges are visible by construction; unchanged edges are re-checked
// against the dynamic object only; all others fully
static __device__ bool mapped_visible(Ctx &c, int g2, const Vtx *x, const Vtx *y, int k, const MapInfo &mi) {
    int i = -1;
    for (int j = 1; j <= k - 2; ++j)
        if (is_dyn(c, y[j])) i = j;
    for (int j = 0; j + 1 < k; ++j) {
        int far = (j + 1 <= i) ? j : j + 1;
        if (mi.replayed & (1u << far)) continue;
        bool unchanged = same3(x[j].p, y[j].p) && same3(x[j + 1].p, y[j + 1].p);
        if (!segment_clear(c, g2, y[j], y[j + 1], unchanged)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// evaluation and splatting of one base path
// ---------------------------------------------------------------------------

static __device__ __forceinline__ void splat(double *img, int pix, float3 v) {
    if (pix < 0) return;
    if (v.x != 0.f) atomicAdd(img + 3 * pix + 0, (double)v.x);
    if (v.y != 0.f) atomicAdd(img + 3 * pix + 1, (double)v.y);
    if (v.z != 0.f) atomicAdd(img + 3 * pix + 2, (double)v.z);
}

static __device__ void emit(Ctx &c, uint32_t root, int tech, int g, int sa, int sb, int pa, float3 va,
                     int pb, float3 vb, int status, float Pg, float Py, float J) {
    const LaunchArgs &A = c.A;
    if (tech == T_3 && A.G.on) {
        // learned proposal: the root's light-side direction was drawn from
        // q = p_cos / 2 + mixture / 2, so its values carry p_cos / q; the
        // magnitude of what the root adds is its training weight
        if (A.G.use_net) {
            const float s = A.G.gratio[root - A.root_begin];
            va = va * s;
            vb = vb * s;
        }
        const uint32_t slot = root < A.G.half ? (uint32_t)(g - 1) * A.G.half + root : ~0u;
        if (slot != ~0u)
            atomicAdd(A.G.smp.wt + slot, fabsf(va.x) + fabsf(va.y) + fabsf(va.z) + fabsf(vb.x) +
                                             fabsf(vb.y) + fabsf(vb.z));
    }
    if (A.rec_count) {
        unsigned long long idx = atomicAdd(A.rec_count, 1ull);
        if (A.rec && idx < A.rec_cap) {
            Record &r = A.rec[idx];
            r.root = root; r.tech = tech; r.frame = g; r.sa = sa; r.sb = sb;
            r.pix_a = pa; r.pix_b = pb;
            r.va[0] = va.x; r.va[1] = va.y; r.va[2] = va.z;
            r.vb[0] = vb.x; r.vb[1] = vb.y; r.vb[2] = vb.z;
            r.status = status; r.Pg = Pg; r.Py = Py; r.J = J;
        }
    }
    if (A.img) {
        splat(A.img, pa, va);
        splat(A.img, pb, vb);
    }
}

struct PathCounts {
    unsigned int paths, accepted, rejected;
};

// static_known: the caller already rejected static paths of technique (7)
static __device__ void evaluate_path(Ctx &c, PathCounts &pc, int g, const Vtx *x, int n, uint32_t root,
                              int tech, int sa, int sb, bool residual, bool static_known = false) {
    int pa, ex;
    const float3 fx = path_throughput(c, g, x, n, pa, ex);
    if (zero3(fx)) return;
    const float invN = c.A.invN;
    if (!residual) {               // primal path tracing: one technique
        SF p{0.f, 0};
        {
            // path tracing density alone
            const DevScene &S = c.A.S;
            if (n == 2) {
                p.m = pdf_camera_area(S, x[1]);
            } else {
                p.m = pdf_camera_area(S, x[1]) / S.emit_area;
                for (int j = 2; j <= n - 2; ++j) p = sf_mul(p, step_pdf(c, g, x, j - 2, j - 1, j));
            }
        }
        ++pc.paths;
        emit(c, root, tech, g, sa, sb, pa, fx * ldexpf(invN / p.m, ex - p.e), -1, f3(0, 0, 0), 0,
             sf_val(p), 0.f, 1.f);
        return;
    }
    if (tech == T_7 && !static_known && path_is_static(c, g, x, n)) return;
    ++pc.paths;
    const SF Pg = mis_denominator(c, g, x, n);
    const float sign = (g == 2) ? 1.0f : -1.0f;
    const int g2 = 3 - g;
    Vtx y[kMaxVerts];
    MapInfo mi;
    mi.J = 1.0f;
    mi.replayed = 0u;
    if (!c.A.E.motion) {
        for (int j = 0; j < n; ++j) y[j] = x[j];
        mi.status = MAP_ACCEPT;
    } else if (c.A.map_mode == 0) {
        mi.status = MAP_OFF;     // each frame estimates its own paths
    } else {
        map_path(c, g, g2, x, n, y, mi);
    }
    float3 fy = f3(0, 0, 0);
    int pb = -1, ey = 0;
    SF Py{0.f, 0};
    if (mi.status == MAP_ACCEPT) {
        if (c.A.E.motion && !mapped_visible(c, g2, x, y, n, mi)) {
            mi.status = MAP_INVALID;
        } else {
            fy = path_throughput(c, g2, y, n, pb, ey);
            if (zero3(fy)) {
                mi.status = MAP_INVALID;
            } else {
                Py = mis_denominator(c, g2, y, n);
                if (!(Py.m > 0.f)) mi.status = MAP_INVALID;
            }
        }
    }
    if (mi.status == MAP_ACCEPT) {
        ++pc.accepted;
        const SF den = sf_add(Pg, SF{Py.m * mi.J, Py.e});
        emit(c, root, tech, g, sa, sb, pa, fx * ldexpf(sign * invN / den.m, ex - den.e), pb,
             fy * ldexpf(-sign * mi.J * invN / den.m, ey - den.e), mi.status, sf_val(Pg), sf_val(Py),
             mi.J);
    } else {
        if (mi.status != MAP_INVALID) ++pc.rejected;
        emit(c, root, tech, g, sa, sb, pa, fx * ldexpf(sign * invN / Pg.m, ex - Pg.e), -1, f3(0, 0, 0),
             mi.status, sf_val(Pg), 0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------
// root sampling and walks
// ---------------------------------------------------------------------------

// the triangle of uniform u = k / 2^24: smallest i with k < cdf[i]
static __device__ __forceinline__ int cdf_pick(const uint32_t *cdf, int n, float u) {
    const uint32_t k = (uint32_t)(u * 16777216.0f);
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (k < __ldg(&cdf[mid])) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

static __device__ __forceinline__ void tri_sample(float u1, float u2, double &b1, double &b2) {
    double s = sqrt((double)u1);
    b1 = s * (1.0 - (double)u2);
    b2 = s * (double)u2;
}

static __device__ Vtx sample_dynamic(const Ctx &c, int g, float4 r) {
    const DevScene &S = c.A.S;
    int t = cdf_pick(S.dyn_cdf, S.n_dyn, r.x);
    double b1, b2;
    tri_sample(r.y, r.z, b1, b2);
    return make_vertex_d(c, g, S.n_static + t, b1, b2);
}

static __device__ Vtx sample_emitter(const Ctx &c, int g, float4 r) {
    const DevScene &S = c.A.S;
    int t = cdf_pick(S.emit_cdf, S.n_emit, r.x);
    double b1, b2;
    tri_sample(r.y, r.z, b1, b2);
    return make_vertex_d(c, g, S.emit_ids[t], b1, b2);
}

static __device__ __forceinline__ bool faces(const Vtx &v, float3 towards) {
    return dot3(v.n, towards - v.p) > 0.f;
}

static __device__ bool camera_visible(Ctx &c, int g, const Vtx &z) {
    float cc;
    if (camera_project(c.A.S, z.p, cc) < 0) return false;
    Vtx cam = camera_vertex(c);
    if (!faces(z, cam.p)) return false;
    return segment_clear(c, g, z, cam, false);
}

static __device__ bool nee(Ctx &c, int g, const Vtx &z, float4 r, Vtx &L) {
    L = sample_emitter(c, g, r);
    if (!faces(z, L.p) || !faces(L, z.p)) return false;
    return segment_clear(c, g, z, L, false);
}

static __device__ bool walk_step(Ctx &c, int g, const Vtx &prev, const Vtx &at, float4 r, Vtx &out) {
    float3 wc = unit3(prev.p - at.p);
    float3 wo;
    Mat m = get_mat(c, g, at.mat);
    if (!bsdf_sample_walk(c.A.S, m, at.n, wc, r.x, r.y, wo)) return false;
    if (!trace_next(c, g, at, wo, out)) return false;
    if (dot3(out.n, wo) >= 0.f) return false;
    return true;
}

static __device__ __forceinline__ bool vtx_black(const Ctx &c, int g, const Vtx &v) {
    return mat_black(get_mat(c, g, v.mat));
}

// (1) dynamic from emitter
static __device__ void root_T1(Ctx &c, PathCounts &pc, int g, uint32_t root) {
    const uint64_t seed = lseed(c.A);
    const int D = c.A.S.max_depth;
    Vtx z[kMaxVerts];
    z[0] = sample_dynamic(c, g, draw(seed, root, T_1, g, SD_ROOT, 0));
    Vtx xL;
    if (!nee(c, g, z[0], draw(seed, root, T_1, g, SD_NEE, 0), xL)) return;
    if (vtx_black(c, g, z[0])) return;
    Vtx path[kMaxVerts];
    for (int t = 0; t <= D - 2; ++t) {
        if (t > 0) {
            const Vtx &prev = (t == 1) ? xL : z[t - 2];
            if (!walk_step(c, g, prev, z[t - 1], draw(seed, root, T_1, g, SD_EYE, t), z[t])) break;
            if (vtx_black(c, g, z[t])) break;
        }
        if (camera_visible(c, g, z[t])) {
            const int n = t + 3;
            path[0] = camera_vertex(c);
            for (int j = 0; j <= t; ++j) path[1 + j] = z[t - j];
            path[n - 1] = xL;
            evaluate_path(c, pc, g, path, n, root, T_1, t, 0, true);
        }
    }
}

// (2) dynamic from sensor
static __device__ void root_T2(Ctx &c, PathCounts &pc, int g, uint32_t root) {
    const uint64_t seed = lseed(c.A);
    const int D = c.A.S.max_depth;
    Vtx yv[kMaxVerts];
    yv[0] = sample_dynamic(c, g, draw(seed, root, T_2, g, SD_ROOT, 0));
    if (vtx_black(c, g, yv[0])) return;
    if (!camera_visible(c, g, yv[0])) return;
    const Vtx cam = camera_vertex(c);
    Vtx path[kMaxVerts];
    for (int t = 1; t <= D - 2; ++t) {
        const Vtx &prev = (t == 1) ? cam : yv[t - 2];
        if (!walk_step(c, g, prev, yv[t - 1], draw(seed, root, T_2, g, SD_LIGHT, t), yv[t])) break;
        if (vtx_black(c, g, yv[t])) break;
        Vtx L;
        if (nee(c, g, yv[t], draw(seed, root, T_2, g, SD_NEE, t), L)) {
            const int n = t + 3;
            path[0] = cam;
            for (int j = 0; j <= t; ++j) path[1 + j] = yv[j];
            path[n - 1] = L;
            evaluate_path(c, pc, g, path, n, root, T_2, 0, t, true);
        }
    }
}

// (3) dynamic two ends
static __device__ void root_T3(Ctx &c, PathCounts &pc, int g, uint32_t root) {
    const uint64_t seed = lseed(c.A);
    const int D = c.A.S.max_depth;
    if (D < 4) return;
    Vtx yv[kMaxVerts], zv[kMaxVerts], Lv[kMaxVerts];
    unsigned Lok = 0u, Cok = 0u;
    int ny = 0, nz = 0;
    yv[0] = sample_dynamic(c, g, draw(seed, root, T_3, g, SD_ROOT, 0));
    if (vtx_black(c, g, yv[0])) return;
    zv[0] = yv[0];
    {
        float4 r = draw(seed, root, T_3, g, SD_LIGHT, 1);
        float3 w = cosine_dir_walk(c.A.S, yv[0].n, r.x, r.y);
        if (dot3(yv[0].n, w) > 0.f && trace_next(c, g, yv[0], w, yv[1]) &&
            dot3(yv[1].n, w) < 0.f && !vtx_black(c, g, yv[1])) {
            ny = 1;
            for (int t = 2; t <= D - 3; ++t) {
                if (!walk_step(c, g, yv[t - 2], yv[t - 1], draw(seed, root, T_3, g, SD_LIGHT, t),
                               yv[t]))
                    break;
                if (vtx_black(c, g, yv[t])) break;
                ny = t;
            }
        }
    }
    if (ny == 0) return;
    for (int t = 1; t <= ny; ++t)
        if (nee(c, g, yv[t], draw(seed, root, T_3, g, SD_NEE, t), Lv[t])) Lok |= 1u << t;
    for (int t = 1; t <= D - 3; ++t) {
        const Vtx &prev = (t == 1) ? yv[1] : zv[t - 2];
        if (!walk_step(c, g, prev, zv[t - 1], draw(seed, root, T_3, g, SD_EYE, t), zv[t])) break;
        if (vtx_black(c, g, zv[t])) break;
        nz = t;
    }
    for (int t = 1; t <= nz; ++t)
        if (camera_visible(c, g, zv[t])) Cok |= 1u << t;
    Vtx path[kMaxVerts];
    for (int te = 1; te <= nz; ++te) {
        if (!(Cok & (1u << te))) continue;
        for (int sl = 1; sl <= ny && te + sl <= D - 2; ++sl) {
            if (!(Lok & (1u << sl))) continue;
            const int n = te + sl + 3;
            path[0] = camera_vertex(c);
            for (int j = 0; j < te; ++j) path[1 + j] = zv[te - j];
            path[te + 1] = yv[0];
            for (int j = 1; j <= sl; ++j) path[te + 1 + j] = yv[j];
            path[n - 1] = Lv[sl];
            evaluate_path(c, pc, g, path, n, root, T_3, te, sl, true);
        }
    }
}

// path tracing with next-event estimation: technique (7) when residual,
// plain path tracing (frame-independent random numbers) when primal
static __device__ void root_PT(Ctx &c, PathCounts &pc, int g, uint32_t root, bool residual) {
    const DevScene &S = c.A.S;
    const uint64_t seed = lseed(c.A);
    const int D = S.max_depth;
    const int tech = residual ? T_7 : T_PT;
    const int rg = residual ? g : 0;
    const uint32_t npix = (uint32_t)(S.W * S.H);
    const int pix = (int)(root % npix);
    float4 r = draw(seed, root, tech, rg, SD_ROOT, 0);
    float3 d = camera_dir(S, pix % S.W, pix / S.W, r.x, r.y);
    Vtx path[kMaxVerts];
    path[0] = camera_vertex(c);
    if (!trace_next(c, g, path[0], d, path[1])) return;
    if (dot3(path[1].n, d) >= 0.f) return;
    if (!zero3(get_mat(c, g, path[1].mat).em))
        evaluate_path(c, pc, g, path, 2, root, tech, 0, 2, residual);
    for (int j = 1; j <= D - 1; ++j) {
        if (vtx_black(c, g, path[j])) break;
        Vtx L;
        if (nee(c, g, path[j], draw(seed, root, tech, rg, SD_NEE, j), L)) {
            path[j + 1] = L;
            evaluate_path(c, pc, g, path, j + 2, root, tech, 0, j + 2, residual);
        }
        if (j == D - 1) break;
        if (!walk_step(c, g, path[j - 1], path[j], draw(seed, root, tech, rg, SD_LIGHT, j),
                       path[j + 1]))
            break;
    }
}

// ---------------------------------------------------------------------------
// warp-aggregated counters
// ---------------------------------------------------------------------------

static __device__ __forceinline__ void add_stat(unsigned long long *stats, int idx, unsigned int v) {
    unsigned long long s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(stats + idx, s);
}

template <int TECH>
static __device__ __forceinline__ void run_roots(const LaunchArgs &A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    PathCounts pc{0, 0, 0};
    unsigned int roots = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = A.root_begin + blockIdx.x * blockDim.x + threadIdx.x; r < A.root_end;
         r += stride) {
        ++roots;
        if (TECH == T_1) root_T1(c, pc, A.frame, r);
        else if (TECH == T_2) root_T2(c, pc, A.frame, r);
        else if (TECH == T_3) root_T3(c, pc, A.frame, r);
        else if (TECH == T_7) root_PT(c, pc, A.frame, r, true);
        else root_PT(c, pc, A.frame, r, false);
    }
    if (A.stats) {
        add_stat(A.stats, ST_ROOTS, roots);
        add_stat(A.stats, ST_PATHS, pc.paths);
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_ACCEPTED, pc.accepted);
        add_stat(A.stats, ST_REJECTED, pc.rejected);
    }
}

}  // namespace rp
