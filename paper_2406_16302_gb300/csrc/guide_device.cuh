// Learned proposal of technique (3) inside the path kernels: integer input
// features of x_D (double precision, then quantised), the von Mises-Fisher
// mixture decoded from the network's exact outputs, its density, and the
// sampled direction (double precision).
#pragma once

#include "guide.h"
#include "rp_device.cuh"

namespace rp {

// input features of an object-space point and (float) unit normal: for each
// coordinate c of u = clamp((p - center) inv_half, -1, 1), then of n,
// sin(2^f pi c), cos(2^f pi c) for f = 0..5; then u and n; quantised to
// rint(128 e) in [-127, 127]; then the constant 127 and a zero.
// The argument a = 2^f c is reduced to r = a - 2 rint(a / 2) in [-1, 1] in
// single precision: c = ch + cl with ch = (float) c, the high part's
// reduction 2^f ch - 2 rintf(2^f ch / 2) is exact (|2^f ch| <= 32, and an
// even integer subtracted from it leaves a representable value), and the
// low part 2^f cl adds a rounding of at most one ulp of r.  sin(pi r) and
// cos(pi r) are then taken in single precision: r is within 2^-24 of the
// exact reduced argument and sincospif within one ulp of the sine and cosine
// of its argument, so 128 e is within 128 (pi 2^-24 + 2^-24) < 3.2e-5 of
// its double-precision value, and the quantised value is the one the
// double-precision sine gives unless 128 e lies within 2.5e-4 of a rounding
// boundary, where it is recomputed in double from the exact argument.
static __device__ void guide_encode_d(const float *box, double3 p, float3 n, int8_t *m) {
    double u[3] = {((double)p.x - box[0]) * box[3], ((double)p.y - box[1]) * box[4],
                   ((double)p.z - box[2]) * box[5]};
    const double nn[3] = {n.x, n.y, n.z};
    for (int c = 0; c < 3; ++c) u[c] = fmin(1.0, fmax(-1.0, u[c]));
    int i = 0;
    auto q = [](double e) -> int8_t {
        const double r = rint(128.0 * e);
        return (int8_t)(int)fmin(127.0, fmax(-127.0, r));
    };
    auto near_half = [](float e) {
        const float v = 128.0f * e;
        return fabsf(v - floorf(v) - 0.5f) < 2.5e-4f;
    };
    for (int v = 0; v < 2; ++v)
        for (int c = 0; c < 3; ++c) {
            const double x = v == 0 ? u[c] : nn[c];
            const float xh = (float)x, xl = (float)(x - (double)xh);
            for (int f = 0; f < 6; ++f) {
                const float ah = ldexpf(xh, f);
                const float r = (ah - 2.0f * rintf(0.5f * ah)) + ldexpf(xl, f);
                float sf, cf;
                sincospif(r, &sf, &cf);
                if (near_half(sf) || near_half(cf)) {
                    const double a = ldexp(x, f);
                    double sd, cd;
                    sincospi(a - 2.0 * rint(0.5 * a), &sd, &cd);
                    m[i++] = q(sd);
                    m[i++] = q(cd);
                } else {
                    m[i++] = (int8_t)(int)fminf(127.0f, fmaxf(-127.0f, rintf(128.0f * sf)));
                    m[i++] = (int8_t)(int)fminf(127.0f, fmaxf(-127.0f, rintf(128.0f * cf)));
                }
            }
        }
    for (int c = 0; c < 3; ++c) m[i++] = q(u[c]);
    for (int c = 0; c < 3; ++c) m[i++] = q(nn[c]);
    m[78] = 127;
    m[79] = 0;
}

// The mixture in single precision.  The density exp(kappa (mu.w - 1))
// multiplies the error of mu.w - 1 by kappa (up to 493), so it is taken as
// exp(-kappa |mu - w|^2 / 2) (the same for unit vectors), whose argument
// has no cancellation: a rounding of mu or w moves |mu - w|^2 by a small
// fraction of itself, or by about 1e-7 |mu - w| across it, and the density
// stays within about 2e-5 of the double-precision value wherever
// kappa |mu - w|^2 / 2 < 20 (beyond that a lobe adds less than e^-20).  The
// sampled direction itself stays in double (guide_lobe_dir_d,
// vmf_sample_d): in single precision 0.1 % of a guided technique's paths
// moved beyond 1e-4 of the oracle's.
struct MixF {
    float3 mu[kGLobes];
    float kappa[kGLobes], pi[kGLobes], norm[kGLobes];   // norm = kappa / (2 pi (1 - e^-2kappa))
};

// lobe j: outputs 5j..5j+2 direction (normalised), 5j+3 log kappa clamped to
// [-4, 6.2], 5j+4 logit (softmax over the lobes)
static __device__ void guide_mixture_f(const float *o, MixF &M) {
    float mx = o[4];
#pragma unroll
    for (int j = 1; j < kGLobes; ++j) mx = fmaxf(mx, o[5 * j + 4]);
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) {
        M.pi[j] = expf(o[5 * j + 4] - mx);
        sum += M.pi[j];
    }
    const float inv = 1.f / sum;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) {
        M.pi[j] *= inv;
        const float3 m = f3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
        const float l = sqrtf(dot3(m, m));
        M.mu[j] = l > 1e-12f ? m * (1.f / l) : f3(0.f, 0.f, 1.f);
        const float k = expf(fminf(6.2f, fmaxf(-4.0f, o[5 * j + 3])));
        M.kappa[j] = k;
        M.norm[j] = k / (2.f * kPi * -expm1f(-2.f * k));
    }
}

static __device__ __forceinline__ float mix_pdf_f(const MixF &M, float3 wf) {
    float p = 0.f;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) {
        const float3 d = M.mu[j] - wf;
        p += M.pi[j] * M.norm[j] * expf(-0.5f * M.kappa[j] * dot3(d, d));
    }
    return p;
}

// the direction of lobe j, normalised in double (for sampling it)
static __device__ double3 guide_lobe_dir_d(const float *o, int j) {
    const double3 m = d3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
    const double l = sqrt(ddot(m, m));
    return l > 1e-12 ? dscale(m, 1.0 / l) : d3(0.0, 0.0, 1.0);
}

// inversion of the vMF cosine CDF (Jakob 2012) and a uniform azimuth in the
// tangent frame of mu
static __device__ double3 vmf_sample_d(const DevScene &S, double3 mu, double kappa, double u1,
                                       double u2) {
    double c = 1.0 + log(u1 + (1.0 - u1) * exp(-2.0 * kappa)) / kappa;
    c = fmin(1.0, fmax(-1.0, c));
    const double s = sqrt(fmax(0.0, 1.0 - c * c));
    double sp, cp;
    sincos2pi(S, u2, sp, cp);
    double3 t, b;
    tangent_frame_d(mu, t, b);
    return dadd(dadd(dscale(t, s * cp), dscale(b, s * sp)), dscale(mu, c));
}

// transpose of the linear part of a 3x4 row-major transform times a
static __device__ __forceinline__ double3 dlinear_T(const float *M, double3 a) {
    return d3((double)M[0] * a.x + (double)M[4] * a.y + (double)M[8] * a.z,
              (double)M[1] * a.x + (double)M[5] * a.y + (double)M[9] * a.z,
              (double)M[2] * a.x + (double)M[6] * a.y + (double)M[10] * a.z);
}

// training-sample slot of a root of frame g (none: ~0u)
static __device__ __forceinline__ uint32_t guide_slot(const GuideLaunch &G, int g, uint32_t root) {
    return root < G.half ? (uint32_t)(g - 1) * G.half + root : ~0u;
}

}  // namespace rp
