// Learned proposal of technique (3) inside the path kernels: integer input
// features of x_D, the von Mises-Fisher mixture decoded from the network's
// outputs, its density and sampling, all in double precision so that the
// sampled direction and the value ratio p_cos / q depend only on the exact
// integer network outputs.
#pragma once

#include "guide.h"
#include "rp_device.cuh"

namespace rp {

// input features of an object-space point and (float) unit normal: for each
// coordinate c of u = clamp((p - center) inv_half, -1, 1), then of n,
// sin(2^f pi c), cos(2^f pi c) for f = 0..5; then u and n; quantised to
// rint(128 e) in [-127, 127]; then the constant 127 and a zero
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
    for (int v = 0; v < 2; ++v)
        for (int c = 0; c < 3; ++c)
            for (int f = 0; f < 6; ++f) {
                const double a = ldexp(v == 0 ? u[c] : nn[c], f);
                double s, co;
                sincos(kPiD * a, &s, &co);
                m[i++] = q(s);
                m[i++] = q(co);
            }
    for (int c = 0; c < 3; ++c) m[i++] = q(u[c]);
    for (int c = 0; c < 3; ++c) m[i++] = q(nn[c]);
    m[78] = 127;
    m[79] = 0;
}

struct MixD {
    double3 mu[kGLobes];
    double kappa[kGLobes], pi[kGLobes];
};

// lobe j: outputs 5j..5j+2 direction (normalised), 5j+3 log kappa clamped to
// [-4, 6.2], 5j+4 logit (softmax over the lobes)
static __device__ void guide_mixture_d(const float *o, MixD &M) {
    double mx = o[4];
    for (int j = 1; j < kGLobes; ++j) mx = fmax(mx, (double)o[5 * j + 4]);
    double sum = 0.0;
    for (int j = 0; j < kGLobes; ++j) {
        M.pi[j] = exp((double)o[5 * j + 4] - mx);
        sum += M.pi[j];
    }
    for (int j = 0; j < kGLobes; ++j) {
        M.pi[j] /= sum;
        const double3 m = d3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
        const double l = sqrt(ddot(m, m));
        M.mu[j] = l > 1e-12 ? dscale(m, 1.0 / l) : d3(0.0, 0.0, 1.0);
        M.kappa[j] = exp(fmin(6.2, fmax(-4.0, (double)o[5 * j + 3])));
    }
}

// kappa / (2 pi (1 - exp(-2 kappa))) exp(kappa (mu.w - 1))
static __device__ __forceinline__ double vmf_pdf_d(double3 mu, double kappa, double3 w) {
    return kappa / (2.0 * kPiD * -expm1(-2.0 * kappa)) * exp(kappa * (ddot(mu, w) - 1.0));
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

static __device__ double mix_pdf_d(const MixD &M, double3 w) {
    double p = 0.0;
    for (int j = 0; j < kGLobes; ++j) p += M.pi[j] * vmf_pdf_d(M.mu[j], M.kappa[j], w);
    return p;
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
