// Small geometric helpers shared by the per-root path evaluation
// (chain_fast.cuh): G terms, BSDF values and area sampling densities of a
// vertex with given neighbours.
#pragma once

#include "rp_device.cuh"

namespace rp {
namespace chain_detail {

// geometric term G(a, b) = cos_a cos_b / |a - b|^2 (zero on back faces)
__device__ __forceinline__ float G2(const Vtx &a, const Vtx &b) {
    float3 e = b.p - a.p;
    float r2 = dot3(e, e);
    float3 w = e * (1.0f / sqrtf(r2));
    float ca = dot3(a.n, w), cb = -dot3(b.n, w);
    if (ca <= 0.f || cb <= 0.f) return 0.f;
    return ca * cb / r2;
}

// BSDF at b with neighbours a (camera side) and c (light side)
__device__ __forceinline__ float3 rho3(const Mat &m, const Vtx &a, const Vtx &b, const Vtx &c) {
    return bsdf_eval(m, b.n, unit3(a.p - b.p), unit3(c.p - b.p));
}

// area density of `to` sampled at b conditioned on `from`
__device__ __forceinline__ float pdf3(const Mat &m, const Vtx &from, const Vtx &b, const Vtx &to) {
    return area_from_dir(bsdf_pdf(m, b.n, unit3(from.p - b.p), unit3(to.p - b.p)), b.p, to);
}

}  // namespace chain_detail
}  // namespace rp
