// Per-root evaluation of every base path of a root from per-vertex tables
// (the cumulative forward/backward pdf tables of Sec. 4.3, kept per vertex).
//
// The walk vertices of one root form a chain c_1 .. c_M ordered from the
// camera side to the light side:
//   technique (1):          z_nz .. z_1, x_D            (light end fixed: x_L)
//   technique (2):          x_D, y_1 .. y_ny            (camera end fixed: x_D)
//   technique (3):          z_nz .. z_1, x_D, y_1 .. y_ny
//   path tracing / (7):     x_1 .. x_len                (camera end fixed: x_1)
// Every base path is a sub-chain c_a .. c_b closed by the camera before c_a
// and by the next-event vertex L_b after c_b.  A chain vertex therefore
// appears in only four neighbourhoods -- interior (c_{i-1}, c_i, c_{i+1}),
// camera end (camera, c_i, c_{i+1}), light end (c_{i-1}, c_i, L_i) or both
// (camera, c_i, L_i) -- and its BSDF values and sampling densities are
// computed once per root, in both frames when the vertex lies on the edited
// object.  A path's contribution f (Eq. pathcontribution) and its balance
// heuristic denominator are then products of table entries, with the same
// definitions as path_throughput() and mis_denominator().
#pragma once

#include "rp_device.cuh"
#include "rp_wave.h"

namespace rp {

constexpr int kChain = 2 * kMaxDepth - 4;  // chain vertices per root: (3) has 2 (D - 3) + 1

struct ChainTables {
    int M;
    // geometry (frame independent)
    float Gn[kChain];      // G(c_i, c_{i+1})
    float pcos[kChain];    // cosine area density of c_{i+1} sampled at c_i
    float WeG0[kChain];    // camera importance times G(camera, c_i); 0 if not in the image
    float pcam[kChain];    // area density of c_i for a camera ray (path tracing)
    int pix[kChain];
    float GL[kChain];      // G(c_i, L_i)
    float3 Le[kChain];     // emission of L_i toward c_i
    unsigned dyn;          // bit i: c_i on the edited object
    unsigned camend, lightend;   // bit i: c_i may close the path on that side
    // per frame f in {0: base frame, 1: other frame}
    float3 rhoI[2][kChain], rhoC[2][kChain], rhoL[2][kChain], rhoB[2][kChain];
    float pEI[2][kChain], pLI[2][kChain], pEC[2][kChain], pLL[2][kChain];
};

namespace chain_detail {

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

// c: chain vertices (M of them), L: next-event vertex of each chain vertex
// (read only where lightend is set); g, g2: base and other frame
__device__ void build_tables(const Ctx &cx, int g, int g2, bool two_frames, const Vtx *c,
                             const Vtx *L, int M, unsigned camend, unsigned lightend,
                             ChainTables &T) {
    using namespace chain_detail;
    const DevScene &S = cx.A.S;
    const Vtx cam = camera_vertex(cx);
    T.M = M;
    T.dyn = 0u;
    T.camend = camend;
    T.lightend = lightend;
    for (int i = 0; i < M; ++i) {
        const bool d = is_dyn(cx, c[i]);
        if (d) T.dyn |= 1u << i;
        const int nf = (two_frames && d) ? 2 : 1;
        const Mat m0 = get_mat(cx, g, c[i].mat);
        const Mat m1 = get_mat(cx, g2, c[i].mat);
        if (i + 1 < M) {
            T.Gn[i] = G2(c[i], c[i + 1]);
            float3 w = unit3(c[i + 1].p - c[i].p);
            T.pcos[i] = area_from_dir(cosine_pdf(c[i].n, w), c[i].p, c[i + 1]);
        }
        if (camend & (1u << i)) {
            float cc;
            T.pix[i] = camera_project(S, c[i].p, cc);
            float3 d01 = cam.p - c[i].p;
            float r2 = dot3(d01, d01);
            float c1 = dot3(c[i].n, d01) / sqrtf(r2);
            if (T.pix[i] < 0 || c1 <= 0.f) {
                T.WeG0[i] = 0.f;
                T.pcam[i] = 0.f;
            } else {
                T.WeG0[i] = c1 / r2 / (S.pix_area * cc * cc * cc);
                T.pcam[i] = c1 / r2 / (S.film_area * cc * cc * cc);
            }
        }
        if (lightend & (1u << i)) {
            T.GL[i] = G2(c[i], L[i]);
            T.Le[i] = get_mat(cx, g, L[i].mat).em;
        }
        for (int f = 0; f < 2; ++f) {
            if (f == 1 && nf == 1) {
                T.rhoI[1][i] = T.rhoI[0][i]; T.rhoC[1][i] = T.rhoC[0][i];
                T.rhoL[1][i] = T.rhoL[0][i]; T.rhoB[1][i] = T.rhoB[0][i];
                T.pEI[1][i] = T.pEI[0][i]; T.pLI[1][i] = T.pLI[0][i];
                T.pEC[1][i] = T.pEC[0][i]; T.pLL[1][i] = T.pLL[0][i];
                break;
            }
            const Mat &m = f ? m1 : m0;
            if (i > 0 && i + 1 < M) {
                T.rhoI[f][i] = rho3(m, c[i - 1], c[i], c[i + 1]);
                T.pEI[f][i] = pdf3(m, c[i - 1], c[i], c[i + 1]);
                T.pLI[f][i] = pdf3(m, c[i + 1], c[i], c[i - 1]);
            }
            if ((camend & (1u << i)) && i + 1 < M) {
                T.rhoC[f][i] = rho3(m, cam, c[i], c[i + 1]);
                T.pEC[f][i] = pdf3(m, cam, c[i], c[i + 1]);
            }
            if ((lightend & (1u << i)) && i > 0) {
                T.rhoL[f][i] = rho3(m, c[i - 1], c[i], L[i]);
                T.pLL[f][i] = pdf3(m, L[i], c[i], c[i - 1]);
            }
            if ((camend & (1u << i)) && (lightend & (1u << i)))
                T.rhoB[f][i] = rho3(m, cam, c[i], L[i]);
        }
    }
}

// contribution of the sub-chain a..b (inclusive, 0-based) in frame slot f
__device__ __forceinline__ float3 chain_f(const ChainTables &T, int f, int a, int b) {
    float3 v = f3(T.WeG0[a], T.WeG0[a], T.WeG0[a]);
    if (a == b) return mul3(mul3(v, T.rhoB[f][a]) * T.GL[b], T.Le[b]);
    v = mul3(v, T.rhoC[f][a]) * T.Gn[a];
    for (int i = a + 1; i < b; ++i) v = mul3(v, T.rhoI[f][i]) * T.Gn[i];
    v = mul3(v, T.rhoL[f][b]) * T.GL[b];
    return mul3(v, T.Le[b]);
}

// balance-heuristic denominator of the sub-chain a..b in frame slot f: the
// sum over enabled techniques that produce the path of their densities
__device__ float chain_mis(const ChainTables &T, int f, int a, int b, int mask, float pD,
                           float pLi, bool residual) {
    const int k = b - a + 3;             // path vertices: camera, c_a..c_b, L_b
    float pE[kMaxVerts], pL[kMaxVerts], pc[kMaxVerts];
    pE[1] = T.pcam[a];
    for (int j = 2; j <= k - 2; ++j) {
        const int i = a + j - 2;
        pE[j] = (i == a) ? T.pEC[f][i] : T.pEI[f][i];
    }
    for (int j = 1; j <= k - 3; ++j) {
        const int i = a + j;
        pL[j] = (i == b) ? T.pLL[f][i] : T.pLI[f][i];
    }
    for (int j = 1; j <= k - 3; ++j) pc[j] = T.pcos[a + j - 1];
    float sum = 0.f;
    if (!residual || (mask & 8)) {
        float p = pLi;
        for (int j = 1; j <= k - 2; ++j) p *= pE[j];
        sum += p;
    }
    if (!residual) return sum;
    for (int i = 1; i <= k - 2; ++i) {
        if (!(T.dyn & (1u << (a + i - 1)))) continue;
        if (i == k - 2) {
            if (!(mask & 1)) continue;
            float p = pD * pLi;
            for (int j = 1; j <= k - 3; ++j) p *= pL[j];
            sum += p;
        } else if (i == 1) {
            if (!(mask & 2)) continue;
            float p = pD * pLi;
            for (int j = 2; j <= k - 2; ++j) p *= pE[j];
            sum += p;
        } else {
            if (!(mask & 4)) continue;
            float p = pD * pLi * pc[i];
            for (int j = i + 2; j <= k - 2; ++j) p *= pE[j];
            for (int j = 1; j <= i - 1; ++j) p *= pL[j];
            sum += p;
        }
    }
    return sum;
}

// no motion: the mapping is the identity; evaluate the sub-chain in both
// frames and splat (or record) the two-way contribution
__device__ void chain_emit(Ctx &cx, PathCounts &pc, const ChainTables &T, int a, int b,
                           uint32_t root, int tech, int sa, int sb) {
    const LaunchArgs &A = cx.A;
    const float pD = 1.0f / A.S.dyn_area, pLi = 1.0f / A.S.emit_area;
    const float invN = A.invN;
    const int g = A.frame;
    float3 fx = chain_f(T, 0, a, b);
    if (zero3(fx)) return;
    const int pa = T.pix[a];
    if (!A.residual) {
        const float p = chain_mis(T, 0, a, b, 0, pD, pLi, false);
        ++pc.paths;
        emit(cx, root, tech, g, sa, sb, pa, fx * (invN / p), -1, f3(0, 0, 0), 0, p, 0.f, 1.f);
        return;
    }
    ++pc.paths;
    const float sign = (g == 2) ? 1.0f : -1.0f;
    const float Pg = chain_mis(T, 0, a, b, A.tech_mask, pD, pLi, true);
    float3 fy = chain_f(T, 1, a, b);
    float Py = 0.f;
    int status = MAP_ACCEPT;
    if (zero3(fy)) {
        status = MAP_INVALID;
    } else {
        Py = chain_mis(T, 1, a, b, A.tech_mask, pD, pLi, true);
        if (!(Py > 0.f)) status = MAP_INVALID;
    }
    if (status == MAP_ACCEPT) {
        ++pc.accepted;
        const float den = (Pg + Py) / invN;
        emit(cx, root, tech, g, sa, sb, pa, fx * (sign / den), pa, fy * (-sign / den), status, Pg,
             Py, 1.0f);
    } else {
        emit(cx, root, tech, g, sa, sb, pa, fx * (sign * invN / Pg), -1, f3(0, 0, 0), status, Pg,
             0.f, 0.f);
    }
}

}  // namespace rp
