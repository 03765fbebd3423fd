// Evaluation of every base path of a root for edits without motion (and the
// primal), from running products along the root's walks -- the cumulative
// forward/backward pdf tables of Sec. 4.3 -- with O(1) work per path.
//
// Notation (p(a | b, c): area density of a sampled at c conditioned on b;
// rho(a, b, c): BSDF at b with camera-side neighbour a and light-side
// neighbour c).  Eye-side walk z_1 .. z_nz with z_0 = x_D; light-side walk
// y_1 .. y_ny with y_0 = x_D; a path of technique (3) is
// (camera, z_t .. z_1, x_D, y_1 .. y_s, L_s).  Per frame:
//   E(t)    = W_e G(cam, z_t) rho(cam, z_t, z_t-1) G(z_t, z_t-1)
//             prod_{m<t} rho(z_m+1, z_m, z_m-1) G(z_m, z_m-1)
//   Pf(t)   = prod_{m<t} p(z_m-1 | z_m+1, z_m)          (toward the light)
//   Pz(t)   = prod_{m<t} p(z_m+1 | z_m-1, z_m)          (toward the camera)
//   Sz(t)   = sum_{m<t, z_m dynamic} pcos(z_m) Pf(m) prod_{m<=m'<t} p(z_m'+1 | z_m'-1, z_m')
//   A(t)    = [7] p_cam(z_t) p(z_t-1 | cam, z_t) Pf(t)
//           + [2][z_t dynamic] pD p(z_t-1 | cam, z_t) Pf(t) + [3] pD Sz(t)
//   Ly(s)   = prod_{m<s} rho(y_m-1, y_m, y_m+1) G(y_m, y_m+1) rho(y_s-1, y_s, L_s) G(y_s, L_s) L_e
//   Py(s)   = prod_{m<s} p(y_m+1 | y_m-1, y_m)
//   PLy(m)  = prod_{m''<=m} p(y_m''-1 | y_m''+1, y_m'')
//   Sy(s)   = sum_{m<s, y_m dynamic} pcos(y_m) PLy(m) prod_{m<m'<s} p(y_m'+1 | y_m'-1, y_m')
//   B(s)    = [3] pD pcos(x_D) Py(s) + [1][y_s dynamic] pD PLy(s-1) p(y_s-1 | L_s, y_s) + [3] pD Sy(s)
// and with the x_D factors rho_D = rho(z_1, x_D, y_1), pE_D = p(y_1 | z_1, x_D),
// pL_D = p(z_1 | y_1, x_D):
//   f(t, s) = E(t) rho_D G(x_D, y_1) Ly(s)
//   P(t, s) = p_L (pE_D Py(s) A(t) + pL_D Pz(t) B(s))
// where [n] marks the terms of technique n (balance heuristic over the
// enabled techniques: path tracing [7] and one dynamic-vertex technique per
// vertex on the edited object, Sec. 4.3).  Techniques (1), (2) and path
// tracing are the same construction with one side fixed.  Both frames are
// evaluated (they differ only at vertices on the edited object).
#pragma once

#include "chain_eval.cuh"
#include "rp_device.cuh"

namespace rp {

namespace fast_detail {

constexpr int kSide = kMaxDepth;   // walk vertices per side (bound)

// frame-independent geometry of the camera connection of v
struct CamTerm {
    int pix;
    float we;      // W_e G(cam, v), 0 if not in the image or facing away
    float pcam;    // area density of v for a camera ray
};

__device__ __forceinline__ CamTerm cam_term(const DevScene &S, const Vtx &cam, const Vtx &v) {
    CamTerm c;
    float cc;
    c.pix = camera_project(S, v.p, cc);
    float3 d01 = cam.p - v.p;
    float r2 = dot3(d01, d01);
    float c1 = dot3(v.n, d01) / sqrtf(r2);
    if (c.pix < 0 || c1 <= 0.f) {
        c.we = 0.f;
        c.pcam = 0.f;
    } else {
        c.we = c1 / r2 / (S.pix_area * cc * cc * cc);
        c.pcam = c1 / r2 / (S.film_area * cc * cc * cc);
    }
    return c;
}

// Power-of-two rescaling of running products.  Near-coincident walk
// vertices make geometric terms and area densities of 1e8 and more per edge,
// so the products overflow single precision over a long walk.  Every value
// f(t, s) and every denominator P(t, s) is linear in the eye-side running
// state (E, A, Pz) and in the light-side running state (L, Py, B), so each
// side may be scaled by a common factor 2^e at any step (the same in both
// frames, whose sums Pg + Py share it) without changing f / P.
__device__ __forceinline__ int rescale_exp(float mx) {
    if (!(mx > 0x1p40f) && !(mx > 0.f && mx < 0x1p-40f)) return 0;
    int e;
    frexpf(mx, &e);
    return -e;
}

}  // namespace fast_detail

// splat one no-motion path (fx, Pg: base frame; fy, Py: other frame)
__device__ __forceinline__ void emit_nomotion(Ctx &cx, PathCounts &pc, uint32_t root, int tech,
                                              int sa, int sb, int pa, float3 fx, float Pg,
                                              float3 fy, float Py) {
    const LaunchArgs &A = cx.A;
    if (zero3(fx)) return;
    ++pc.paths;
    const float invN = A.invN;
    if (!A.residual) {            // primal: a single frame, path tracing alone
        emit(cx, root, tech, A.frame, sa, sb, pa, fx * (invN / Pg), -1, f3(0, 0, 0), 0, Pg, 0.f, 1.f);
        return;
    }
    const float sign = (A.frame == 2) ? 1.0f : -1.0f;
    if (!zero3(fy) && Py > 0.f) {
        ++pc.accepted;
        const float den = (Pg + Py) / invN;
        const float3 va = fx * (sign / den), vb = fy * (-sign / den);
        if (A.rec_count || (tech == T_3 && A.G.on)) {
            // records, or the learned proposal's value ratio and sample weights
            emit(cx, root, tech, A.frame, sa, sb, pa, va, pa, vb, MAP_ACCEPT, Pg, Py, 1.0f);
        } else if (A.img) {
            splat(A.img, pa, va + vb);    // both splats land on one pixel
        }
    } else {
        emit(cx, root, tech, A.frame, sa, sb, pa, fx * (sign * invN / Pg), -1, f3(0, 0, 0),
             MAP_INVALID, Pg, 0.f, 0.f);
    }
}

// Running states of the eye side (E, Pf, Pz, Sz) and of the light side
// (Ly, Py, PLy, Sy) for both frames, advanced one walk vertex at a time: the
// evaluators below read each vertex from the root's slots where it is
// needed (no thread-local copies of whole walks).  The rescaling exponent
// of a step is chosen in frame 0 and applied to both frames.
struct EyeRun {
    float3 rho[2];
    float Pf[2], Pz[2], Sz[2];
    __device__ void init() {
        for (int f = 0; f < 2; ++f) {
            rho[f] = f3(1.f, 1.f, 1.f);
            Pf[f] = Pz[f] = 1.f;
            Sz[f] = 0.f;
        }
    }
    // E(m), A(m), Pz(m) of the camera connection at z_m (zp = z_m-1)
    __device__ void cam_values(const Ctx &cx, const int *frames, int mask, float pD,
                               const fast_detail::CamTerm &ct, const Vtx &camv, const Vtx &zm,
                               const Vtx &zp, float G, bool dyn, float3 *E, float *A,
                               float *Pzt) const {
        using namespace chain_detail;
        for (int f = 0; f < 2; ++f) {
            const Mat mm = get_mat(cx, frames[f], zm.mat);
            const float pEC = pdf3(mm, camv, zm, zp);
            E[f] = mul3(rho[f], rho3(mm, camv, zm, zp)) * (ct.we * G);
            A[f] = ((mask & 8) ? ct.pcam * pEC * Pf[f] : 0.f) +
                   ((mask & 2) && dyn ? pD * pEC * Pf[f] : 0.f) + ((mask & 4) ? pD * Sz[f] : 0.f);
            Pzt[f] = Pz[f];
        }
    }
    // from z_m to z_m+1 = zn
    __device__ void advance(const Ctx &cx, const int *frames, const Vtx &zm, const Vtx &zp,
                            const Vtx &zn, float G, bool dyn) {
        using namespace chain_detail;
        int sh = 0;
        for (int f = 0; f < 2; ++f) {
            const Mat mm = get_mat(cx, frames[f], zm.mat);
            const float pLI = pdf3(mm, zp, zm, zn);
            if (dyn) Sz[f] += area_from_dir(cosine_pdf(zm.n, unit3(zp.p - zm.p)), zm.p, zp) * Pf[f];
            Sz[f] *= pLI;
            rho[f] = mul3(rho[f], rho3(mm, zn, zm, zp)) * G;
            Pf[f] *= pdf3(mm, zn, zm, zp);
            Pz[f] *= pLI;
            if (f == 0)
                sh = fast_detail::rescale_exp(fmaxf(fmaxf(fmaxf(rho[0].x, rho[0].y), fmaxf(rho[0].z, Pf[0])),
                                                    fmaxf(Pz[0], Sz[0])));
            if (sh) {
                const float sc = ldexpf(1.f, sh);
                rho[f] = rho[f] * sc; Pf[f] *= sc; Pz[f] *= sc; Sz[f] *= sc;
            }
        }
    }
};

struct LightRun {
    float3 rho[2];
    float Py[2], PLy[2], Sy[2];
    __device__ void init() {
        for (int f = 0; f < 2; ++f) {
            rho[f] = f3(1.f, 1.f, 1.f);
            Py[f] = PLy[f] = 1.f;
            Sy[f] = 0.f;
        }
    }
    // Ly(m), Py(m), B(m) of the next-event connection of y_m to Ls (yp = y_m-1)
    __device__ void nee_values(const Ctx &cx, const int *frames, int mask, float pD, float pcosD,
                               const Vtx &ym, const Vtx &yp, const Vtx &Ls, bool dyn, float3 *L,
                               float *Pyt, float *B) const {
        using namespace chain_detail;
        for (int f = 0; f < 2; ++f) {
            const Mat mm = get_mat(cx, frames[f], ym.mat);
            L[f] = mul3(mul3(rho[f], rho3(mm, yp, ym, Ls)) * G2(ym, Ls), get_mat(cx, frames[f], Ls.mat).em);
            Pyt[f] = Py[f];
            const float pLL = pdf3(mm, Ls, ym, yp);
            B[f] = ((mask & 4) ? pD * (pcosD * Py[f] + Sy[f]) : 0.f) +
                   ((mask & 1) && dyn ? pD * PLy[f] * pLL : 0.f);
        }
    }
    // from y_m to y_m+1 = yn
    __device__ void advance(const Ctx &cx, const int *frames, const Vtx &ym, const Vtx &yp,
                            const Vtx &yn, bool dyn) {
        using namespace chain_detail;
        int sh = 0;
        for (int f = 0; f < 2; ++f) {
            const Mat mm = get_mat(cx, frames[f], ym.mat);
            const float pLI = pdf3(mm, yn, ym, yp);
            const float pEI = pdf3(mm, yp, ym, yn);
            PLy[f] *= pLI;
            Sy[f] *= pEI;
            if (dyn) Sy[f] += area_from_dir(cosine_pdf(ym.n, unit3(yn.p - ym.p)), ym.p, yn) * PLy[f];
            rho[f] = mul3(rho[f], rho3(mm, yp, ym, yn)) * G2(ym, yn);
            Py[f] *= pEI;
            if (f == 0)
                sh = fast_detail::rescale_exp(fmaxf(fmaxf(fmaxf(rho[0].x, rho[0].y), fmaxf(rho[0].z, Py[0])),
                                                    fmaxf(PLy[0], Sy[0])));
            if (sh) {
                const float sc = ldexpf(1.f, sh);
                rho[f] = rho[f] * sc; Py[f] *= sc; PLy[f] *= sc; Sy[f] *= sc;
            }
        }
    }
};

// technique (3): all (t, s) paths of one root.  The light side is walked
// once: for each s with a next-event vertex its Ly(s), Py(s), B(s) of both
// frames (10 values) go to the thread's column of `sl` (shared memory,
// entry e of s at sl[((s - 1) * 10 + e) * stride]); then the eye-side state
// advances along t and pairs with them.  Vertices come from ld.vtx(slot),
// ld.eye(m), ld.light(m), ld.nee(m).  s never exceeds D - 3 (t >= 1).
constexpr int kT3LightSlots = kMaxDepth - 3;

template <class Ld>
__device__ void fast_t3(Ctx &cx, PathCounts &pc, uint32_t root, const Ld &ld, int nz,
                        uint32_t cam, int ny, uint32_t nee, float *sl, int stride) {
    using namespace chain_detail;
    using namespace fast_detail;
    const LaunchArgs &A = cx.A;
    const DevScene &Sc = A.S;
    const int g = A.frame, D = Sc.max_depth, mask = A.tech_mask;
    const int frames[2] = {g, 3 - g};
    const float pLi = 1.0f / Sc.emit_area, pD = 1.0f / Sc.dyn_area;
    const Vtx xD = ld.vtx(0);
    const Vtx y1 = ld.light(1);
    const float pcosD = area_from_dir(cosine_pdf(xD.n, unit3(y1.p - xD.p)), xD.p, y1);
    const int smax = ny < D - 3 ? ny : D - 3;
    {
        LightRun lr;
        lr.init();
        Vtx ym = y1, yp = xD;
        for (int s = 1; s <= smax; ++s) {
            const bool dyny = is_dyn(cx, ym);
            if (nee & (1u << s)) {
                float3 Ly[2];
                float Pyt[2], B[2];
                lr.nee_values(cx, frames, mask, pD, pcosD, ym, yp, ld.nee(s), dyny, Ly, Pyt, B);
                float *e = sl + (size_t)(s - 1) * 10 * stride;
                for (int f = 0; f < 2; ++f) {
                    e[(5 * f + 0) * stride] = Ly[f].x;
                    e[(5 * f + 1) * stride] = Ly[f].y;
                    e[(5 * f + 2) * stride] = Ly[f].z;
                    e[(5 * f + 3) * stride] = Pyt[f];
                    e[(5 * f + 4) * stride] = B[f];
                }
            }
            if (s < smax) {
                const Vtx yn = ld.light(s + 1);
                lr.advance(cx, frames, ym, yp, yn, dyny);
                yp = ym;
                ym = yn;
            }
        }
    }
    Vtx zm = ld.eye(1), zp = xD;
    const float Gd = G2(xD, y1);
    float3 rD[2];
    float pE[2], pL[2];
    for (int f = 0; f < 2; ++f) {
        const Mat m = get_mat(cx, frames[f], xD.mat);
        rD[f] = rho3(m, zm, xD, y1) * Gd;
        pE[f] = pdf3(m, zm, xD, y1);
        pL[f] = pdf3(m, y1, xD, zm);
    }
    const Vtx camv = camera_vertex(cx);
    EyeRun er;
    er.init();
    for (int t = 1; t <= nz; ++t) {
        const float G = G2(zm, zp);
        const bool dynz = is_dyn(cx, zm);
        if (cam & (1u << t)) {
            const CamTerm ct = cam_term(Sc, camv, zm);
            float3 E[2];
            float At[2], Pzt[2];
            er.cam_values(cx, frames, mask, pD, ct, camv, zm, zp, G, dynz, E, At, Pzt);
            for (int s = 1; s <= ny && t + s <= D - 2; ++s) {
                if (!(nee & (1u << s))) continue;
                const float *e = sl + (size_t)(s - 1) * 10 * stride;
                float3 fv[2];
                float P[2];
                for (int f = 0; f < 2; ++f) {
                    const float3 Ly = f3(e[(5 * f + 0) * stride], e[(5 * f + 1) * stride],
                                         e[(5 * f + 2) * stride]);
                    const float Pyt = e[(5 * f + 3) * stride], B = e[(5 * f + 4) * stride];
                    fv[f] = mul3(mul3(E[f], rD[f]), Ly);
                    P[f] = pLi * (pE[f] * Pyt * At[f] + pL[f] * Pzt[f] * B);
                }
                emit_nomotion(cx, pc, root, T_3, t, s, ct.pix, fv[0], P[0], fv[1], P[1]);
            }
        }
        if (t < nz) {
            const Vtx zn = ld.eye(t + 1);
            er.advance(cx, frames, zm, zp, zn, G, dynz);
            zp = zm;
            zm = zn;
        }
    }
}

// technique (1): paths (camera, z_t .. z_1, x_D, x_L), t = 0 .. nz
template <class Ld>
__device__ void fast_t1(Ctx &cx, PathCounts &pc, uint32_t root, const Ld &ld, int nz,
                               uint32_t cam) {
    using namespace chain_detail;
    using namespace fast_detail;
    const LaunchArgs &A = cx.A;
    const DevScene &Sc = A.S;
    const int g = A.frame, mask = A.tech_mask;
    const int frames[2] = {g, 3 - g};
    const float pD = 1.0f / Sc.dyn_area, pLi = 1.0f / Sc.emit_area;
    const Vtx xD = ld.vtx(0), xL = ld.vtx(1);
    const float3 Le = get_mat(cx, g, xL.mat).em * G2(xD, xL);
    const Vtx camv = camera_vertex(cx);
    if (cam & 1u) {                              // t = 0: (camera, x_D, x_L)
        const CamTerm ct = cam_term(Sc, camv, xD);
        if (ct.we > 0.f) {
            const float P = pLi * (((mask & 8) ? ct.pcam : 0.f) + ((mask & 1) ? pD : 0.f));
            const float3 base = Le * ct.we;
            emit_nomotion(cx, pc, root, T_1, 0, 0, ct.pix,
                          mul3(base, rho3(get_mat(cx, frames[0], xD.mat), camv, xD, xL)), P,
                          mul3(base, rho3(get_mat(cx, frames[1], xD.mat), camv, xD, xL)), P);
        }
    }
    if (nz == 0) return;
    Vtx zm = ld.eye(1), zp = xD;
    float3 rD[2];
    float pLL[2];
    for (int f = 0; f < 2; ++f) {
        const Mat m = get_mat(cx, frames[f], xD.mat);
        rD[f] = mul3(rho3(m, zm, xD, xL), Le);
        pLL[f] = pdf3(m, xL, xD, zm);
    }
    EyeRun er;
    er.init();
    for (int t = 1; t <= nz; ++t) {
        const float G = G2(zm, zp);
        const bool dynz = is_dyn(cx, zm);
        if (cam & (1u << t)) {
            const CamTerm ct = cam_term(Sc, camv, zm);
            float3 E[2];
            float At[2], Pzt[2];
            er.cam_values(cx, frames, mask, pD, ct, camv, zm, zp, G, dynz, E, At, Pzt);
            float3 fv[2];
            float P[2];
            for (int f = 0; f < 2; ++f) {
                fv[f] = mul3(E[f], rD[f]);
                P[f] = pLi * (At[f] + ((mask & 1) ? pD * Pzt[f] * pLL[f] : 0.f));
            }
            emit_nomotion(cx, pc, root, T_1, t, 0, ct.pix, fv[0], P[0], fv[1], P[1]);
        }
        if (t < nz) {
            const Vtx zn = ld.eye(t + 1);
            er.advance(cx, frames, zm, zp, zn, G, dynz);
            zp = zm;
            zm = zn;
        }
    }
}

// technique (2): paths (camera, x_D, y_1 .. y_s, L_s), s = 1 .. ny
template <class Ld>
__device__ void fast_t2(Ctx &cx, PathCounts &pc, uint32_t root, const Ld &ld, int ny,
                               uint32_t nee) {
    using namespace chain_detail;
    using namespace fast_detail;
    const LaunchArgs &A = cx.A;
    const DevScene &Sc = A.S;
    const int g = A.frame, mask = A.tech_mask;
    const int frames[2] = {g, 3 - g};
    const float pD = 1.0f / Sc.dyn_area, pLi = 1.0f / Sc.emit_area;
    const Vtx xD = ld.vtx(0);
    const Vtx camv = camera_vertex(cx);
    const CamTerm ct = cam_term(Sc, camv, xD);
    if (ct.we <= 0.f || ny == 0) return;
    Vtx ym = ld.light(1), yp = xD;
    const float Gd = G2(xD, ym);
    const float a = ((mask & 8) ? ct.pcam : 0.f) + ((mask & 2) ? pD : 0.f);
    float3 rD[2];
    float pEC[2];
    for (int f = 0; f < 2; ++f) {
        const Mat m = get_mat(cx, frames[f], xD.mat);
        rD[f] = rho3(m, camv, xD, ym) * (ct.we * Gd);
        pEC[f] = pdf3(m, camv, xD, ym);
    }
    LightRun lr;
    lr.init();
    for (int s = 1; s <= ny; ++s) {
        const bool dyny = is_dyn(cx, ym);
        if (nee & (1u << s)) {
            float3 Ly[2];
            float Pyt[2], B[2];
            // x_D is technique (2) here: no technique-(3) term at x_D
            lr.nee_values(cx, frames, mask, pD, 0.f, ym, yp, ld.nee(s), dyny, Ly, Pyt, B);
            float3 fv[2];
            float P[2];
            for (int f = 0; f < 2; ++f) {
                fv[f] = mul3(rD[f], Ly[f]);
                P[f] = pLi * (a * pEC[f] * Pyt[f] + B[f]);
            }
            emit_nomotion(cx, pc, root, T_2, 0, s, ct.pix, fv[0], P[0], fv[1], P[1]);
        }
        if (s < ny) {
            const Vtx yn = ld.light(s + 1);
            lr.advance(cx, frames, ym, yp, yn, dyny);
            yp = ym;
            ym = yn;
        }
    }
}

// path tracing: paths (camera, x_1 .. x_j, L_j); residual (technique (7),
// both frames, static paths skipped) or primal (one frame, path tracing only)
template <class Ld>
__device__ void fast_pt(Ctx &cx, PathCounts &pc, uint32_t root, const Ld &ld, int len,
                        uint32_t nee, int tech) {
    using namespace chain_detail;
    const LaunchArgs &A = cx.A;
    const DevScene &Sc = A.S;
    const int g = A.frame;
    const bool res = A.residual != 0;
    const int mask = res ? A.tech_mask : 8;
    const int nf = res ? 2 : 1;
    const int frames[2] = {g, 3 - g};
    const float pD = 1.0f / Sc.dyn_area, pLi = 1.0f / Sc.emit_area;
    const Vtx camv = camera_vertex(cx);
    Vtx xj = ld.vtx(0), xp = camv;      // x_1 is in slot 0, x_m (m >= 2) in light slot m - 1
    const fast_detail::CamTerm ct = fast_detail::cam_term(Sc, camv, xj);
    if (ct.we <= 0.f) return;
    if (!res) {                    // the camera ray sees an emitter: (camera, x_1)
        const float3 em = get_mat(cx, g, xj.mat).em;
        if (!zero3(em)) emit_nomotion(cx, pc, root, tech, 0, 2, ct.pix, em * ct.we, ct.pcam, em, 0.f);
    }
    const bool d1 = is_dyn(cx, xj);
    float3 R[2] = {f3(ct.we, ct.we, ct.we), f3(ct.we, ct.we, ct.we)};
    float PE[2] = {1.f, 1.f}, PL[2] = {1.f, 1.f}, S3[2] = {0.f, 0.f};
    bool any_dyn = false;
    for (int j = 1; j <= len; ++j) {
        const bool dj = is_dyn(cx, xj);
        any_dyn = any_dyn || dj;
        if ((nee & (1u << j)) && (!res || any_dyn)) {
            const Vtx Lj = ld.nee(j);
            const float GL = G2(xj, Lj);
            float3 fv[2];
            float P[2] = {0.f, 0.f};
            for (int f = 0; f < nf; ++f) {
                const Mat m = get_mat(cx, frames[f], xj.mat);
                fv[f] = mul3(mul3(R[f], rho3(m, xp, xj, Lj)) * GL, get_mat(cx, frames[f], Lj.mat).em);
                float p = ((mask & 8) ? ct.pcam * PE[f] : 0.f) +
                          ((mask & 2) && d1 && j >= 2 ? pD * PE[f] : 0.f) + ((mask & 4) ? pD * S3[f] : 0.f);
                if ((mask & 1) && dj) p += pD * (j == 1 ? 1.f : PL[f] * pdf3(m, Lj, xj, xp));
                P[f] = pLi * p;
            }
            emit_nomotion(cx, pc, root, tech, 0, j + 2, ct.pix, fv[0], P[0], fv[1], P[1]);
        }
        if (j < len) {
            const Vtx xn = ld.light(j);
            for (int f = 0; f < nf; ++f) {
                const Mat m = get_mat(cx, frames[f], xj.mat);
                const float pE = pdf3(m, xp, xj, xn);
                R[f] = mul3(R[f], rho3(m, xp, xj, xn)) * G2(xj, xn);
                S3[f] *= pE;
                if (j >= 2) {
                    PL[f] *= pdf3(m, xn, xj, xp);
                    if (dj) S3[f] += area_from_dir(cosine_pdf(xj.n, unit3(xn.p - xj.p)), xj.p, xn) * PL[f];
                }
                PE[f] *= pE;
            }
            float mx = 0.f;
            for (int f = 0; f < nf; ++f)
                mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(R[f].x, R[f].y), fmaxf(R[f].z, PE[f])),
                                     fmaxf(PL[f], S3[f])));
            const int e = fast_detail::rescale_exp(mx);
            if (e) {
                const float sc = ldexpf(1.f, e);
                for (int f = 0; f < nf; ++f) {
                    R[f] = R[f] * sc; PE[f] *= sc; PL[f] *= sc; S3[f] *= sc;
                }
            }
            xp = xj;
            xj = xn;
        }
    }
}

}  // namespace rp
