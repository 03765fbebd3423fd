// The per-element work of the wavefront kernels: root generation, walks,
// traversal, path enumeration and evaluation, and the path mapping, each as a
// device function (*_body) applied to one root, ray or mapping task of one
// wave described by a LaunchArgs.  The kernels of k_wave.cu run one wave per
// launch over these functions; the persistent batch kernel of k_batch.cu
// runs many waves (jobs) in one launch over the same functions.
//
// Wavefront execution of one wave of roots of one technique in one frame.
//
// Stage A (walks):   k_gen -> [k_trace_shadow -> k_start] ->
//                    { k_trace_closest -> k_extend -> k_trace_shadow } x depth
//   Rays live in SoA queues; kernels append with one atomic per coalesced
//   group of threads.  Walk vertices are stored in per-root vertex slots,
//   connection visibility in per-root bit masks.
// Stage B (k_eval):  one thread per root enumerates the base paths of its
//   technique from the slots and masks.  Without motion (material or
//   identity edits) the mapping is the identity and the path is evaluated and
//   splatted here with no ray at all; with motion every non-static path
//   becomes a mapping task.
// Stage C (motion):  the path mapping as queued rounds: k_map_start runs
//   each task's mapping program (object transform or camera replay, then
//   per walk vertex unchanged, reconnection or random replay) until it
//   needs a replay ray; k_replay_dir finds the round's replay directions,
//   k_trace_map traces the replay rays in the other frame and k_map_step
//   resumes the tasks with their hits.  k_map_fin
//   evaluates base and mapped paths with two-way MIS; the mapped path's
//   edges that need a visibility test go to a queue traced by k_trace_vis,
//   and k_map_b emits the pairs.
//
// The random numbers, walk termination rules and path enumeration are those
// of the one-thread-per-root kernels (rp_device.cuh), so both modes produce
// the same samples.
#pragma once

#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "chain_fast.cuh"
#include "guide_device.cuh"
#include "rp_device.cuh"

namespace cg = cooperative_groups;

// blocks per SM the mapping kernels are compiled for (register budgets:
// 6 blocks of 128 threads, up to 80 registers and less local memory, did
// 0.3-0.6 % better per render than 8 blocks at 64 registers, 4 worse)
#ifndef RP_MAP_MINBLOCKS
#define RP_MAP_MINBLOCKS 6
#endif
#ifndef RP_MAPFIN_MINBLOCKS
#define RP_MAPFIN_MINBLOCKS 6
#endif

namespace rp {

// Per-thread state a kernel carries across the elements it processes (work
// counters of the statistics, scratch arrays), handed to the per-element
// work functions below.
struct BodyState {
    PathCounts pc;
    unsigned int roots, accepted;
    Vtx *x;                     // a path vertex array (kMaxVerts) of the mapping kernels
    float *s_light;             // technique (3)'s shared light-side values
};


namespace {

enum { SIDE_ROOT = 0, SIDE_EYE = 1, SIDE_LIGHT = 2 };

// one atomicAdd per coalesced group of appending threads
__device__ __forceinline__ uint32_t append(unsigned int *counter) {
    cg::coalesced_group g = cg::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned int)g.size());
    base = g.shfl(base, 0);
    return base + g.thread_rank();
}

__device__ __forceinline__ void store3(float *a, uint32_t stride, uint32_t i, float3 v) {
    a[i] = v.x;
    a[stride + i] = v.y;
    a[2 * stride + i] = v.z;
}

__device__ __forceinline__ float3 load3(const float *a, uint32_t stride, uint32_t i) {
    return f3(a[i], a[stride + i], a[2 * stride + i]);
}

__device__ __forceinline__ void store_vtx(const WaveBuf &W, int slot, uint32_t r, const Vtx &v) {
    const size_t i = (size_t)slot * W.R + r;
    W.px[i] = v.p.x; W.py[i] = v.p.y; W.pz[i] = v.p.z;
    W.nx[i] = v.n.x; W.ny[i] = v.n.y; W.nz[i] = v.n.z;
    W.b1[i] = v.b1; W.b2[i] = v.b2;
    W.prim[i] = v.prim;
}

__device__ __forceinline__ Vtx load_vtx(const Ctx &c, const WaveBuf &W, int slot, uint32_t r) {
    const size_t i = (size_t)slot * W.R + r;
    Vtx v;
    v.p = f3(W.px[i], W.py[i], W.pz[i]);
    v.n = f3(W.nx[i], W.ny[i], W.nz[i]);
    v.b1 = W.b1[i];
    v.b2 = W.b2[i];
    v.prim = W.prim[i];
    v.mat = v.prim < c.A.S.n_static ? (int)c.A.S.stat_mat[v.prim] : kMatDynamic - inst_of(c.A.S, v.prim);
    return v;
}

// a root's walk vertices read from its slots where they are needed
struct SlotLoader {
    const Ctx &c;
    const WaveBuf &W;
    uint32_t r;
    int D;
    __device__ Vtx vtx(int slot) const { return load_vtx(c, W, slot, r); }
    __device__ Vtx eye(int m) const { return load_vtx(c, W, slot_eye(D, m), r); }
    __device__ Vtx light(int m) const { return load_vtx(c, W, slot_light(D, m), r); }
    __device__ Vtx nee(int m) const { return load_vtx(c, W, slot_nee(D, m), r); }
};

__device__ __forceinline__ void push_closest(const LaunchArgs &A, int buf, int it, float3 o,
                                             float3 d, int ex, uint32_t tag) {
    const WaveBuf &W = A.W;
    uint32_t i = append(W.counts + cnt_closest(it));
    if (i >= W.qc) return;          // capacity is sized so that this cannot happen
    W.c_o[buf][i] = o.x; W.c_o[buf][W.qc + i] = o.y; W.c_o[buf][2 * W.qc + i] = o.z;
    W.c_d[buf][i] = d.x; W.c_d[buf][W.qc + i] = d.y; W.c_d[buf][2 * W.qc + i] = d.z;
    W.c_ex[buf][i] = ex;
    W.c_tag[buf][i] = tag;
}

// shadow ray over the open segment a -> b
__device__ __forceinline__ void push_shadow(const LaunchArgs &A, int it, const Vtx &a, const Vtx &b,
                                            uint32_t tag) {
    const WaveBuf &W = A.W;
    float3 e = b.p - a.p;
    float dist = len3(e);
    float3 d = e * (1.0f / dist);
    uint32_t i = append(W.counts + cnt_shadow(it));
    if (i >= W.qa) return;
    W.a_o[i] = a.p.x; W.a_o[W.qa + i] = a.p.y; W.a_o[2 * W.qa + i] = a.p.z;
    W.a_d[i] = d.x; W.a_d[W.qa + i] = d.y; W.a_d[2 * W.qa + i] = d.z;
    W.a_tmax[i] = dist - A.S.eps;
    W.a_ex0[i] = a.prim;
    W.a_ex1[i] = b.prim;
    W.a_tag[i] = tag;
}

__device__ __forceinline__ bool in_image_facing(const Ctx &c, const Vtx &z) {
    float cc;
    if (camera_project(c.A.S, z.p, cc) < 0) return false;
    return faces(z, c.A.S.cam_pos);
}

// push the BSDF-sampled continuation of a walk at `at` (previous vertex
// `prev`) with the numbers of (side, step)
__device__ __forceinline__ void continue_walk(const Ctx &c, int buf, int it, uint32_t r,
                                              const Vtx &prev, const Vtx &at, int tech, int rg,
                                              int side, int step) {
    const LaunchArgs &A = c.A;
    float4 u = draw(lseed(A), A.root_begin + r, tech, rg, side, step);
    float3 wc = unit3(prev.p - at.p);
    float3 wo;
    Mat m = get_mat(c, A.frame, at.mat);
    if (!bsdf_sample_walk(A.S, m, at.n, wc, u.x, u.y, wo)) return;
    push_closest(A, buf, it, at.p, wo, at.prim, make_tag(r, side, step));
}

}  // namespace

// --- stage A ---------------------------------------------------------------

// the per-element work of k_gen
template <int T>
__device__ __forceinline__ void gen_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t r, int it) {
    const WaveBuf &W = A.W;
    const int g = A.frame, D = A.S.max_depth;
    do {
        const uint32_t root = A.root_begin + r;
        W.len_eye[r] = 0;
        W.len_light[r] = 0;
        W.flags[r] = 0;
        W.cam_ok[r] = 0u;
        W.nee_ok[r] = 0u;
        W.ghost_w[r] = 0u;
        W.ghost_n[r] = 0u;
        if (T == T_1 || T == T_2 || T == T_3) {
            Vtx xD = sample_dynamic(c, g, draw(lseed(A), root, T, g, SD_ROOT, 0));
            store_vtx(W, 0, r, xD);
            if (T == T_1) {
                Vtx xL = sample_emitter(c, g, draw(lseed(A), root, T_1, g, SD_NEE, 0));
                store_vtx(W, 1, r, xL);
                if (faces(xD, xL.p) && faces(xL, xD.p)) push_shadow(A, 0, xD, xL, make_tag(r, CK_NEE, 0));
            } else if (T == T_2) {
                if (!vtx_black(c, g, xD) && in_image_facing(c, xD))
                    push_shadow(A, 0, xD, camera_vertex(c), make_tag(r, CK_CAMERA, 0));
            } else {
                const bool live = D >= 4 && !vtx_black(c, g, xD);
                if (A.G.on) {
                    // learned proposal: object-space x_D and normal for the
                    // network's input and the training samples (edits of one
                    // object only)
                    const float4 ur = draw(lseed(A), root, T_3, g, SD_ROOT, 0);
                    const int q = xD.prim - A.S.n_static;
                    double b1, b2;
                    tri_sample(ur.y, ur.z, b1, b2);
                    const float4 *tq = A.S.inst[0].tri + 3 * q;
                    const float4 ta = tq[0], tb = tq[1], tcv = tq[2];
                    const double3 v0 = d3(ta);
                    const double3 po = dadd(dadd(v0, dscale(dsub(d3(tb), v0), b1)),
                                            dscale(dsub(d3(tcv), v0), b2));
                    const float3 no = f3(ta.w, tb.w, tcv.w);
                    const uint32_t slot = guide_slot(A.G, g, root);
                    if (slot != ~0u) {
                        const uint32_t C = A.G.smp.cap;
                        A.G.smp.p[slot] = (float)po.x; A.G.smp.p[C + slot] = (float)po.y;
                        A.G.smp.p[2 * C + slot] = (float)po.z;
                        A.G.smp.n[slot] = no.x; A.G.smp.n[C + slot] = no.y; A.G.smp.n[2 * C + slot] = no.z;
                        A.G.smp.wt[slot] = 0.f;
                    }
                    if (A.G.use_net) {
                        if (live) W.flags[r] = RF_GUIDE;
                        continue;       // encoded by k_encode3, drawn after inference by k_start3g
                    }
                }
                if (live) {
                    float4 u = draw(lseed(A), root, T_3, g, SD_LIGHT, 1);
                    float3 w = cosine_dir_walk(A.S, xD.n, u.x, u.y);
                    if (A.G.on) {
                        const uint32_t slot = guide_slot(A.G, g, root);
                        if (slot != ~0u) {
                            const double3 wl = dlinear_T(A.E.M(0, g), d3(w));
                            const uint32_t C = A.G.smp.cap;
                            A.G.smp.w[slot] = (float)wl.x; A.G.smp.w[C + slot] = (float)wl.y;
                            A.G.smp.w[2 * C + slot] = (float)wl.z;
                        }
                    }
                    if (dot3(xD.n, w) > 0.f) push_closest(A, 0, 0, xD.p, w, xD.prim, make_tag(r, SIDE_LIGHT, 1));
                }
            }
        } else if (T == T_4 || T == T_5 || T == T_6) {
            // ghost techniques: a point on the ghost (the object at its pose
            // of the other frame) by area (Sec. 4.2)
            const Vtx xG = sample_dynamic(c, 3 - g, draw(lseed(A), root, T, g, SD_ROOT, 0));
            if (T == T_4) {
                const Vtx xL = sample_emitter(c, g, draw(lseed(A), root, T_4, g, SD_NEE, 0));
                store_vtx(W, 1, r, xL);
                const float3 w = unit3(xG.p - xL.p);
                if (dot3(xL.n, w) > 0.f) push_closest(A, 0, 0, xL.p, w, xL.prim, make_tag(r, SIDE_ROOT, 0));
            } else if (T == T_5) {
                float cc;
                if (camera_project(A.S, xG.p, cc) >= 0)
                    push_closest(A, 0, 0, A.S.cam_pos, unit3(xG.p - A.S.cam_pos), -1,
                                 make_tag(r, SIDE_ROOT, 0));
            } else if (D >= 3) {
                // two rays from x_G along a uniform direction w and along -w
                Vtx g0 = xG;
                g0.prim = -1;
                store_vtx(W, 0, r, g0);
                const float4 u = draw(lseed(A), root, T_6, g, SD_ROOT, 1);
                const double zc = 1.0 - 2.0 * (double)u.x, rs = sqrt(fmax(0.0, 1.0 - zc * zc));
                double sp, cp;
                sincos2pi(A.S, u.y, sp, cp);
                const float3 w = tof(d3(rs * cp, rs * sp, zc));
                push_closest(A, 0, 0, xG.p, w, -1, make_tag(r, SIDE_LIGHT, 1));
                push_closest(A, 0, 0, xG.p, w * -1.f, -1, make_tag(r, SIDE_EYE, 1));
            }
        } else {
            // path tracing: a stratified camera ray through pixel root mod (W H)
            const int tech = A.residual ? T_7 : T_PT;
            const int rg = A.residual ? g : 0;
            const uint32_t npix = (uint32_t)(A.S.W * A.S.H);
            const int pix = (int)(root % npix);
            float4 u = draw(lseed(A), root, tech, rg, SD_ROOT, 0);
            float3 d = camera_dir(A.S, pix % A.S.W, pix / A.S.W, u.x, u.y);
            push_closest(A, 0, 0, A.S.cam_pos, d, -1, make_tag(r, SIDE_ROOT, 0));
        }
    } while (0);
}






// the per-element work of k_start
template <int T>
__device__ __forceinline__ void start_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t r, int it) {
    const WaveBuf &W = A.W;
    const int g = A.frame, D = A.S.max_depth;
    do {
        if (T == T_1) {
            if (!(W.nee_ok[r] & 1u)) continue;
            Vtx xD = load_vtx(c, W, 0, r);
            if (vtx_black(c, g, xD)) continue;
            W.flags[r] = RF_ROOT_OK;
            if (in_image_facing(c, xD)) push_shadow(A, 1, xD, camera_vertex(c), make_tag(r, CK_CAMERA, 0));
            if (D - 2 >= 1) {
                Vtx xL = load_vtx(c, W, 1, r);
                continue_walk(c, 0, 0, r, xL, xD, T_1, g, SD_EYE, 1);
            }
        } else {
            if (!(W.cam_ok[r] & 1u)) continue;
            W.flags[r] = RF_ROOT_OK;
            if (D - 2 >= 1) {
                Vtx xD = load_vtx(c, W, 0, r);
                continue_walk(c, 0, 0, r, camera_vertex(c), xD, T_2, g, SD_LIGHT, 1);
            }
        }
    } while (0);
}


// the per-element work of k_extend
template <int T>
__device__ __forceinline__ void extend_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int in = (it - 1) & 1, out = it & 1;
    const int g = A.frame, D = A.S.max_depth;
    const int tech = (T == T_PT) ? (A.residual ? T_7 : T_PT) : T;
    const int rg = (T == T_PT && !A.residual) ? 0 : g;
    const bool ghosts = (T == T_PT) && A.residual && A.E.motion;
    constexpr bool camera_walk = (T == T_PT || T == T_5);      // x_1 from the camera, NEE at every vertex
    do {
        const int prim = W.h_prim[i];
        if (prim < 0) continue;
        const uint32_t tag = W.c_tag[in][i];
        const uint32_t r = tag_root(tag);
        const int side = tag_side(tag), m = tag_step(tag);
        const uint32_t root = A.root_begin + r;
        const float3 d = f3(W.c_d[in][i], W.c_d[in][W.qc + i], W.c_d[in][2 * W.qc + i]);
        Vtx v = make_vertex_at(c, g, prim, W.h_b1[i], W.h_b2[i],
                               f3(W.h_p[i], W.h_p[W.qc + i], W.h_p[2 * W.qc + i]));
        if (dot3(v.n, d) >= 0.f) continue;                     // back face
        if ((T == T_4 || T == T_5) && side == SIDE_ROOT) {
            // the first vertex must lie behind the ghost point on its ray
            const Vtx xG = sample_dynamic(c, 3 - g, draw(lseed(A), root, T, g, SD_ROOT, 0));
            const float3 o = (T == T_4) ? load_vtx(c, W, 1, r).p : A.S.cam_pos;
            if (len3(v.p - o) <= len3(xG.p - o)) continue;
        }
        if (T == T_4 && side == SIDE_ROOT) {
            // technique (4): x_1 from x_L through the ghost, then as technique (1)
            if (vtx_black(c, g, v)) continue;
            store_vtx(W, 0, r, v);
            W.flags[r] = RF_ROOT_OK;
            if (in_image_facing(c, v)) push_shadow(A, it + 1, v, camera_vertex(c), make_tag(r, CK_CAMERA, 0));
            if (D - 2 >= 1) continue_walk(c, out, it, r, load_vtx(c, W, 1, r), v, T_4, g, SD_EYE, 1);
            continue;
        }
        if (camera_walk) {
            // x_{j} with j = 1 (camera hit) or j = m + 1 (walk step m)
            const int j = (side == SIDE_ROOT) ? 1 : m + 1;
            store_vtx(W, j == 1 ? 0 : slot_light(D, m), r, v);
            W.len_light[r] = j;
            Vtx prev = (j == 1) ? camera_vertex(c) : load_vtx(c, W, j == 2 ? 0 : slot_light(D, j - 2), r);
            if (ghosts) push_shadow(A, it + 1, prev, v, make_tag(r, CK_GHOST_WALK, j));
            if (vtx_black(c, g, v)) continue;
            Vtx L = sample_emitter(c, g, draw(lseed(A), root, tech, rg, SD_NEE, j));
            store_vtx(W, slot_nee(D, j), r, L);
            if (faces(v, L.p) && faces(L, v.p)) {
                push_shadow(A, it + 1, v, L, make_tag(r, CK_NEE, j));
                if (ghosts) push_shadow(A, it + 1, v, L, make_tag(r, CK_GHOST_NEE, j));
            }
            if (j < D - 1) continue_walk(c, out, it, r, prev, v, tech, rg, SD_LIGHT, j);
            continue;
        }
        // the previous vertex of a walk's first vertex: x_D, or for technique (6)
        // the ghost point (on the same line as the other first vertex)
        auto first_prev = [&]() -> Vtx {
            if (T == T_6) {
                Vtx p;
                const size_t i0 = r;
                p.p = f3(W.px[i0], W.py[i0], W.pz[i0]);
                p.n = f3(0.f, 0.f, 0.f);
                p.prim = -1;
                p.mat = kMatCamera;
                p.b1 = p.b2 = 0.f;
                return p;
            }
            return load_vtx(c, W, 0, r);
        };
        if (vtx_black(c, g, v)) continue;
        if (side == SIDE_EYE) {
            // techniques (1) and (3): eye-side walk vertex z_m
            store_vtx(W, slot_eye(D, m), r, v);
            W.len_eye[r] = m;
            if (in_image_facing(c, v)) push_shadow(A, it + 1, v, camera_vertex(c), make_tag(r, CK_CAMERA, m));
            const int last = (T == T_1 || T == T_4 || T == T_6) ? D - 2 : D - 3;
            if (m < last) {
                Vtx prev = m == 1 ? first_prev() : load_vtx(c, W, slot_eye(D, m - 1), r);
                continue_walk(c, out, it, r, prev, v, T, g, SD_EYE, m + 1);
            }
        } else {
            // techniques (2) and (3): light-side walk vertex y_m with next-event estimation
            store_vtx(W, slot_light(D, m), r, v);
            W.len_light[r] = m;
            Vtx L = sample_emitter(c, g, draw(lseed(A), root, T, g, SD_NEE, m));
            store_vtx(W, slot_nee(D, m), r, L);
            if (faces(v, L.p) && faces(L, v.p)) push_shadow(A, it + 1, v, L, make_tag(r, CK_NEE, m));
            const int last = (T == T_2 || T == T_6) ? D - 2 : D - 3;
            Vtx prev = m == 1 ? first_prev() : load_vtx(c, W, slot_light(D, m - 1), r);
            if (m < last) continue_walk(c, out, it, r, prev, v, T, g, SD_LIGHT, m + 1);
            if (T == T_3 && m == 1) {
                // the eye side of (3) starts at x_D, conditioned on y_1
                continue_walk(c, out, it, r, v, prev, T_3, g, SD_EYE, 1);
            }
        }
    } while (0);
}


// the per-element work of k_trace_closest
__device__ __forceinline__ void trace_closest_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int b = it & 1;
    const float inf = __int_as_float(0x7f800000);
    do {
        float3 o = f3(W.c_o[b][i], W.c_o[b][W.qc + i], W.c_o[b][2 * W.qc + i]);
        float3 d = f3(W.c_d[b][i], W.c_d[b][W.qc + i], W.c_d[b][2 * W.qc + i]);
        Hit h;
        ++c.cnt.rays_closest;
        if (scene_trace(c, A.frame, o, d, A.S.eps, inf, W.c_ex[b][i], -1, false, false, h)) {
            W.h_prim[i] = h.prim;
            W.h_b1[i] = h.b1;
            W.h_b2[i] = h.b2;
            W.h_p[i] = h.p.x;
            W.h_p[W.qc + i] = h.p.y;
            W.h_p[2 * W.qc + i] = h.p.z;
        } else {
            W.h_prim[i] = -1;
        }
    } while (0);
}


// the per-element work of k_trace_shadow
__device__ __forceinline__ void trace_shadow_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    do {
        const uint32_t tag = W.a_tag[i];
        const uint32_t r = tag_root(tag);
        const int kind = tag_side(tag), step = tag_step(tag);
        float3 o = f3(W.a_o[i], W.a_o[W.qa + i], W.a_o[2 * W.qa + i]);
        float3 d = f3(W.a_d[i], W.a_d[W.qa + i], W.a_d[2 * W.qa + i]);
        const bool ghost = kind >= CK_GHOST_WALK;
        Hit h;
        ++c.cnt.rays_shadow;
        bool hit = scene_trace(c, ghost ? 3 - A.frame : A.frame, o, d, A.S.eps, W.a_tmax[i],
                               W.a_ex0[i], W.a_ex1[i], true, ghost, h);
        const uint32_t bit = 1u << step;
        if (kind == CK_CAMERA && !hit) atomicOr(W.cam_ok + r, bit);
        else if (kind == CK_NEE && !hit) atomicOr(W.nee_ok + r, bit);
        else if (kind == CK_GHOST_WALK && hit) atomicOr(W.ghost_w + r, bit);
        else if (kind == CK_GHOST_NEE && hit) atomicOr(W.ghost_n + r, bit);
    } while (0);
}


// --- stage B ---------------------------------------------------------------

namespace {

// queue a mapping task for base path (tech, sa, sb) of root r
__device__ __forceinline__ void dispatch_path(Ctx &c, PathCounts &pc, const Vtx *x, int n,
                                              uint32_t r, int tech, int sa, int sb) {
    (void)pc; (void)x; (void)n;
    const LaunchArgs &A = c.A;
    uint32_t i = append(A.W.counts + cnt_tasks());
    if (i < A.W.qt) A.W.tasks[i] = make_int4((int)r, tech, sa, sb);
}

// the vertices of base path (tech, sa, sb) of root r, read from the slots;
// returns the vertex count
__device__ int assemble(const Ctx &c, uint32_t r, int tech, int sa, int sb, Vtx *x) {
    const WaveBuf &W = c.A.W;
    const int D = c.A.S.max_depth;
    x[0] = camera_vertex(c);
    if (tech == T_6) {                       // (cam, z_te..z_1, y_1..y_sl, L_sl)
        const int te = sa, sl = sb;
        for (int j = 0; j < te; ++j) x[1 + j] = load_vtx(c, W, slot_eye(D, te - j), r);
        for (int j = 1; j <= sl; ++j) x[te + j] = load_vtx(c, W, slot_light(D, j), r);
        x[te + sl + 1] = load_vtx(c, W, slot_nee(D, sl), r);
        return te + sl + 2;
    }
    if (tech == T_1 || tech == T_4) {        // (cam, z_t, ..., z_1, x_D, x_L), t = sa
        const int t = sa;
        for (int j = 0; j < t; ++j) x[1 + j] = load_vtx(c, W, slot_eye(D, t - j), r);
        x[t + 1] = load_vtx(c, W, 0, r);
        x[t + 2] = load_vtx(c, W, 1, r);
        return t + 3;
    }
    if (tech == T_2) {                       // (cam, x_D, y_1, ..., y_s, L_s), s = sb
        const int s = sb;
        x[1] = load_vtx(c, W, 0, r);
        for (int j = 1; j <= s; ++j) x[1 + j] = load_vtx(c, W, slot_light(D, j), r);
        x[s + 2] = load_vtx(c, W, slot_nee(D, s), r);
        return s + 3;
    }
    if (tech == T_3) {                       // (cam, z_te..z_1, x_D, y_1..y_sl, L_sl)
        const int te = sa, sl = sb;
        for (int j = 0; j < te; ++j) x[1 + j] = load_vtx(c, W, slot_eye(D, te - j), r);
        x[te + 1] = load_vtx(c, W, 0, r);
        for (int j = 1; j <= sl; ++j) x[te + 1 + j] = load_vtx(c, W, slot_light(D, j), r);
        x[te + sl + 2] = load_vtx(c, W, slot_nee(D, sl), r);
        return te + sl + 3;
    }
    // path tracing: k = sb vertices (cam, x_1, ..., x_{k-2}, L_{k-2}) or (cam, x_1)
    const int k = sb;
    x[1] = load_vtx(c, W, 0, r);
    if (k == 2) return 2;
    for (int j = 2; j <= k - 2; ++j) x[j] = load_vtx(c, W, slot_light(D, j - 1), r);
    x[k - 1] = load_vtx(c, W, slot_nee(D, k - 2), r);
    return k;
}

}  // namespace

// the per-element work of k_enum
template <int T>
__device__ __forceinline__ void enum_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t r, int it) {
    const WaveBuf &W = A.W;
    PathCounts &pc = st.pc;
    const int D = A.S.max_depth;
    const int g = A.frame;
    Vtx *x = st.x;
    unsigned int &roots = st.roots;
    do {
        ++roots;
        const uint32_t cam = W.cam_ok[r], nee = W.nee_ok[r];
        // enumerate the non-static base paths into mapping tasks
        if (T == T_1 || T == T_4) {
            if (!(W.flags[r] & RF_ROOT_OK)) continue;
            for (int t = 0; t <= W.len_eye[r]; ++t)
                if (cam & (1u << t)) dispatch_path(c, pc, x, 0, r, T, t, 0);
        } else if (T == T_5) {
            for (int j = 1; j <= W.len_light[r]; ++j)
                if (nee & (1u << j)) dispatch_path(c, pc, x, 0, r, T_5, 0, j + 2);
        } else if (T == T_6) {
            const int nz = W.len_eye[r], ny = W.len_light[r];
            for (int te = 1; te <= nz; ++te) {
                if (!(cam & (1u << te))) continue;
                for (int sl = 1; sl <= ny && te + sl <= D - 1; ++sl)
                    if (nee & (1u << sl)) dispatch_path(c, pc, x, 0, r, T_6, te, sl);
            }
        } else if (T == T_2) {
            if (!(W.flags[r] & RF_ROOT_OK)) continue;
            for (int s2 = 1; s2 <= W.len_light[r]; ++s2)
                if (nee & (1u << s2)) dispatch_path(c, pc, x, 0, r, T_2, 0, s2);
        } else if (T == T_3) {
            const int nz = W.len_eye[r], ny = W.len_light[r];
            for (int te = 1; te <= nz; ++te) {
                if (!(cam & (1u << te))) continue;
                for (int sl = 1; sl <= ny && te + sl <= D - 2; ++sl)
                    if (nee & (1u << sl)) dispatch_path(c, pc, x, 0, r, T_3, te, sl);
            }
        } else {
            const int len = W.len_light[r];
            if (len == 0) continue;
            const uint32_t gw = W.ghost_w[r], gn = W.ghost_n[r];
            unsigned dynmask = 0u;
            for (int j = 1; j <= len; ++j) {
                const int prim = W.prim[(size_t)(j == 1 ? 0 : slot_light(D, j - 1)) * W.R + r];
                if (prim >= A.S.n_static) dynmask |= 1u << j;
            }
            const Vtx x1 = load_vtx(c, W, 0, r);
            if (!zero3(get_mat(c, g, x1.mat).em) && ((dynmask & 2u) || (gw & 2u)))
                dispatch_path(c, pc, x, 0, r, T_7, 0, 2);
            for (int j = 1; j <= len; ++j) {
                if (!(nee & (1u << j))) continue;
                const unsigned upto = (2u << j) - 2u;
                if ((dynmask & upto) || (gw & upto) || (gn & (1u << j)))
                    dispatch_path(c, pc, x, 0, r, T_7, 0, j + 2);
            }
        }
    } while (0);
}


// the per-element work of k_eval_fast
template <int T>
__device__ __forceinline__ void eval_fast_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t r, int it) {
    const WaveBuf &W = A.W;
    PathCounts &pc = st.pc;
    unsigned int &roots = st.roots;
    const int D = A.S.max_depth;
    float *s_light = st.s_light;
    do {
        ++roots;
        const uint32_t root = A.root_begin + r;
        const uint32_t cam = W.cam_ok[r], nee = W.nee_ok[r];
        if (T == T_PT) {
            const int len = W.len_light[r];
            if (len == 0) continue;
            if (A.residual) {
                // without motion only paths through the edited object contribute
                bool any_dyn = false;
                for (int j = 1; j <= len && !any_dyn; ++j)
                    any_dyn = W.prim[(size_t)(j == 1 ? 0 : slot_light(D, j - 1)) * W.R + r] >= A.S.n_static;
                if (!any_dyn) continue;
            }
            fast_pt(c, pc, root, SlotLoader{c, W, r, D}, len, nee, A.residual ? T_7 : T_PT);
            continue;
        }
        if ((T == T_1 || T == T_2) && !(W.flags[r] & RF_ROOT_OK)) continue;
        const int nz = (T == T_2) ? 0 : W.len_eye[r];
        const int ny = (T == T_1) ? 0 : W.len_light[r];
        if (T == T_3 && (nz == 0 || ny == 0)) continue;
        if constexpr (T == T_3) {
            fast_t3(c, pc, root, SlotLoader{c, W, r, D}, nz, cam, ny, nee, s_light + threadIdx.x,
                    blockDim.x);
        } else if constexpr (T == T_1) {
            fast_t1(c, pc, root, SlotLoader{c, W, r, D}, nz, cam);
        } else {
            fast_t2(c, pc, root, SlotLoader{c, W, r, D}, ny, nee);
        }
    } while (0);
}


// --- stage C ---------------------------------------------------------------

namespace {

// reserve `k` consecutive entries of a queue with one atomic per coalesced
// group of threads; returns the first
__device__ __forceinline__ uint32_t append_n(unsigned int *counter, uint32_t k) {
    cg::coalesced_group g = cg::coalesced_threads();
    const uint32_t ex = cg::exclusive_scan(g, k);
    const uint32_t tot = g.shfl(ex + k, g.size() - 1);
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, tot);
    return g.shfl(base, 0) + ex;
}

// Stage C3, the base path's side: f(x), the balance denominator P_g(x) and
// the one-way value of base path x (n vertices); false when f(x) = 0 (the
// path adds nothing).
struct XSide {
    float3 fx, v1;
    int pa, ex;
    SF Pg;
    uint32_t searched, crossed;
};

__device__ bool finish_x(Ctx &c, PathCounts &pc, const Vtx *x, int n, XSide &xs) {
    const LaunchArgs &A = c.A;
    const int g = A.frame;
    xs.fx = path_throughput(c, g, x, n, xs.pa, xs.ex);
    if (zero3(xs.fx)) return false;
    ++pc.paths;
    const float sign = (g == 2) ? 1.0f : -1.0f;
    // the ghost terms of P_g(x) search x's edges against the objects at
    // their frame-g' pose: the same query as the dynamic-only visibility of
    // an edge the mapping leaves unchanged
    xs.searched = 0u;
    xs.crossed = 0u;
    xs.Pg = mis_denominator(c, g, x, n, &xs.searched, &xs.crossed);
    xs.v1 = xs.fx * ldexpf(sign * A.invN / xs.Pg.m, xs.ex - xs.Pg.e);     // one-way value
    return true;
}

// Stage C3, the mapped path's side, for base path x of task ti (its side in
// xs) mapped to y with `mi` (y is read only when the pair is accepted);
// `same` holds the edges the mapping leaves unchanged.  Both splats of the
// two-way estimator (Eq. shiftmapped; R3).  A rejected or invalid pair emits
// the one-way value now.  An accepted pair needs the mapped path's edges to
// be clear (replayed edges are clear by construction, unchanged edges are
// tested against the dynamic objects only): those rays are queued for
// k_trace_vis and the task waits for k_map_b; when the queue is full they
// are traced here.
__device__ void finish_y(Ctx &c, PathCounts &pc, const XSide &xs, const Vtx *y, int n, uint32_t same,
                         uint32_t ti, uint32_t root, int tech, int sa, int sb, MapInfo mi) {
    const LaunchArgs &A = c.A;
    const WaveBuf &W = A.W;
    const int g = A.frame, g2 = 3 - g;
    const float invN = A.invN;
    const float sign = (g == 2) ? 1.0f : -1.0f;
    const float3 fx = xs.fx, v1 = xs.v1;
    const int pa = xs.pa, ex = xs.ex;
    const SF Pg = xs.Pg;
    const uint32_t searched = xs.searched;
    int pb = -1, ey = 0;
    float3 fy = f3(0, 0, 0);
    SF Py{0.f, 0};
    // an unchanged edge that crosses the objects at their frame-g' pose
    // blocks the mapped path
    if (mi.status == MAP_ACCEPT && (same & xs.crossed)) mi.status = MAP_INVALID;
    if (mi.status == MAP_ACCEPT) {
        fy = path_throughput(c, g2, y, n, pb, ey);
        // an unchanged edge of y crosses nothing at the frame-g pose: it is
        // an edge of x, which is clear in frame g
        if (!zero3(fy)) Py = mis_denominator(c, g2, y, n, nullptr, nullptr, same);
        if (zero3(fy) || !(Py.m > 0.f)) mi.status = MAP_INVALID;
    }
    if (mi.status != MAP_ACCEPT) {
        if (mi.status != MAP_INVALID) ++pc.rejected;
        emit(c, root, tech, g, sa, sb, pa, v1, -1, f3(0, 0, 0), mi.status, sf_val(Pg), 0.f, 0.f);
        return;
    }
    const SF den = sf_add(Pg, SF{Py.m * mi.J, Py.e});
    const float3 va = fx * ldexpf(sign * invN / den.m, ex - den.e);
    const float3 vb = fy * ldexpf(-sign * mi.J * invN / den.m, ey - den.e);
    // the mapped path's edges that need a test: not the replayed ones (the
    // end farther from the dynamic vertex was found by tracing the edge)
    int last = -1;
    for (int j = 1; j <= n - 2; ++j)
        if (is_dyn(c, y[j])) last = j;
    uint32_t need = 0u, dyn_only = 0u;
    for (int j = 0; j + 1 < n; ++j) {
        const int far = (j + 1 <= last) ? j : j + 1;
        if (mi.replayed & (1u << far)) continue;
        if ((same >> j) & 1u) {
            if ((searched >> j) & 1u) continue;       // already known clear (above)
            dyn_only |= 1u << j;
        }
        need |= 1u << j;
    }
    const uint32_t ne = (uint32_t)__popc(need);
    uint32_t base = ne ? append_n(W.counts + cnt_vis(), ne) : 0u;
    if (ne && base + ne > W.qv) {
        // queue full: mark the reserved entries void and trace here
        for (uint32_t i = base; i < W.qv && i < base + ne; ++i) W.v_task[i] = ~0u;
        bool clear = true;
        for (int j = 0; j + 1 < n && clear; ++j)
            if (need & (1u << j)) clear = segment_clear(c, g2, y[j], y[j + 1], (dyn_only >> j) & 1u);
        if (!clear) {
            emit(c, root, tech, g, sa, sb, pa, v1, -1, f3(0, 0, 0), MAP_INVALID, sf_val(Pg), 0.f, 0.f);
            return;
        }
        ++pc.accepted;
        emit(c, root, tech, g, sa, sb, pa, va, pb, vb, MAP_ACCEPT, sf_val(Pg), sf_val(Py), mi.J);
        return;
    }
    if (!ne) {
        ++pc.accepted;
        emit(c, root, tech, g, sa, sb, pa, va, pb, vb, MAP_ACCEPT, sf_val(Pg), sf_val(Py), mi.J);
        return;
    }
    for (int j = 0; j + 1 < n; ++j) {
        if (!(need & (1u << j))) continue;
        const float3 e = y[j + 1].p - y[j].p;
        const float dist = len3(e);
        store3(W.v_o, W.qv, base, y[j].p);
        store3(W.v_d, W.qv, base, e * (1.0f / dist));
        W.v_tmax[base] = dist - A.S.eps;
        W.v_ex0[base] = y[j].prim;
        W.v_ex1[base] = y[j + 1].prim;
        W.v_task[base] = ti | (((dyn_only >> j) & 1u) << 31);
        ++base;
    }
    W.m_pix[ti] = pa;
    W.m_pix[W.qt + ti] = pb;
    store3(W.m_val, W.qt, ti, va);
    store3(W.m_val + 3 * (size_t)W.qt, W.qt, ti, vb);
    store3(W.m_val + 6 * (size_t)W.qt, W.qt, ti, v1);
    if (A.rec) {
        W.m_w[ti] = sf_val(Pg);
        W.m_w[W.qt + ti] = sf_val(Py);
        W.m_w[2 * W.qt + ti] = mi.J;
    }
    W.m_vis[ti] = 1u;
    const uint32_t p = append(W.counts + cnt_pend());
    W.pend[p] = ti;                   // p < qt: one entry per task at most
}

// stage C3 for base path x and its mapped path y held in separate arrays
__device__ void finish_task(Ctx &c, PathCounts &pc, const Vtx *x, int n, uint32_t ti, uint32_t root,
                            int tech, int sa, int sb, const Vtx *y, MapInfo mi) {
    XSide xs;
    if (!finish_x(c, pc, x, n, xs)) return;
    uint32_t same = 0u;              // edges the mapping leaves unchanged
    if (mi.status == MAP_ACCEPT)
        for (int j = 0; j + 1 < n; ++j)
            if (same3(x[j].p, y[j].p) && same3(x[j + 1].p, y[j + 1].p)) same |= 1u << j;
    finish_y(c, pc, xs, y, n, same, ti, root, tech, sa, sb, mi);
}

// the whole of stages C1-C3 for one task in one thread (tasks that find the
// replayed-vertex pool full)
__device__ __noinline__ void map_task_inline(Ctx &c, PathCounts &pc, const Vtx *x, int n, uint32_t ti,
                                uint32_t root, int tech, int sa, int sb) {
    Vtx y[kMaxVerts];
    MapInfo mi;
    mi.J = 1.0f;
    mi.replayed = 0u;
    if (c.A.map_mode == 0) {
        mi.status = MAP_OFF;
        for (int j = 0; j < n; ++j) y[j] = x[j];
    } else {
        map_path(c, c.A.frame, 3 - c.A.frame, x, n, y, mi);
    }
    finish_task(c, pc, x, n, ti, root, tech, sa, sb, y, mi);
}

// --- the wavefront mapping (stages C1, C2) ---------------------------------
//
// Path mapping (Sec. 5) walks the base path vertex by vertex: the object
// transform or the camera replay, then per walk vertex "unchanged", "keep
// the vertex" (reconnection) or random replay, which traces a ray in the
// other frame.  Each task's mapping runs as a small program of steps; a
// replay step queues its ray and suspends the task, k_trace_map traces the
// queue, and k_map_step resumes the tasks with their hits.  The replayed
// vertices go to a pool (slots base + j); the state word holds the rest.

// state word: status (bits 0-3; kRunning while steps remain, kInline when the
// task was mapped and evaluated in one thread), camera mode (bit 4), the
// dynamic vertex's index (bits 5-8), the next step (bits 9-12), replayed
// vertices (bit 16 + j)
constexpr uint32_t kRunning = 7u, kInline = 8u;
__device__ __forceinline__ uint32_t ms_status(uint32_t w) { return w & 15u; }
__device__ __forceinline__ bool ms_camera(uint32_t w) { return (w >> 4) & 1u; }
__device__ __forceinline__ int ms_dyn(uint32_t w) { return (int)((w >> 5) & 15u); }
__device__ __forceinline__ int ms_step(uint32_t w) { return (int)((w >> 9) & 15u); }
__device__ __forceinline__ uint32_t ms_replayed(uint32_t w) { return (w >> 16) & 0xfffu; }
__device__ __forceinline__ uint32_t ms_with_status(uint32_t w, uint32_t st) { return (w & ~15u) | st; }
__device__ __forceinline__ uint32_t ms_with_step(uint32_t w, int s) {
    return (w & ~(15u << 9)) | ((uint32_t)s << 9);
}

// a task's mapping has ended with state w: record it and list the task for
// stage C3, accepted pairs from the front of W.fin, the others from the back
// (so that the lanes of a warp of k_map_fin take the same branch)
__device__ __forceinline__ void map_done(const WaveBuf &W, uint32_t ti, uint32_t w, float J) {
    W.ms_info[ti] = w;
    W.ms_J[ti] = J;
    if (ms_status(w) == MAP_ACCEPT) W.fin[append(W.counts + cnt_fin_acc())] = ti;
    else W.fin[W.qt - 1u - append(W.counts + cnt_fin_rej())] = ti;
}

// a base path by reference: root, its technique's slot layout and counts
struct PathRef {
    uint32_t r;
    int lay, sa, sb, k;
};

// the slot of vertex j of path (lay, sa, sb) (the layout of assemble());
// -1 for the pinhole
__device__ __forceinline__ int path_slot(int lay, int sa, int sb, int D, int j) {
    if (j == 0) return -1;
    if (lay == T_6) {
        const int te = sa, sl = sb;
        if (j <= te) return slot_eye(D, te - j + 1);
        if (j <= te + sl) return slot_light(D, j - te);
        return slot_nee(D, sl);
    }
    if (lay == T_1 || lay == T_4) {
        const int t = sa;
        if (j <= t) return slot_eye(D, t - j + 1);
        return j == t + 1 ? 0 : 1;
    }
    if (lay == T_2) {
        const int s2 = sb;
        if (j == 1) return 0;
        if (j <= s2 + 1) return slot_light(D, j - 1);
        return slot_nee(D, s2);
    }
    if (lay == T_3) {
        const int te = sa, sl = sb;
        if (j <= te) return slot_eye(D, te - j + 1);
        if (j == te + 1) return 0;
        if (j <= te + sl + 1) return slot_light(D, j - te - 1);
        return slot_nee(D, sl);
    }
    const int k = sb;                 // path tracing
    if (j == 1) return 0;
    if (j <= k - 2) return slot_light(D, j - 1);
    return slot_nee(D, k - 2);
}

__device__ __forceinline__ int path_len(int lay, int sa, int sb) {
    if (lay == T_6) return sa + sb + 2;
    if (lay == T_1 || lay == T_4) return sa + 3;
    if (lay == T_2) return sb + 3;
    if (lay == T_3) return sa + sb + 3;
    return sb;
}

__device__ __forceinline__ PathRef task_path(const LaunchArgs &A, uint32_t ti) {
    const int4 t = A.W.tasks[ti];
    PathRef P;
    P.r = (uint32_t)t.x;
    P.lay = (t.y == T_7 || t.y == T_5) ? T_PT : t.y;
    P.sa = t.z;
    P.sb = t.w;
    P.k = path_len(P.lay, P.sa, P.sb);
    return P;
}

// vertex j of the base path
__device__ __forceinline__ Vtx xv(const Ctx &c, const PathRef &P, int j) {
    const int sl = path_slot(P.lay, P.sa, P.sb, c.A.S.max_depth, j);
    return sl < 0 ? camera_vertex(c) : load_vtx(c, c.A.W, sl, P.r);
}

// the triangle of vertex j of the base path (-1: the pinhole)
__device__ __forceinline__ int xprim(const Ctx &c, const PathRef &P, int j) {
    const int sl = path_slot(P.lay, P.sa, P.sb, c.A.S.max_depth, j);
    return sl < 0 ? -1 : c.A.W.prim[(size_t)sl * c.A.W.R + P.r];
}

__device__ __forceinline__ void pool_store(const WaveBuf &W, uint32_t i, const Vtx &v) {
    store3(W.y_p, W.yc, i, v.p);
    store3(W.y_n, W.yc, i, v.n);
    W.y_b[i] = v.b1;
    W.y_b[W.yc + i] = v.b2;
    W.y_prim[i] = v.prim;
}

__device__ __forceinline__ Vtx pool_load(const Ctx &c, const WaveBuf &W, uint32_t i) {
    Vtx v;
    v.p = load3(W.y_p, W.yc, i);
    v.n = load3(W.y_n, W.yc, i);
    v.b1 = W.y_b[i];
    v.b2 = W.y_b[W.yc + i];
    v.prim = W.y_prim[i];
    v.mat = v.prim < c.A.S.n_static ? (int)c.A.S.stat_mat[v.prim] : kMatDynamic - inst_of(c.A.S, v.prim);
    return v;
}

// vertex j of the mapped path so far: a replayed vertex from the pool, the
// transformed dynamic vertex, else the base path's vertex
__device__ __forceinline__ Vtx yv(const Ctx &c, const PathRef &P, uint32_t w, uint32_t base, int j) {
    if ((ms_replayed(w) >> j) & 1u) return pool_load(c, c.A.W, base + (uint32_t)j);
    const Vtx x = xv(c, P, j);
    if (!ms_camera(w) && j == ms_dyn(w)) return make_vertex(c, 3 - c.A.frame, x.prim, x.b1, x.b2);
    return x;
}

// step s of the mapping program: vertex b from its predecessor a, sampled
// with conditioning vertex cc (-1: cosine step); the order of map_path and
// map_camera.  False past the last step.
__device__ __forceinline__ bool map_program(bool camera, int i, int k, int s, int &a, int &b, int &cc) {
    if (camera) {                                   // step 0 is the camera ray
        b = s + 1;
        a = b - 1;
        cc = b - 2;
        return b <= k - 2;
    }
    if (i == k - 2) {                               // (1): eye side from x_D
        b = i - 1 - s;
        a = b + 1;
        cc = (b == i - 1) ? k - 1 : b + 2;
        return b >= 1;
    }
    if (i == 1) {                                   // (2): light side
        b = 2 + s;
        a = b - 1;
        cc = b - 2;
        return b <= k - 2;
    }
    const int nl = k - 2 - i;                       // (3): light side, then eye side
    if (s < nl) {
        b = i + 1 + s;
        a = b - 1;
        cc = (b == i + 1) ? -1 : b - 2;
        return true;
    }
    b = i - 1 - (s - nl);
    a = b + 1;
    cc = b + 2;
    return b >= 1;
}

// the first edge of (v0, v1) in frame g is dynamic (first_edge_dynamic)
__device__ __forceinline__ bool first_edge_dyn2(Ctx &c, int g, const Vtx &v0, const Vtx &v1) {
    if (is_dyn(c, v1)) return true;
    return !segment_clear(c, 3 - g, v0, v1, true);
}

// the acceptance tests at the end of a mapping program (map_path, map_camera)
__device__ uint32_t map_finish(Ctx &c, const PathRef &P, uint32_t w, uint32_t base, float J) {
    const int g2 = 3 - c.A.frame;
    const float jm = c.A.S.jac_max;
    const bool jac_ok = J <= jm && 1.0f / J <= jm;
    if (ms_camera(w)) {
        if (!first_edge_dyn2(c, g2, camera_vertex(c), yv(c, P, w, base, 1))) return MAP_REJECT_INVERT;
        return jac_ok ? MAP_ACCEPT : MAP_REJECT_JAC;
    }
    if (!jac_ok) return MAP_REJECT_JAC;
    if (c.A.map_mode == 2 && first_edge_dyn2(c, g2, camera_vertex(c), yv(c, P, w, base, 1)))
        return MAP_REJECT_INVERT;
    return MAP_ACCEPT;
}

// push a replay ray of task ti into queue `round`; false when it is full
__device__ __forceinline__ bool push_replay(const LaunchArgs &A, int round, float3 o, float3 d, int ex,
                                            uint32_t ti) {
    const WaveBuf &W = A.W;
    const uint32_t i = append(W.counts + cnt_replay(round));
    if (i >= W.qr) return false;
    const int b = round & 1;
    store3(W.r_o[b], W.qr, i, o);
    store3(W.r_d[b], W.qr, i, d);
    W.r_ex[b][i] = ex;
    W.r_task[b][i] = ti;
    return true;
}

// The direction of the random-seed replay of step (a, b, cc) of task P in
// state w (Sec. 5): the step's sampling routine inverted at x_a for the
// direction to x_b, then run at y_a with the numbers found (double
// precision); false when that direction is invalid.
__device__ bool replay_direction(Ctx &c, const PathRef &P, uint32_t w, uint32_t base, int a, int b,
                                 int cc, float3 &w2) {
    const LaunchArgs &A = c.A;
    const int g = A.frame, g2 = 3 - g;
    const Vtx xa = xv(c, P, a), ya = yv(c, P, w, base, a), xb = xv(c, P, b);
    const float3 wo = unit3(xb.p - xa.p);
    double u1, u2;
    if (cc < 0) {
        cosine_inverse(xa.n, wo, u1, u2);
        w2 = cosine_dir(A.S, ya.n, u1, u2);
        return dot3(ya.n, w2) > 0.f;
    }
    const Vtx xc = xv(c, P, cc), yc = yv(c, P, w, base, cc);
    bsdf_inverse(get_mat(c, g, xa.mat), xa.n, unit3(xc.p - xa.p), wo, u1, u2);
    return bsdf_sample(A.S, get_mat(c, g2, ya.mat), ya.n, unit3(yc.p - ya.p), u1, u2, w2);
}

// the tests and Jacobian factor of replayed vertex nb = y[b] (map_step after
// its trace); stores nb in the pool.  Returns MAP_ACCEPT to go on.
__device__ uint32_t replay_hit(Ctx &c, const PathRef &P, uint32_t &w, uint32_t base, float &J, int a,
                               int b, int cc, float3 w2, bool hit, const Vtx &nb) {
    const int g = c.A.frame, g2 = 3 - g;
    if (!hit) return MAP_INVALID;
    if (a == 0 && ms_camera(w)) {                   // the camera ray of the camera replay
        if (dot3(nb.n, w2) >= 0.f) return MAP_INVALID;
        const float px = pdf_camera_area(c.A.S, xv(c, P, 1)), py = pdf_camera_area(c.A.S, nb);
        if (!(px > 0.f) || !(py > 0.f)) return MAP_INVALID;
        pool_store(c.A.W, base + 1, nb);
        w |= 2u << 16;
        J *= px / py;
        return MAP_ACCEPT;
    }
    if (dot3(nb.n, w2) >= 0.f) return MAP_INVALID;
    if (is_dyn(c, nb)) return MAP_REJECT_MULTI;
    const Vtx xa = xv(c, P, a), ya = yv(c, P, w, base, a);
    if (reconnect_ok(c, g2, ya, g, xa, g2, nb)) return MAP_REJECT_INVERT;
    const Vtx xb = xv(c, P, b);
    float px, py;
    if (cc < 0) {
        const float3 wo = unit3(xb.p - xa.p);
        px = area_from_dir(cosine_pdf(xa.n, wo), xa.p, xb);
        py = area_from_dir(cosine_pdf(ya.n, w2), ya.p, nb);
    } else {
        const Vtx xc = xv(c, P, cc), yc = yv(c, P, w, base, cc);
        {
            const float3 wc = unit3(xc.p - xa.p), wo = unit3(xb.p - xa.p);
            px = area_from_dir(bsdf_pdf(get_mat(c, g, xa.mat), xa.n, wc, wo), xa.p, xb);
        }
        {
            const float3 wc = unit3(yc.p - ya.p), wo = unit3(nb.p - ya.p);
            py = area_from_dir(bsdf_pdf(get_mat(c, g2, ya.mat), ya.n, wc, wo), ya.p, nb);
        }
    }
    pool_store(c.A.W, base + (uint32_t)b, nb);
    w |= 1u << (16 + b);
    if (!(px > 0.f) || !(py > 0.f)) return MAP_INVALID;
    J *= px / py;
    return MAP_ACCEPT;
}

// run task ti's mapping program from its current step until a replay ray is
// queued into `round` (the task is suspended) or the program ends; writes the
// state back
__device__ void map_run(Ctx &c, const PathRef &P, uint32_t ti, uint32_t w, uint32_t base, float J,
                        int round) {
    const LaunchArgs &A = c.A;
    const WaveBuf &W = A.W;
    const int g = A.frame, g2 = 3 - g;
    uint32_t st = MAP_ACCEPT;
    for (;;) {
        const int s = ms_step(w);
        int a, b, cc;
        if (!map_program(ms_camera(w), ms_dyn(w), P.k, s, a, b, cc)) {
            st = map_finish(c, P, w, base, J);
            break;
        }
        const Vtx xa = xv(c, P, a), ya = yv(c, P, w, base, a);
        w = ms_with_step(w, s + 1);
        if (same3(ya.p, xa.p)) continue;            // predecessor unchanged: y_b = x_b
        const Vtx xb = xv(c, P, b);
        if (reconnect_ok(c, g, xa, g2, ya, g, xb)) continue;    // keep the vertex
        // random-seed replay: queued with its direction still to be found
        // (k_replay_dir computes the directions of a whole round's queue at
        // once, so that the double-precision inversion runs with every lane
        // of a warp busy); a replay queued into `round` is traced only if
        // that round runs (rounds 0 .. max_depth - 2, see map_stage)
        const float nan = __int_as_float(0x7fc00000);
        if (round < A.S.max_depth - 1 && round < kMaxIter &&
            push_replay(A, round, ya.p, f3(nan, nan, nan), ya.prim, ti)) {
            W.ms_info[ti] = ms_with_step(ms_with_status(w, kRunning), s);
            W.ms_J[ti] = J;
            return;
        }
        // queue full: the direction and the trace here
        float3 w2;
        if (!replay_direction(c, P, w, base, a, b, cc, w2)) {
            st = MAP_INVALID;
            break;
        }
        Vtx nb{};
        const bool hit = trace_next(c, g2, ya, w2, nb);
        st = replay_hit(c, P, w, base, J, a, b, cc, w2, hit, nb);
        if (st != MAP_ACCEPT) break;
    }
    map_done(W, ti, ms_with_status(w, st), J);
}

}  // namespace

// the per-element work of k_map_start
__device__ __forceinline__ void map_start_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t ti, int it) {
    PathCounts &pc = st.pc;
    const WaveBuf &W = A.W;
    const int g = A.frame;
    do {
        const PathRef P = task_path(A, ti);
        if (A.map_mode == 0) {
            map_done(W, ti, MAP_OFF, 1.0f);
            continue;
        }
        const uint32_t base = append_n(W.counts + cnt_pool(), (uint32_t)P.k);
        if (base + (uint32_t)P.k > W.yc) {
            // no pool slots left: the whole task in this thread
            Vtx x[kMaxVerts];
            const int4 t = W.tasks[ti];
            assemble(c, P.r, P.lay, P.sa, P.sb, x);
            map_task_inline(c, pc, x, P.k, ti, A.root_begin + P.r, t.y, t.z, t.w);
            W.ms_info[ti] = kInline;
            continue;
        }
        W.ms_base[ti] = base;
        const Vtx x1 = xv(c, P, 1);
        if (A.map_mode == 2 && first_edge_dyn2(c, g, camera_vertex(c), x1)) {
            // camera replay: the walk vertices must be static
            uint32_t st = kRunning;
            for (int j = 2; j <= P.k - 2 && st == kRunning; ++j)
                if (xprim(c, P, j) >= A.S.n_static) st = MAP_REJECT_MULTI;
            const uint32_t w = (1u << 4) | (1u << 9);
            if (st == kRunning) {
                const float3 d = unit3(x1.p - A.S.cam_pos);
                if (push_replay(A, 0, A.S.cam_pos, d, -1, ti)) {
                    W.ms_info[ti] = (w & ~(15u << 9)) | kRunning;      // step 0 pending
                    W.ms_J[ti] = 1.0f;
                    continue;
                }
                Vtx nb{};
                const bool hit = trace_next(c, 3 - g, camera_vertex(c), d, nb);
                uint32_t ww = w;
                float J = 1.0f;
                st = replay_hit(c, P, ww, base, J, 0, 1, -1, d, hit, nb);
                if (st == MAP_ACCEPT) {
                    map_run(c, P, ti, ww, base, J, 0);
                    continue;
                }
            }
            map_done(W, ti, ms_with_status(w, st), 1.0f);
            continue;
        }
        int nd = 0, i = -1;
        for (int j = 1; j <= P.k - 2; ++j)
            if (xprim(c, P, j) >= A.S.n_static) {
                ++nd;
                i = j;
            }
        if (nd != 1) {
            map_done(W, ti, nd == 0 ? MAP_REJECT_NODYN : MAP_REJECT_MULTI, 1.0f);
            continue;
        }
        map_run(c, P, ti, (uint32_t)i << 5, base, 1.0f, 0);
    } while (0);
}


// the per-element work of k_replay_dir: the direction of replay ray i of
// round `it` whose direction is still to be found (a NaN there; the camera
// rays of the camera replay carry theirs).  An invalid direction stays NaN:
// its trace finds no hit, and k_map_step ends the task as MAP_INVALID, as
// the replay's own step would have.
__device__ __forceinline__ void replay_dir_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int bq = it & 1;
    do {
        if (!isnan(W.r_d[bq][i])) continue;
        const uint32_t ti = W.r_task[bq][i];
        const PathRef P = task_path(A, ti);
        const uint32_t w = W.ms_info[ti];
        int a, b, cc;
        map_program(ms_camera(w), ms_dyn(w), P.k, ms_step(w), a, b, cc);
        float3 w2;
        if (replay_direction(c, P, w, W.ms_base[ti], a, b, cc, w2)) store3(W.r_d[bq], W.qr, i, w2);
    } while (0);
}


// the per-element work of k_trace_map
__device__ __forceinline__ void trace_map_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int b = it & 1;
    const int g2 = 3 - A.frame;
    const float inf = __int_as_float(0x7f800000);
    do {
        Hit h;
        ++c.cnt.rays_closest;
        if (scene_trace(c, g2, load3(W.r_o[b], W.qr, i), load3(W.r_d[b], W.qr, i), A.S.eps, inf,
                        W.r_ex[b][i], -1, false, false, h)) {
            W.rh_prim[i] = h.prim;
            W.rh_b1[i] = h.b1;
            W.rh_b2[i] = h.b2;
            store3(W.rh_p, W.qr, i, h.p);
        } else {
            W.rh_prim[i] = -1;
        }
    } while (0);
}


// the per-element work of k_map_step
__device__ __forceinline__ void map_step_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int round = it;
    const int bq = round & 1;
    const int g2 = 3 - A.frame;
    do {
        const uint32_t ti = W.r_task[bq][i];
        const PathRef P = task_path(A, ti);
        uint32_t w = W.ms_info[ti];
        const uint32_t base = W.ms_base[ti];
        float J = W.ms_J[ti];
        const int s = ms_step(w);
        int a, b, cc;
        if (ms_camera(w) && s == 0) {
            a = 0;
            b = 1;
            cc = -1;
        } else {
            map_program(ms_camera(w), ms_dyn(w), P.k, s, a, b, cc);
        }
        const int prim = W.rh_prim[i];
        Vtx nb{};
        if (prim >= 0)
            nb = make_vertex_at(c, g2, prim, W.rh_b1[i], W.rh_b2[i], load3(W.rh_p, W.qr, i));
        const uint32_t st = replay_hit(c, P, w, base, J, a, b, cc, load3(W.r_d[bq], W.qr, i),
                                       prim >= 0, nb);
        w = ms_with_step(w, s + 1);
        if (st != MAP_ACCEPT) {
            map_done(W, ti, ms_with_status(w, st), J);
            continue;
        }
        map_run(c, P, ti, w, base, J, round + 1);
    } while (0);
}


// the per-element work of k_map_fin
__device__ __forceinline__ void map_fin_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t j, int it) {
    PathCounts &pc = st.pc;
    const WaveBuf &W = A.W;
    const uint32_t n_acc = min(W.counts[cnt_fin_acc()], W.qt);
    const int g2 = 3 - A.frame;
    Vtx *x = st.x;
    const uint32_t ti = W.fin[j < n_acc ? j : W.qt - 1u - (j - n_acc)];
    const uint32_t w = W.ms_info[ti];
    const int4 t = W.tasks[ti];
    const PathRef P = task_path(A, ti);
    const int k = assemble(c, P.r, P.lay, P.sa, P.sb, x);
    MapInfo mi;
    mi.status = (int)ms_status(w);
    mi.J = W.ms_J[ti];
    mi.replayed = 0u;
    XSide xs;
    if (!finish_x(c, pc, x, k, xs)) return;
    uint32_t same = 0u;
    if (mi.status == MAP_ACCEPT) {
        // the mapped path overwrites the base path in the one array: its
        // replayed vertices from the pool, the transformed dynamic vertex,
        // the others unchanged; `vs` marks the unchanged vertices
        const uint32_t base = W.ms_base[ti];
        const uint32_t rep = ms_replayed(w);
        mi.replayed = rep;
        uint32_t vs = 0u;
        for (int q = 0; q < k; ++q) {
            if ((rep >> q) & 1u) {
                const Vtx yq = pool_load(c, W, base + (uint32_t)q);
                if (same3(x[q].p, yq.p)) vs |= 1u << q;
                x[q] = yq;
            } else if (!ms_camera(w) && q == ms_dyn(w)) {
                const Vtx yq = make_vertex(c, g2, x[q].prim, x[q].b1, x[q].b2);
                if (same3(x[q].p, yq.p)) vs |= 1u << q;
                x[q] = yq;
            } else {
                vs |= 1u << q;
            }
        }
        same = vs & (vs >> 1) & ((1u << (k - 1)) - 1u);
    }
    finish_y(c, pc, xs, x, k, same, ti, A.root_begin + P.r, t.y, t.z, t.w, mi);
}


// the per-element work of k_trace_vis
__device__ __forceinline__ void trace_vis_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    const int g2 = 3 - A.frame;
    do {
        const uint32_t tv = W.v_task[i];
        if (tv == ~0u) continue;
        const uint32_t ti = tv & 0x7fffffffu;
        if (!W.m_vis[ti]) continue;               // another edge already blocked
        Hit h;
        ++c.cnt.rays_shadow;
        if (scene_trace(c, g2, load3(W.v_o, W.qv, i), load3(W.v_d, W.qv, i), A.S.eps, W.v_tmax[i],
                        W.v_ex0[i], W.v_ex1[i], true, (tv >> 31) != 0u, h))
            W.m_vis[ti] = 0u;
    } while (0);
}


// the per-element work of k_map_b
__device__ __forceinline__ void map_b_body(const LaunchArgs &A, Ctx &c, BodyState &st, uint32_t i, int it) {
    const WaveBuf &W = A.W;
    unsigned int &accepted = st.accepted;
    do {
        const uint32_t ti = W.pend[i];
        const int4 t = W.tasks[ti];
        const uint32_t root = A.root_begin + (uint32_t)t.x;
        const float Pg = A.rec ? W.m_w[ti] : 0.f;
        if (W.m_vis[ti]) {
            ++accepted;
            emit(c, root, t.y, A.frame, t.z, t.w, W.m_pix[ti], load3(W.m_val, W.qt, ti),
                 W.m_pix[W.qt + ti], load3(W.m_val + 3 * (size_t)W.qt, W.qt, ti), MAP_ACCEPT, Pg,
                 A.rec ? W.m_w[W.qt + ti] : 0.f, A.rec ? W.m_w[2 * W.qt + ti] : 0.f);
        } else {
            emit(c, root, t.y, A.frame, t.z, t.w, W.m_pix[ti], load3(W.m_val + 6 * (size_t)W.qt, W.qt, ti),
                 -1, f3(0, 0, 0), MAP_INVALID, Pg, 0.f, 0.f);
        }
    } while (0);
}


}  // namespace rp
