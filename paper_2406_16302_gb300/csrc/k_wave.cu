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
// Stage C (motion):  k_map_a, one thread per mapping task: object
//   transform, camera replay, reconnection or random replay in the other
//   frame, two-way MIS; the mapped path's edges that need a visibility test
//   go to a queue traced by k_trace_vis, and k_map_b emits the pairs.
//
// The random numbers, walk termination rules and path enumeration are those
// of the one-thread-per-root kernels (rp_device.cuh), so both modes produce
// the same samples.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "chain_fast.cuh"
#include "guide_device.cuh"
#include "rp_device.cuh"

namespace cg = cooperative_groups;

namespace rp {

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

template <int T>
__global__ void __launch_bounds__(256) k_gen(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    const WaveBuf &W = A.W;
    Ctx c(A, nullptr);
    const int g = A.frame, D = A.S.max_depth;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
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
    }
}

namespace {
// one row of input features, built locally and written as five 16-byte
// vectors (a row is 80 bytes, rows are 16-byte aligned)
__device__ __forceinline__ void store_features(int8_t *dst, const float *box, double3 p, float3 n) {
    alignas(16) int8_t m[kGIn];
    guide_encode_d(box, p, n, m);
    const int4 *src = reinterpret_cast<const int4 *>(m);
    int4 *d = reinterpret_cast<int4 *>(dst);
#pragma unroll
    for (int k = 0; k < kGIn / 16; ++k) d[k] = src[k];
}

}  // namespace

// technique (3) with the learned proposal: the network's integer input
// features of x_D (object space, recomputed from the root's numbers)
__global__ void __launch_bounds__(128) k_encode3(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    const int g = A.frame;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        if (!(A.W.flags[r] & RF_GUIDE)) continue;
        const uint32_t root = A.root_begin + r;
        const float4 ur = draw(lseed(A), root, T_3, g, SD_ROOT, 0);
        // x_D's triangle, as k_gen picked it (slot 0); its barycentrics in
        // double again from the root's numbers
        const int q = A.W.prim[r] - A.S.n_static;
        double b1, b2;
        tri_sample(ur.y, ur.z, b1, b2);
        const float4 *tq = A.S.inst[0].tri + 3 * q;
        const float4 ta = tq[0], tb = tq[1], tcv = tq[2];
        const double3 v0 = d3(ta);
        const double3 po = dadd(dadd(v0, dscale(dsub(d3(tb), v0), b1)), dscale(dsub(d3(tcv), v0), b2));
        store_features(A.G.gin + (size_t)r * kGIn, A.G.net.box, po, f3(ta.w, tb.w, tcv.w));
    }
}

namespace {
struct EncodeArgs {
    float box[6];
    const double *p;
    const float *nrm;
    uint32_t n;
    int8_t *out;
};
}  // namespace

// the learned proposal's input features of given points (rp_guide_encode)
__global__ void __launch_bounds__(128) k_guide_encode(const __grid_constant__ EncodeArgs E) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < E.n; i += gridDim.x * blockDim.x)
        store_features(E.out + (size_t)i * kGIn, E.box, d3(E.p[3 * i], E.p[3 * i + 1], E.p[3 * i + 2]),
                       f3(E.nrm[3 * i], E.nrm[3 * i + 1], E.nrm[3 * i + 2]));
}

cudaError_t launch_guide_encode(const float *box, const double *p, const float *nrm, uint32_t n,
                                int8_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    EncodeArgs E;
    for (int k = 0; k < 6; ++k) E.box[k] = box[k];
    E.p = p;
    E.nrm = nrm;
    E.n = n;
    E.out = out;
    const uint32_t g = (n + 127) / 128;
    k_guide_encode<<<g < 4096u ? g : 4096u, 128, 0, s>>>(E);
    return cudaGetLastError();
}

// technique (3) with the learned proposal: draw the first light-side
// direction from q = p_cos / 2 + (vMF mixture of the network's outputs) / 2
// with the step's numbers (u.z < 1/2 picks the cosine part, else 2 u.z - 1
// picks a lobe), record p_cos / q for the root's values
__global__ void __launch_bounds__(256) k_start3g(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    const WaveBuf &W = A.W;
    Ctx c(A, nullptr);
    const int g = A.frame;
    const float *M = A.E.M(0, g);
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        if (!(W.flags[r] & RF_GUIDE)) continue;
        const uint32_t root = A.root_begin + r;
        const Vtx xD = load_vtx(c, W, 0, r);
        const float4 u = draw(lseed(A), root, T_3, g, SD_LIGHT, 1);
        MixF mix;
        guide_mixture_f(A.G.gout + (size_t)r * kGOut, mix);
        const double3 nw = d3(xD.n);
        double3 w, wl;
        if (u.z < 0.5f) {
            w = cosine_dir_d(A.S, nw, u.x, u.y);
            wl = dlinear_T(M, w);
        } else {
            const float v = 2.f * u.z - 1.f;       // exact: u is on the 2^-24 grid
            float acc = 0.f;
            int j = kGLobes - 1;
            for (int i = 0; i < kGLobes; ++i) {
                acc += mix.pi[i];
                if (v < acc) { j = i; break; }
            }
            wl = vmf_sample_d(A.S, mix.mu[j], (double)mix.kappa[j], u.x, u.y);
            w = dlinear(M, wl);
        }
        const double cw = ddot(nw, w);
        const float pc = cw > 0.0 ? (float)(cw / kPiD) : 0.f;
        const float pv = mix_pdf_f(mix, wl);
        A.G.gratio[r] = pc / (0.5f * pc + 0.5f * pv);
        const uint32_t slot = guide_slot(A.G, g, root);
        if (slot != ~0u) {
            const uint32_t C = A.G.smp.cap;
            A.G.smp.w[slot] = (float)wl.x; A.G.smp.w[C + slot] = (float)wl.y;
            A.G.smp.w[2 * C + slot] = (float)wl.z;
        }
        const float3 wf = tof(w);
        if (dot3(xD.n, wf) > 0.f) push_closest(A, 0, 0, xD.p, wf, xD.prim, make_tag(r, SIDE_LIGHT, 1));
    }
}

// techniques (1) and (2): start the walk of roots whose root connection is visible
template <int T>
__global__ void __launch_bounds__(256) k_start(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    const WaveBuf &W = A.W;
    Ctx c(A, nullptr);
    const int g = A.frame, D = A.S.max_depth;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
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
    }
}

// consume the hits of iteration it-1's closest rays; emit iteration it's rays
template <int T>
__global__ void __launch_bounds__(256) k_extend(const __grid_constant__ LaunchArgs A, int it) {
    const WaveBuf &W = A.W;
    const int in = (it - 1) & 1, out = it & 1;
    const uint32_t n = min(W.counts[cnt_closest(it - 1)], W.qc);
    Ctx c(A, nullptr);
    const int g = A.frame, D = A.S.max_depth;
    const int tech = (T == T_PT) ? (A.residual ? T_7 : T_PT) : T;
    const int rg = (T == T_PT && !A.residual) ? 0 : g;
    const bool ghosts = (T == T_PT) && A.residual && A.E.motion;
    constexpr bool camera_walk = (T == T_PT || T == T_5);      // x_1 from the camera, NEE at every vertex
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    }
}

// closest hits of a queue
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_closest(const __grid_constant__ LaunchArgs A, int it) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const WaveBuf &W = A.W;
    const int b = it & 1;
    const uint32_t n = min(W.counts[cnt_closest(it)], W.qc);
    const float inf = __int_as_float(0x7f800000);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    }
    if (A.stats) {
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_NODES_C, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS_C, c.cnt.tris);
    }
}

// shadow rays: visibility of connections, or ghost crossings of edges
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_shadow(const __grid_constant__ LaunchArgs A, int it) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const WaveBuf &W = A.W;
    const uint32_t n = min(W.counts[cnt_shadow(it)], W.qa);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    }
    if (A.stats) {
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_NODES_S, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS_S, c.cnt.tris);
    }
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

// motion: every non-static base path of a root becomes a mapping task
template <int T>
__global__ void __launch_bounds__(128) k_enum(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    const WaveBuf &W = A.W;
    Ctx c(A, nullptr);
    PathCounts pc{0, 0, 0};
    const int D = A.S.max_depth;
    const int g = A.frame;
    Vtx x[1];
    unsigned int roots = 0;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
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
    }
    if (A.stats) add_stat(A.stats, ST_ROOTS, roots);
}

// edits without motion, and the primal: every base path of a root from
// running products along its walks (chain_fast.cuh), O(1) work per path
template <int T>
// (register budgets: technique (3)'s nested walks at 4 blocks per SM, the
// others at 5)
__global__ void __launch_bounds__(128, T == T_3 ? 4 : 5) k_eval_fast(const __grid_constant__ LaunchArgs A) {
    // technique (3): each thread's light-side values per s (fast_t3)
    __shared__ float s_light[T == T_3 ? kT3LightSlots * 10 * 128 : 1];
    const uint32_t n = A.root_end - A.root_begin;
    const WaveBuf &W = A.W;
    Ctx c(A, nullptr);
    PathCounts pc{0, 0, 0};
    unsigned int roots = 0;
    const int D = A.S.max_depth;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
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
    }
    if (A.stats) {
        add_stat(A.stats, ST_ROOTS, roots);
        add_stat(A.stats, ST_PATHS, pc.paths);
        add_stat(A.stats, ST_ACCEPTED, pc.accepted);
    }
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

__device__ __forceinline__ void store3(float *a, uint32_t stride, uint32_t i, float3 v) {
    a[i] = v.x;
    a[stride + i] = v.y;
    a[2 * stride + i] = v.z;
}

__device__ __forceinline__ float3 load3(const float *a, uint32_t stride, uint32_t i) {
    return f3(a[i], a[stride + i], a[2 * stride + i]);
}

// Stage C1 for base path x (n vertices) of task ti: its value, the mapped
// path in the other frame and both splats of the two-way estimator
// (Eq. shiftmapped; R3).  A rejected or invalid pair emits the one-way
// value now.  An accepted pair needs the mapped path's edges to be clear
// (replayed edges are clear by construction, unchanged edges are tested
// against the dynamic objects only): those rays are queued for k_trace_vis
// and the task waits for k_map_b; when the queue is full they are traced
// here.
__device__ void map_task(Ctx &c, PathCounts &pc, const Vtx *x, int n, uint32_t ti, uint32_t root,
                         int tech, int sa, int sb) {
    const LaunchArgs &A = c.A;
    const WaveBuf &W = A.W;
    const int g = A.frame, g2 = 3 - g;
    int pa, ex;
    const float3 fx = path_throughput(c, g, x, n, pa, ex);
    if (zero3(fx)) return;
    ++pc.paths;
    const float invN = A.invN;
    const float sign = (g == 2) ? 1.0f : -1.0f;
    // the ghost terms of P_g(x) search x's edges against the objects at
    // their frame-g' pose: the same query as the dynamic-only visibility of
    // an edge the mapping leaves unchanged
    uint32_t searched = 0u, crossed = 0u;
    const SF Pg = mis_denominator(c, g, x, n, &searched, &crossed);
    const float3 v1 = fx * ldexpf(sign * invN / Pg.m, ex - Pg.e);     // one-way value
    Vtx y[kMaxVerts];
    MapInfo mi;
    mi.J = 1.0f;
    mi.replayed = 0u;
    if (A.map_mode == 0) mi.status = MAP_OFF;
    else map_path(c, g, g2, x, n, y, mi);
    int pb = -1, ey = 0;
    float3 fy = f3(0, 0, 0);
    SF Py{0.f, 0};
    uint32_t same = 0u;              // edges the mapping leaves unchanged
    if (mi.status == MAP_ACCEPT) {
        for (int j = 0; j + 1 < n; ++j)
            if (same3(x[j].p, y[j].p) && same3(x[j + 1].p, y[j + 1].p)) same |= 1u << j;
        // an unchanged edge that crosses the objects at their frame-g' pose
        // blocks the mapped path
        if (same & crossed) mi.status = MAP_INVALID;
    }
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

}  // namespace

// stage C1: one thread per mapping task (map_task).  Latency-bound (long
// dependent loads, divergent lanes): 8 blocks per SM at 64 registers run it
// faster than 4 blocks at 128 despite the spills
__global__ void __launch_bounds__(kBlock, 8) k_map_a(const __grid_constant__ LaunchArgs A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    PathCounts pc{0, 0, 0};
    const uint32_t n = min(A.W.counts[cnt_tasks()], A.W.qt);
    Vtx x[kMaxVerts];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 t = A.W.tasks[i];
        const int lay = (t.y == T_7 || t.y == T_5) ? T_PT : t.y;   // slot layout of the technique
        const int k = assemble(c, (uint32_t)t.x, lay, t.z, t.w, x);
        map_task(c, pc, x, k, i, A.root_begin + (uint32_t)t.x, t.y, t.z, t.w);
    }
    if (A.stats) {
        add_stat(A.stats, ST_PATHS, pc.paths);
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_ACCEPTED, pc.accepted);
        add_stat(A.stats, ST_REJECTED, pc.rejected);
    }
}

// stage C2: the queued edges of mapped paths, in the other frame; a blocked
// edge makes its task's pair invalid
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_vis(const __grid_constant__ LaunchArgs A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const WaveBuf &W = A.W;
    const uint32_t n = min(W.counts[cnt_vis()], W.qv);
    const int g2 = 3 - A.frame;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t tv = W.v_task[i];
        if (tv == ~0u) continue;
        const uint32_t ti = tv & 0x7fffffffu;
        if (!W.m_vis[ti]) continue;               // another edge already blocked
        Hit h;
        ++c.cnt.rays_shadow;
        if (scene_trace(c, g2, load3(W.v_o, W.qv, i), load3(W.v_d, W.qv, i), A.S.eps, W.v_tmax[i],
                        W.v_ex0[i], W.v_ex1[i], true, (tv >> 31) != 0u, h))
            W.m_vis[ti] = 0u;
    }
    if (A.stats) {
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_NODES_S, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS_S, c.cnt.tris);
    }
}

// stage C3: the waiting tasks emit their two-way pair, or the one-way value
// when an edge of the mapped path was blocked (an invalid image, R4)
__global__ void __launch_bounds__(256) k_map_b(const __grid_constant__ LaunchArgs A) {
    Ctx c(A, nullptr);
    const WaveBuf &W = A.W;
    const uint32_t n = min(W.counts[cnt_pend()], W.qt);
    unsigned int accepted = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
    }
    if (A.stats) add_stat(A.stats, ST_ACCEPTED, accepted);
}

// --- host: one wave --------------------------------------------------------

namespace {

cudaEvent_t timer_event(KernelTimer *t) {
    if (t->pool_used == t->pool_n) {
        if (t->pool_n == t->pool_cap) {
            int cap = t->pool_cap ? 2 * t->pool_cap : 256;
            cudaEvent_t *p = new cudaEvent_t[cap];
            for (int i = 0; i < t->pool_n; ++i) p[i] = t->pool[i];
            delete[] t->pool;
            t->pool = p;
            t->pool_cap = cap;
        }
        cudaEventCreate(&t->pool[t->pool_n++]);
    }
    return t->pool[t->pool_used++];
}

void timer_begin(KernelTimer *t, cudaStream_t s, cudaEvent_t *e0, cudaEvent_t *e1) {
    *e0 = timer_event(t);
    *e1 = timer_event(t);
    cudaEventRecord(*e0, s);
}

void timer_end(KernelTimer *t, const char *name, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    cudaEventRecord(e1, s);
    if (t->n == t->cap) {
        int cap = t->cap ? 2 * t->cap : 256;
        KernelTimer::Entry *p = new KernelTimer::Entry[cap];
        for (int i = 0; i < t->n; ++i) p[i] = t->entries[i];
        delete[] t->entries;
        t->entries = p;
        t->cap = cap;
    }
    t->entries[t->n++] = KernelTimer::Entry{name, e0, e1};
}

inline int grid_for(uint32_t n, int block, int cap) {
    uint32_t g = (n + block - 1) / block;
    return (int)(g < (uint32_t)cap ? (g > 0 ? g : 1) : cap);
}

// one launch, optionally bracketed by timing events
#define RP_LAUNCH(name, grid, block, kernel, ...)                                    \
    do {                                                                             \
        cudaEvent_t e0_ = nullptr, e1_ = nullptr;                                    \
        if (a.timer) timer_begin(a.timer, s, &e0_, &e1_);                           \
        kernel<<<(grid), (block), 0, s>>>(__VA_ARGS__);                             \
        if (a.timer) timer_end(a.timer, name, s, e0_, e1_);                         \
    } while (0)

// stage C: map every task, trace the mapped paths' queued edges, emit
void map_stage(const LaunchArgs &a, cudaStream_t s, int gQ) {
    RP_LAUNCH("k_map_a", gQ, kBlock, k_map_a, a);
    RP_LAUNCH("k_trace_vis", gQ, kBlock, k_trace_vis, a);
    RP_LAUNCH("k_map_b", gQ, 256, k_map_b, a);
}

template <int T>
cudaError_t run_wave(const LaunchArgs &a, cudaStream_t s) {
    const uint32_t n = a.root_end - a.root_begin;
    const int D = a.S.max_depth;
    const int gR = grid_for(n, 256, 1 << 20);
    const int gQ = a.grid_q > 0 ? a.grid_q : 152 * 16;   // persistent-style grids over device-side counts
    cudaError_t e = cudaMemsetAsync(a.W.counts, 0, sizeof(unsigned int) * kCountSlots, s);
    if (e != cudaSuccess) return e;
    RP_LAUNCH("k_gen", gR, 256, k_gen<T>, a);
    if (T == T_3 && a.G.use_net) {
        RP_LAUNCH("k_encode3", gR, 128, k_encode3, a);
        cudaEvent_t e0_ = nullptr, e1_ = nullptr;
        if (a.timer) timer_begin(a.timer, s, &e0_, &e1_);
        e = launch_guide_infer(a.G.net, a.G.gin, n, a.G.gout, a.G.err, s);
        if (a.timer) timer_end(a.timer, "k_guide_infer", s, e0_, e1_);
        if (e != cudaSuccess) return e;
        RP_LAUNCH("k_start3g", gR, 256, k_start3g, a);
    }
    int it0 = 1;
    if (T == T_1 || T == T_2) {
        RP_LAUNCH("k_trace_shadow", gQ, kBlock, k_trace_shadow, a, 0);
        RP_LAUNCH("k_start", gR, 256, k_start<T>, a);
        RP_LAUNCH("k_trace_shadow", gQ, kBlock, k_trace_shadow, a, 1);
        it0 = 1;
    }
    // iterations: closest rays pushed at iteration it-1 are traced, extended
    // into iteration it's rays, and the new shadow rays (slot it+1) traced
    const int iters = D + 1;
    for (int it = it0; it <= iters && it + 1 < kMaxIter; ++it) {
        RP_LAUNCH("k_trace_closest", gQ, kBlock, k_trace_closest, a, it - 1);
        RP_LAUNCH("k_extend", gQ, 256, k_extend<T>, a, it);
        RP_LAUNCH("k_trace_shadow", gQ, kBlock, k_trace_shadow, a, it + 1);
    }
    const int gE = grid_for(n, 128, 1 << 20);
    if constexpr (T == T_4 || T == T_5 || T == T_6) {
        // ghost techniques exist only with motion: always mapped
        RP_LAUNCH("k_enum", gE, 128, k_enum<T>, a);
        map_stage(a, s, gQ);
    } else {
        if (a.residual && a.E.motion) {
            RP_LAUNCH("k_enum", gE, 128, k_enum<T>, a);
            map_stage(a, s, gQ);
        } else {
            // per-technique names in the kernel timings
            const char *ename = T == T_1 ? "k_eval_t1" : T == T_2 ? "k_eval_t2" : T == T_3 ? "k_eval_t3" : "k_eval_pt";
            RP_LAUNCH(ename, gE, 128, k_eval_fast<T>, a);
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wave(int tech, const LaunchArgs &a, cudaStream_t s) {
    switch (tech) {
    case 1: return run_wave<T_1>(a, s);
    case 2: return run_wave<T_2>(a, s);
    case 3: return run_wave<T_3>(a, s);
    case 4: return a.E.motion ? run_wave<T_4>(a, s) : cudaSuccess;
    case 5: return a.E.motion ? run_wave<T_5>(a, s) : cudaSuccess;
    case 6: return a.E.motion ? run_wave<T_6>(a, s) : cudaSuccess;
    case 7:
    case 0: return run_wave<T_PT>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rp
