// Wavefront buffers: per-root vertex slots and flags, SoA ray queues and the
// mapping task queue.  Owned by a scene, reused across renders.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rp {

// Vertex slots of one root (D = max depth):
//   0            root vertex: x_D (techniques 1-3) or x_1 (path tracing)
//   1            x_L of technique (1)
//   2 + m - 1    eye-side walk vertex z_m,   m = 1 .. D-2
//   D + m - 1    light-side walk vertex y_m, m = 1 .. D-2 (path tracing: x_{m+1})
//   2D-2 + m-1   next-event vertex L_m,      m = 1 .. D-1
__host__ __device__ __forceinline__ int slot_count(int D) { return 3 * D - 3; }
__host__ __device__ __forceinline__ int slot_eye(int D, int m) { (void)D; return 2 + m - 1; }
__host__ __device__ __forceinline__ int slot_light(int D, int m) { return D + m - 1; }
__host__ __device__ __forceinline__ int slot_nee(int D, int m) { return 2 * D - 2 + m - 1; }

// ray tags: wave-local root (24 bits) | side or connection kind (2 bits) |
// step (4 bits)
__host__ __device__ __forceinline__ uint32_t make_tag(uint32_t r, int side, int step) {
    return r | ((uint32_t)side << 24) | ((uint32_t)step << 26);
}
__host__ __device__ __forceinline__ uint32_t tag_root(uint32_t t) { return t & 0xffffffu; }
__host__ __device__ __forceinline__ int tag_side(uint32_t t) { return (int)((t >> 24) & 3u); }
__host__ __device__ __forceinline__ int tag_step(uint32_t t) { return (int)((t >> 26) & 15u); }

// connection kinds of shadow rays
enum { CK_CAMERA = 0, CK_NEE = 1, CK_GHOST_WALK = 2, CK_GHOST_NEE = 3 };

// per-root flag bits
enum { RF_ROOT_OK = 1, RF_GUIDE = 2 };

constexpr int kMaxIter = 16;      // counter slots per queue


struct WaveBuf {
    uint32_t R;                    // root capacity of a wave
    int S;                         // vertex slots per root
    // vertex slots, [S][R]
    float *px, *py, *pz, *nx, *ny, *nz, *b1, *b2;
    int *prim;
    // per-root state, [R]
    int *len_eye, *len_light, *flags;
    uint32_t *cam_ok, *nee_ok, *ghost_w, *ghost_n;
    // closest-hit ray queues (double-buffered) and their hits, capacity qc
    uint32_t qc;
    float *c_o[2], *c_d[2];        // [3][qc] each (x plane, then y, then z)
    int *c_ex[2];
    uint32_t *c_tag[2];
    int *h_prim;
    float *h_b1, *h_b2;
    float *h_p;                    // [3][qc] refined hit positions
    // shadow-ray queue, capacity qa
    uint32_t qa;
    float *a_o, *a_d, *a_tmax;     // a_o, a_d: [3][qa]
    int *a_ex0, *a_ex1;
    uint32_t *a_tag;
    int a_dyn_frame;               // unused placeholder for alignment
    // mapping tasks: (root, technique, sa, sb)
    uint32_t qt;
    int4 *tasks;
    // deferred visibility of mapped paths: the edges of accepted mapped
    // paths that need a test, queued by k_map_a and traced by k_trace_vis;
    // per task the splats k_map_b emits once the rays are traced
    uint32_t qv;                   // ray capacity
    float *v_o, *v_d, *v_tmax;     // v_o, v_d: [3][qv]
    int *v_ex0, *v_ex1;
    uint32_t *v_task;              // task index | 1 << 31 for a dynamic-only test; ~0u: none
    int *m_pix;                    // [2][qt] pixel of the base path, of the mapped path
    float *m_val;                  // [9][qt] two-way base splat, mapped splat, one-way splat
    float *m_w;                    // [3][qt] P_g(x), P_g'(y), J (for records)
    uint32_t *m_vis;               // [qt] 1 while none of the task's rays is blocked
    uint32_t *pend;                // [qt] tasks waiting for their rays
    // wavefront mapping: per task its mapping state, and the vertices the
    // mapping replays (a pool; a task reserves one slot per path vertex)
    uint32_t *ms_info;             // [qt] status | mode | dynamic index | step | replayed mask
    float *ms_J;                   // [qt] Jacobian so far
    uint32_t *ms_base;             // [qt] first pool slot of the task's replayed vertices
    uint32_t *fin;                 // [qt] tasks whose mapping ended: accepted from the front,
                                   // the others from the back
    uint32_t yc;                   // pool capacity (vertices)
    float *y_p, *y_n, *y_b;        // [3][yc] positions, [3][yc] normals, [2][yc] barycentrics
    int *y_prim;                   // [yc]
    // replay rays of the mapping (double-buffered queues of capacity qr)
    // and their closest hits
    uint32_t qr;
    float *r_o[2], *r_d[2];        // [3][qr] each
    int *r_ex[2];
    uint32_t *r_task[2];
    int *rh_prim;
    float *rh_b1, *rh_b2, *rh_p;   // rh_p: [3][qr]
    // counters: closest [kMaxIter], shadow [kMaxIter], tasks, rays, pending,
    // replay rays [kMaxIter], pool slots, finished tasks (accepted, others)
    unsigned int *counts;
};

__host__ __device__ __forceinline__ int cnt_closest(int it) { return it; }
__host__ __device__ __forceinline__ int cnt_shadow(int it) { return kMaxIter + it; }
__host__ __device__ __forceinline__ int cnt_tasks() { return 2 * kMaxIter; }
__host__ __device__ __forceinline__ int cnt_vis() { return 2 * kMaxIter + 1; }
__host__ __device__ __forceinline__ int cnt_pend() { return 2 * kMaxIter + 2; }
__host__ __device__ __forceinline__ int cnt_replay(int round) { return 2 * kMaxIter + 3 + round; }
__host__ __device__ __forceinline__ int cnt_pool() { return 3 * kMaxIter + 3; }
__host__ __device__ __forceinline__ int cnt_fin_acc() { return 3 * kMaxIter + 4; }
__host__ __device__ __forceinline__ int cnt_fin_rej() { return 3 * kMaxIter + 5; }
constexpr int kCountSlots = 3 * kMaxIter + 6;

}  // namespace rp
