// Internal layout of scenes and edits on the device, shared by the host
// library code and the kernels (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "guide.h"
#include "rp_wave.h"

namespace rp {

constexpr int kMaxDepth = 10;          // maximum path edges accepted by the API
constexpr int kMaxVerts = kMaxDepth + 2;
constexpr int kStackDepth = 40;        // traversal stack entries per thread
constexpr int kBvhMaxDepth = 38;       // the builder never exceeds this depth
constexpr int kBlock = 128;            // threads per block of the path kernels
constexpr int kMaxInst = 8;            // objects moved together by one edit

// BVH node: both children's boxes, 64 bytes.
//   a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   c = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   d = (child0, child1, count0, count1) as int; child >= 0 is an inner
//       node, child < 0 a leaf whose first triangle is ~child.
// Leaf triangles: 3 float4 (v0, v1, v2); v0.w holds the global triangle id.
struct DevBVH {
    const float4 *nodes;
    const float4 *tris;
    int n_nodes;
    int n_tris;
};

// one object of an edit's dynamic set: its BVH in object space (leaf ids
// n_static + local id), triangles by local id (object-space vertices, .w =
// unit normal), bounding sphere (object space, radius inflated so that the
// test is conservative).  Its dynamic triangle ids are n_static + base +
// local id.
struct DevInst {
    DevBVH bvh;
    const float4 *tri;
    int base, n;
    float4 bs;
};

struct DevScene {
    DevBVH stat;
    const float4 *stat_tri;     // [n_static][3] world vertices by triangle id; .w = unit normal
    const uint32_t *stat_mat;   // [n_static] material index
    const float *mats;          // [n_mats][12]
    const uint32_t *dyn_cdf;    // [n_dyn] area CDF thresholds over the dynamic triangles of all
                                // instances (in instance order), see below
    const uint32_t *emit_cdf;   // [n_emit] area CDF thresholds of the emitters
    // uniforms are k / 2^24; triangle i is picked for the smallest i with
    // k < cdf[i], where cdf[i] = ceil(CDF_i * 2^24) in double precision
    const double2 *cs_hi, *cs_lo;   // (cos, sin) of 2 pi h / 2^12 and 2 pi l / 2^24, h, l < 4096
    const int *emit_ids;        // [n_emit] static triangle ids
    int n_static, n_dyn, n_emit, n_mats;
    float dyn_area, emit_area;
    int n_inst;                 // objects in the dynamic set (1..kMaxInst)
    DevInst inst[kMaxInst];
    float3 cam_pos, cam_fwd, cam_right, cam_up;
    float hw, hh, pix_area, film_area;
    int W, H;
    int max_depth;
    float alpha_min, d_min, jac_max, eps;
};

// An edit of up to kMaxInst objects; per object and frame (g = 1 original,
// 2 edited) its transforms and material, read through M(o, g), Minv(o, g)
// and mat(o, g).
struct DevEdit {
    float M_[kMaxInst][2][12];      // object -> world (row-major 3x4)
    float Minv_[kMaxInst][2][12];   // world -> object
    float mat_[kMaxInst][2][12];    // the object's material
    int n_inst;
    int object[kMaxInst];       // the edited objects (0: the scene's dynamic mesh)
    int motion;                 // some object has M1 != M2
    int skip_lo, skip_n;        // static triangles [skip_lo, skip_lo + skip_n) hold the moved
                                // objects' base poses: static traversal skips them
    const uint32_t *skip_bits;  // if set, only ids whose bit (id - skip_lo) is set are skipped
    const uint32_t *cdf;        // several objects: the area CDF over all of them (edit-owned)
    __host__ __device__ __forceinline__ const float *M(int o, int g) const { return M_[o][g - 1]; }
    __host__ __device__ __forceinline__ const float *Minv(int o, int g) const { return Minv_[o][g - 1]; }
    __host__ __device__ __forceinline__ const float *mat(int o, int g) const { return mat_[o][g - 1]; }
};

// a movable object: its BVH in object space, triangles, area sampling table
struct DevObject {
    DevBVH bvh;
    const float4 *tri;
    const uint32_t *cdf;
    int n;
    float area;
    float4 bs;                  // bounding sphere (object space, conservative)
    int skip_lo, skip_n;
};

struct Record {
    uint32_t root;
    int32_t tech, frame;
    int32_t sa, sb;
    int32_t pix_a, pix_b;
    float va[3], vb[3];
    int32_t status;
    float Pg, Py, J;
};

enum StatIndex {
    ST_ROOTS = 0, ST_PATHS, ST_RAYS_CLOSEST, ST_RAYS_SHADOW, ST_NODES, ST_TRIS,
    ST_ACCEPTED, ST_REJECTED, ST_NODES_C, ST_TRIS_C, ST_NODES_S, ST_TRIS_S, ST_COUNT
};

// host-side record of kernel launches bracketed by events (per-kernel timing)
struct KernelTimer {
    struct Entry {
        const char *name;
        cudaEvent_t start, stop;
    };
    Entry *entries = nullptr;
    int n = 0, cap = 0;
    cudaEvent_t *pool = nullptr;
    int pool_n = 0, pool_cap = 0, pool_used = 0;
    char only[32] = {0};        // if set: only launches of the kernel of this name are timed
    bool wants(const char *name) const {
        if (!only[0]) return true;
        for (int i = 0; i < 32; ++i) {
            if (only[i] != name[i]) return false;
            if (!name[i]) return true;
        }
        return true;
    }
};


// learned proposal of technique (3) during a render
struct GuideLaunch {
    int on;                     // training samples of technique (3) are collected
    int use_net;                // technique (3) draws its light-side direction from the network
    GuideNet net;
    int8_t *gin;                // [R][80] integer input features (wave-local roots)
    float *gout;                // [R][48] network outputs
    float *gratio;              // [R] p_cos / q of the drawn direction
    GuideSamples smp;           // training samples; frame g, root r < half at (g - 1) half + r
    uint32_t half;
    int *err;                   // tensor-core wait timeout flag
};

struct LaunchArgs {
    DevScene S;
    DevEdit E;
    int frame;
    uint32_t root_begin, root_end;
    uint64_t seed;
    const unsigned long long *seed_dev;   // if set, the seed is read from device memory
    int grid_q;                 // blocks of the queue kernels (0: by the wave's roots)
    float invN;                 // 1 / (spp * W * H)
    int tech_mask;
    double *img;                // accumulation image or null
    Record *rec;                // records or null
    unsigned long long rec_cap;
    unsigned long long *rec_count;
    unsigned long long *stats;  // ST_COUNT counters or null
    WaveBuf W;                  // wavefront buffers (wavefront mode)
    int residual;               // 1: residual techniques, 0: primal path tracing
    int map_mode;               // 2: camera replay for dynamic first edges, else object
                                // transform (default); 1: object transform only; 0: off
    KernelTimer *timer;         // host only: per-kernel event timing, or null
    GuideLaunch G;              // learned proposal (G.on = 0: none)
};

// launchers implemented in the .cu files
cudaError_t launch_residual(int tech, const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_primal(const LaunchArgs &a, cudaStream_t s);
// closest hits of n rays; node visits, triangle tests and rays are added to
// stats[ST_*] when stats is not null
cudaError_t launch_trace(const DevScene &S, const DevEdit &E, int frame, uint32_t n,
                         const float *o, const float *d, float *t, int32_t *prim, float *b1,
                         float *b2, unsigned long long *stats, cudaStream_t s);
cudaError_t launch_philox(uint32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                          cudaStream_t s);
// streaming multiprocessors of the current device (cached per device)
int device_sm_count();
cudaError_t launch_add_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t s);
// one wave [root_begin, root_end) of one technique (0 = primal path tracing)
// in frame a.frame through the wavefront kernels
cudaError_t launch_wave(int tech, const LaunchArgs &a, cudaStream_t s);

// persistent batch kernel (k_batch.cu): one launch runs every stage of up to
// kMaxBatchJobs waves (jobs) of one technique, frame and edit kind
constexpr int kMaxBatchJobs = 128;
// stages of one wave at the largest depth (kMaxDepth = 10, motion): clear,
// generate, 3 root steps, 3 per walk iteration (11), enumerate, map start,
// 3 per mapping round (9), finish, visibility, pairs = 70
constexpr int kMaxBatchStages = 72;
struct BatchRound {
    const LaunchArgs *jobs;     // [n_jobs] in device memory, each with its own wave buffers
    int n_jobs;
    int n_stages;
    int2 stages[kMaxBatchStages];   // (stage kind, iteration), from batch_stages
    unsigned int *work;         // [n_stages] work-item counters, zero at launch
    unsigned int *bar;          // [2] grid barrier: arrivals, generation; zero at launch
    int *err;                   // set when a barrier wait gave up
    uint32_t chunk;             // elements (roots, rays, tasks) per work item of one warp
};
// the stage sequence of one wave (as run_wave launches it); returns its length
int batch_stages(int tech, int D, bool mapped, int2 *out);
// cooperative launch of one round; blocks_per_sm caps the blocks per SM
// (0: as many as fit)
cudaError_t launch_batch_round(int tech, const BatchRound &R, int blocks_per_sm, cudaStream_t s);

}  // namespace rp
