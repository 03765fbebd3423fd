/*
 * rp.h -- C ABI of librp, a GB300 (sm_103a) implementation of residual path
 * integrals for re-rendering (Xu, Li, Georgiev, Hedstrom, Ramamoorthi,
 * EGSR 2024, arXiv 2406.16302).
 *
 * Given a scene, an original frame (1) and an edit that produces frame 2
 * (a rigid motion of one object, or a material change of it), the library
 * estimates only the residual image I2 - I1 (Sec. 3.2, "The residual path
 * integral"): Monte Carlo paths are rooted on the edited object and traced
 * toward the camera and the lights (Sec. 4.1), each path is mapped into the
 * other frame with its Jacobian (Sec. 5), weighted by the balance heuristic
 * over all techniques (Sec. 4.3) and splatted.
 *
 * Conventions shared by every entry point:
 *   - All pointers named `d_*` are device pointers; all others are host
 *     pointers.  The caller owns every buffer it passes; the library owns
 *     scenes and edits.
 *   - Images are row-major [height][width][3] linear RGB radiance, row 0 at
 *     the top.  Render calls ACCUMULATE into the caller's image.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Render and query calls are stream-ordered and asynchronous;
 *     argument errors are returned synchronously, launch errors as
 *     RP_ERR_CUDA.  rp_last_error() returns a thread-local message for the
 *     last failing call.
 *   - Every path is fixed by (scene, edit, spp, seed): random numbers come
 *     from Philox4x32-10 counters keyed by (root, technique, frame, walk side,
 *     step), never by call order.  Only the order of floating-point atomic
 *     additions into the image varies between runs.
 *   - The library never falls back to a CPU path: without a usable CUDA
 *     device every call that needs one returns RP_ERR_CUDA.
 */
#ifndef RP_H
#define RP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RP_OK = 0,
    RP_ERR_INVALID_ARG = 1,
    RP_ERR_OOM = 2,
    RP_ERR_CUDA = 3,
    RP_ERR_TIMEOUT = 4,
    RP_ERR_UNSUPPORTED = 5
} rp_status;

/* techniques, as bits of a technique mask (Sec. 4.1 and 4.3) */
#define RP_TECH_DYNAMIC_FROM_EMITTER 1u  /* (1): x_D, NEE to x_L, walk to the sensor */
#define RP_TECH_DYNAMIC_FROM_SENSOR  2u  /* (2): x_D seen by the sensor, walk to the lights */
#define RP_TECH_DYNAMIC_TWO_ENDS     4u  /* (3): x_D, cosine light side, BSDF eye side */
#define RP_TECH_PATH_TRACING         8u  /* path tracing with static paths rejected */
#define RP_TECH_ALL                 15u  /* (1), (2), (3) and path tracing */
/* ghost techniques (Sec. 4.2), for edits with motion: a point x_G sampled by
 * area on the ghost (the edited object at its pose of the other frame) */
#define RP_TECH_GHOST_FROM_EMITTER  16u  /* (4): the ray from x_L through x_G, walk to the sensor */
#define RP_TECH_GHOST_FROM_SENSOR   32u  /* (5): the camera ray through x_G, walk to the lights */
#define RP_TECH_GHOST_TWO_ENDS      64u  /* (6): rays from x_G along +w and -w, uniform w, walks */
#define RP_TECH_GHOSTS             112u
#define RP_TECH_SEVEN              127u

/* Material row: 12 floats
 *   [type, albedo r g b, alpha, f0 r g b, emission r g b, unused]
 * type 0 = Lambert (albedo / pi), 1 = GGX microfacet reflection (Walter et
 * al. 2007: D = GGX, separable Smith masking, Schlick Fresnel with F0).
 * Triangles are one-sided: the front side is cross(v1 - v0, v2 - v0).
 * A triangle whose material has non-zero emission is an area light that
 * emits from its front side. */
#define RP_MATERIAL_FLOATS 12

typedef struct {
    /* static geometry, world space */
    const float *static_vertices;      /* [n_static_vertices][3] */
    uint32_t n_static_vertices;
    const uint32_t *static_triangles;  /* [n_static_triangles][3] vertex indices */
    const uint32_t *static_material;   /* [n_static_triangles] material index */
    uint32_t n_static_triangles;
    /* the edited (dynamic) object, object space; its material comes from the edit */
    const float *dyn_vertices;         /* [n_dyn_vertices][3] */
    uint32_t n_dyn_vertices;
    const uint32_t *dyn_triangles;     /* [n_dyn_triangles][3] */
    uint32_t n_dyn_triangles;
    const float *materials;            /* [n_materials][RP_MATERIAL_FLOATS] */
    uint32_t n_materials;
    /* pinhole camera: position, look-at point, up vector, vertical field of
     * view in degrees; a box pixel filter over width x height pixels */
    float camera[10];
    uint32_t width, height;
    /* maximum number of path edges (Eq. pathcontribution with k - 1 <= max_depth) */
    uint32_t max_depth;
    /* reconnection thresholds alpha_min and d_min and the Jacobian threshold
     * (Sec. 5, "Keep vertex the same" criteria 2 and 3, "Path rejection") */
    float alpha_min, d_min, jacobian_max;
    /* further movable objects (may be 0 / NULL): object k (k = 1 .. n_objects)
     * is the range object_ranges[2(k-1)] (first static triangle) ..
     * + object_ranges[2(k-1)+1] (count) of the static triangles; it stays
     * static unless an edit moves it, and its given coordinates are its
     * object space (an edit's M1, M2 map them to each frame).  Movable
     * objects may not be emissive. */
    uint32_t n_objects;
    const uint32_t *object_ranges;
} rp_scene_desc;

typedef struct rp_scene_s rp_scene;
typedef struct rp_edit_s rp_edit_handle;

/* Build a scene: copies all host arrays, builds SAH BVHs for the static
 * geometry and for the dynamic object (object space), sampling tables for
 * the dynamic object's area (p(x_D), Sec. 4.1) and the emitters' area
 * (p(x_L)), and uploads them to the current CUDA device.  Synchronous.
 * Errors: RP_ERR_INVALID_ARG (null pointers, indices out of range, no
 * emitter, no dynamic triangle, max_depth outside [2, 12], emissive dynamic
 * material), RP_ERR_OOM, RP_ERR_CUDA. */
rp_status rp_scene_create(const rp_scene_desc *desc, rp_scene **out);
/* Frees a scene and its device memory (NULL: no-op).  Destroy the edits,
 * guides attached to it and batches made from it first; the frees wait for
 * the device, so queued work that uses the scene completes first. */
void rp_scene_destroy(rp_scene *scene);

/* An edit: the dynamic object's object-to-world transform (row-major 3x4)
 * and material row in frame 1 (original) and frame 2 (edited).  A rigid
 * motion keeps the material ("Transform with object movement", Sec. 5); a
 * material edit keeps the transform (Sec. 6, "Scene editing"); both may
 * change at once.  Transforms must be rigid (orthonormal 3x3 part within
 * 1e-4), else RP_ERR_UNSUPPORTED.  Synchronous, small upload. */
typedef struct {
    float M1[12], M2[12];
    float mat1[RP_MATERIAL_FLOATS], mat2[RP_MATERIAL_FLOATS];
    /* the edited object: 0 = the dynamic mesh of the scene description,
     * k >= 1 = movable object k (its base pose in the static geometry is
     * replaced by the object under M1 / M2) */
    uint32_t object;
} rp_edit_desc;

/* Errors: RP_ERR_INVALID_ARG (null pointers, object out of range, bad
 * material), RP_ERR_UNSUPPORTED (non-rigid transform, emissive material),
 * RP_ERR_OOM. */
rp_status rp_edit(rp_scene *scene, const rp_edit_desc *desc, rp_edit_handle **out);

/* An edit of n objects at once (1 <= n <= 8; Sec. 6 measures scenes with
 * several moving objects): descs[k] names object k of the edit (distinct
 * objects) with its transforms and materials, as for rp_edit.  The objects
 * form one dynamic set: x_D is sampled by area over all of them (p = 1 /
 * total area), a path with more than one dynamic vertex is rejected by the
 * mapping (R4) whichever objects they lie on, and the ghost is every object
 * at its other-frame pose.  The edit owns device tables (the area CDF over
 * the objects, and a bit mask of the moved base poses when they are not one
 * contiguous range of static triangles): keep it alive while any render or
 * batch that uses it may run.  Errors: RP_ERR_INVALID_ARG (n out of range,
 * an object listed twice or out of range, bad material), RP_ERR_UNSUPPORTED
 * (non-rigid transform, emissive material), RP_ERR_OOM.  A scene with a
 * learned proposal renders edits of one object only (RP_ERR_UNSUPPORTED). */
rp_status rp_edit_multi(rp_scene *scene, const rp_edit_desc *descs, uint32_t n,
                        rp_edit_handle **out);
/* Frees an edit and its device tables (NULL: no-op); no render or batch that
 * uses it may still be queued. */
void rp_edit_destroy(rp_edit_handle *edit);

/* Residual image I2 - I1 (Eq. shiftmapped restricted to dynamic paths,
 * Eq. difference_integral): N = spp * width * height roots for every
 * technique in `tech_mask` and both frames; accumulated with FP64 atomics
 * into d_out[height][width][3] (double).  Unbiased when tech_mask contains
 * RP_TECH_PATH_TRACING.  Asynchronous on `stream`. */
rp_status rp_render_residual(rp_scene *scene, const rp_edit_handle *edit, uint32_t spp,
                             uint64_t seed, uint32_t tech_mask, double *d_out, void *stream);

/* Same estimate written into a float32 image: accumulated in a library-owned
 * FP64 scratch image, then added to d_out[height][width][3] (float).
 * The scratch image is allocated on first use per scene and reused; calls on
 * one scene must not overlap. */
rp_status rp_render_residual_f32(rp_scene *scene, const rp_edit_handle *edit, uint32_t spp,
                                 uint64_t seed, uint32_t tech_mask, float *d_out, void *stream);

/* rp_render_residual_f32 without any device allocation.  The paper has no
 * counterpart: this serves hosts that cannot let a library allocate device
 * memory (they manage every byte through their own pool, run under a hard
 * memory cap, or forbid allocation after start-up because cudaMalloc may
 * synchronise the device).  Instead of a cudaMalloc'd scratch image the call
 * uses a fixed FP64 array of RP_NOALLOC_MAX_PIXELS * 3 doubles (24 MiB)
 * compiled into the library's device image.  A device holds it from the
 * first call on that device (CUDA loads the library's device code lazily by
 * default) or from library load when CUDA_MODULE_LOADING=EAGER, until the
 * process exits.  Same arguments and accumulation into d_out as
 * rp_render_residual_f32, with two differences:
 *   - it runs the one-thread-per-root kernels, which have no ghost
 *     techniques: a tech_mask with any RP_TECH_GHOSTS bit returns
 *     RP_ERR_UNSUPPORTED;
 *   - a learned proposal attached to the scene (rp_scene_set_guide) is not
 *     used, so with a guide the image differs from rp_render_residual_f32's
 *     (both are unbiased estimates of the same residual).
 * Errors and sharing:
 *   - width * height above RP_NOALLOC_MAX_PIXELS: RP_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address
 *     (once per device, with that device current); make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and clears it first: calls
 *     that overlap on the GPU (other streams, other threads) race and give
 *     wrong images.  Serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define RP_NOALLOC_MAX_PIXELS (1024u * 1024u)
rp_status rp_render_residual_f32_noalloc(rp_scene *scene, const rp_edit_handle *edit,
                                         uint32_t spp, uint64_t seed, uint32_t tech_mask,
                                         float *d_out, void *stream);

/* End-to-end convenience call with HOST buffers: uploads the edit, renders
 * the residual and copies it into host_out[height][width][3] (double,
 * overwritten, not accumulated).  Synchronous on `stream`. */
rp_status rp_render_residual_host(rp_scene *scene, const rp_edit_desc *edit, uint32_t spp,
                                  uint64_t seed, uint32_t tech_mask, double *host_out,
                                  void *stream);

/* Primal image of frame 1 or 2 by path tracing with next-event estimation
 * (Eq. pathIntegral): the "PT from scratch" baseline of Sec. 6 and, with the
 * same seed in both frames, correlated path tracing.  Accumulates into
 * d_out (double).  Asynchronous. */
rp_status rp_render_primal(rp_scene *scene, const rp_edit_handle *edit, int frame, uint32_t spp,
                           uint64_t seed, double *d_out, void *stream);

/* Per-sample records for roots [root_begin, root_end) of one technique
 * (1, 2, 3 or 7 = path tracing) in one frame, for parity testing.  Each
 * base path with non-zero contribution yields one record; d_count receives
 * the number of records produced (may exceed capacity; only the first
 * `capacity` are written).  This is the deterministic mode: each record's
 * values are bitwise reproducible for (scene, edit, spp, seed) and carry no
 * atomic summation; only the order of the records varies (sort by root,
 * technique, frame and strategy).  Asynchronous. */
typedef struct {
    uint32_t root;
    int32_t tech, frame;
    int32_t sa, sb;          /* strategy: (t', s') walk lengths or path length */
    int32_t pix_a, pix_b;    /* pixel of the base path and of the mapped path (-1: none) */
    float va[3], vb[3];      /* the two splats */
    int32_t status;          /* 0 accepted pair, 1 invalid mapped path, 2-5 rejected */
    float Pg, Py, J;         /* MIS denominators of x and T(x), Jacobian */
} rp_record;

rp_status rp_dump_samples(rp_scene *scene, const rp_edit_handle *edit, int tech, int frame,
                          uint32_t spp, uint64_t seed, uint32_t root_begin, uint32_t root_end,
                          uint32_t tech_mask, rp_record *d_records, uint64_t capacity,
                          unsigned long long *d_count, void *stream);

/* Closest hits of n rays in frame 1 or 2 (static BVH and the dynamic BVH
 * under that frame's transform; watertight ray/triangle test of Woop,
 * Benthin and Wald 2013).  t = +inf and prim = -1 on a miss; prim numbers
 * static triangles first, then the dynamic object's.  Asynchronous. */
rp_status rp_trace_closest(rp_scene *scene, const rp_edit_handle *edit, int frame, uint32_t n,
                           const float *d_origins, const float *d_dirs, float *d_t,
                           int32_t *d_prim, float *d_b1, float *d_b2, void *stream);

/* The BVH that rp_scene_create builds for a mesh, built on the host only
 * (no device needed), for inspection and tests.  verts: [n_verts][3] float;
 * tris: [n_tris][3] vertex indices.  Writes *n_nodes (inner nodes) and
 * *depth (inner levels); if nodes_out is not NULL it receives n_nodes x 16
 * floats in the 64-byte node layout (four float4: child 0 x/y bounds,
 * child 1 x/y bounds, both z bounds, then child0, child1, count0, count1 as
 * int bits; a child >= 0 is an inner node, < 0 a leaf whose first triangle
 * in leaf order is ~child), node_cap >= n_nodes; if tris_out is not NULL it
 * receives n_tris x 12 floats (v0, v1, v2 as float4, v0.w = the triangle's
 * index as int bits) in leaf order.  The binned-SAH build stands in for the
 * ray-tracing library of the paper's implementation (Sec. 6).  Synchronous;
 * RP_ERR_INVALID_ARG for null arguments, no triangles, an index out of
 * range or a short node buffer. */
rp_status rp_bvh_build_host(const float *verts, uint32_t n_verts, const uint32_t *tris,
                            uint32_t n_tris, float *nodes_out, uint32_t node_cap,
                            float *tris_out, uint32_t *n_nodes, int *depth);

/* Philox4x32-10 on the device for n (counter[4], key[2]) pairs, for
 * known-answer tests.  Asynchronous. */
rp_status rp_philox(uint32_t n, const uint32_t *d_counters, const uint32_t *d_keys,
                    uint32_t *d_out, void *stream);

/* Work counters of the most recent render or rp_trace_closest call on a
 * scene (synchronises the scene's last stream): roots, base paths splatted,
 * rays traced by kind and BVH nodes / triangles visited, used for the
 * traversal roofline.  rp_trace_closest counts its rays, node visits and
 * triangle tests as closest-hit work. */
typedef struct {
    unsigned long long roots;
    unsigned long long paths;
    unsigned long long rays_closest, rays_shadow;
    unsigned long long nodes_visited, tris_tested;      /* all traversals */
    unsigned long long accepted, rejected;
    unsigned long long nodes_closest, tris_closest;     /* closest-hit trace kernel */
    unsigned long long nodes_shadow, tris_shadow;       /* shadow-ray trace kernel */
} rp_stats;

rp_status rp_enable_stats(rp_scene *scene, int on);
rp_status rp_get_stats(rp_scene *scene, rp_stats *out);

/* Waits for the work most recently enqueued on a scene's stream and reports
 * how it ended: RP_OK, or RP_ERR_CUDA with the CUDA error text in
 * rp_last_error() when a kernel or copy of it failed (render calls return
 * launch errors at once but device-side failures only here or at the next
 * synchronising call).  RP_ERR_INVALID_ARG for a null scene. */
rp_status rp_sync_status(rp_scene *scene);

/* Per-kernel device times of the wavefront kernels: when enabled, every
 * launch on a scene is bracketed by CUDA events recorded on its stream.
 * rp_get_kernel_times synchronises the scene's last stream, writes up to
 * `capacity` entries (kernel name, launches, milliseconds summed over the
 * launches since the previous call) and resets the sums; *count receives the
 * number of kernels. */
typedef struct {
    char name[32];
    unsigned long long launches;
    double ms;
} rp_kernel_time;

rp_status rp_enable_timing(rp_scene *scene, int on);
rp_status rp_get_kernel_times(rp_scene *scene, rp_kernel_time *out, int capacity, int *count);

/* Timing of one kernel only: like rp_enable_timing(scene, 1), but only the
 * launches of the wavefront kernel named `kernel` (as rp_get_kernel_times
 * names it, e.g. "k_trace_closest") are bracketed by events, so that the
 * other launches run without them; NULL times every kernel.  The name is
 * copied (at most 31 characters, else RP_ERR_INVALID_ARG).  Turned off by
 * rp_enable_timing(scene, 0). */
rp_status rp_enable_timing_of(rp_scene *scene, const char *kernel);

/* ------------------------------------------------------------------------
 * Learned proposal for technique (3) (not in the paper, which names better
 * importance sampling as future work in Sec. 7).  A small network maps the
 * object-space position and normal of x_D to an 8-lobe von Mises-Fisher
 * mixture over directions.  With a guide attached to a scene, technique (3)
 * draws its first light-side direction from the defensive one-sample
 * mixture q = p_cos / 2 + (vMF mixture) / 2 and multiplies the values of the
 * root's paths by p_cos / q; the balance-heuristic weights of Sec. 4.3 stay
 * those of the plain techniques, so every network leaves the residual
 * estimator unbiased.
 *
 * Network: 80 input features, four hidden layers of 64 with ReLU, 48
 * outputs (lobe j: direction 5j..5j+2, log kappa 5j+3 clamped to
 * [-4, 6.2], logit 5j+4; 40..47 unused); weights layer-major [out][in]:
 * 64x80, 64x64, 64x64, 64x64, 48x64 (20480 values), no biases besides the
 * constant input feature.  Features of (p, n): for each coordinate of
 * u = clamp((p - center) * inv_half, -1, 1), then of n, sin(2^f pi c) and
 * cos(2^f pi c) for f = 0..5; then u; then n; then a constant and a zero.
 *
 * Rendering uses an integer network: inputs rint(128 e) in [-127, 127]
 * (the constant is 127), weights in [-127, 127], hidden activations
 * clamp(rint(z 2^-shift_l), 0, 255) (round half to even), outputs
 * z 2^-out_exp.  Every partial sum stays below 2^24, so the BF16 tensor-core
 * products with FP32 accumulation are exact.  Training uses the float
 * network (BF16 operands, FP32 accumulation) and the weighted loss
 * -sum_i wt_i log q_vmf(w_i) / sum_i wt_i over samples of guided renders
 * (w_i the drawn direction in object space, wt_i the magnitude of what
 * the root added to the image); each step ends with Adam and a
 * re-quantisation into the integer network. */
typedef struct rp_guide_s rp_guide;

/* box: (center xyz, inverse half extent xyz) of object-space positions;
 * batch: training samples per step (even, in [256, 2^24]; half per frame,
 * the roots below batch / 2 of each frame's technique (3)); seed: He
 * initialisation of the float network.  The guide has no integer network
 * until rp_guide_set_int or the first rp_guide_train_step: until then
 * technique (3) samples as without a guide and only collects samples.
 * Synchronous.  Errors: RP_ERR_INVALID_ARG, RP_ERR_OOM, RP_ERR_CUDA. */
rp_status rp_guide_create(const float *box, uint32_t batch, uint64_t seed, rp_guide **out);
/* Frees a guide (NULL: no-op); detach it from its scene first. */
void rp_guide_destroy(rp_guide *guide);

/* Float network weights (host arrays of 20480 floats); setting resets Adam. */
rp_status rp_guide_set_weights(rp_guide *guide, const float *weights);
rp_status rp_guide_get_weights(rp_guide *guide, float *weights);

/* Integer network used by renders: weights[20480] in [-127, 127], shift[4]
 * in [0, 24], out_exp in [-30, 60].  Synchronous. */
rp_status rp_guide_set_int(rp_guide *guide, const int8_t *weights, const int32_t *shift,
                           int32_t out_exp);
rp_status rp_guide_get_int(rp_guide *guide, int8_t *weights, int32_t *shift, int32_t *out_exp);

/* Integer network on n rows of device features d_in[n][80] (int8) into
 * d_out[n][48] (float, exact).  Asynchronous; a tensor-core wait that
 * times out is reported by rp_guide_status. */
rp_status rp_guide_infer(rp_guide *guide, const int8_t *d_in, uint32_t n, float *d_out,
                         void *stream);

/* The network's input features of n object-space points d_p[n][3] (double)
 * with unit normals d_n[n][3] (float), in the guide's box: for each
 * coordinate of u = clamp((p - center) * inv_half, -1, 1) and of the normal,
 * sin and cos of 2^f pi x for f = 0..5, then u and the normal, each
 * quantised to rint(128 e) in [-127, 127], then 127 and 0: d_out[n][80]
 * (int8), the rows rp_guide_infer takes and technique (3) computes for x_D.
 * Asynchronous.  Errors: RP_ERR_INVALID_ARG, RP_ERR_CUDA. */
rp_status rp_guide_encode(rp_guide *guide, const double *d_p, const float *d_n, uint32_t n,
                          int8_t *d_out, void *stream);

/* Float network: the mean loss (1/n) sum_i -wt_i log q_vmf(w_i) of n rows
 * (d_x[n][80] features, rounded to BF16; d_omega[n][3] unit directions;
 * d_wt[n] weights; rows with wt <= 0 add nothing) and its gradient with
 * respect to the weights, ADDED into d_grad[20480] and d_loss[1].
 * Asynchronous. */
rp_status rp_guide_loss_grad(rp_guide *guide, const float *d_x, const float *d_omega,
                             const float *d_wt, uint32_t n, float *d_grad, float *d_loss,
                             void *stream);

/* One training step on the samples of the most recent guided render: batch
 * features, loss gradient, Adam (lr; beta 0.9, 0.99), re-quantisation.
 * Synchronises `stream`; *loss receives the weighted loss (may be NULL).
 * Errors: RP_ERR_TIMEOUT (a tensor-core wait gave up), RP_ERR_CUDA. */
rp_status rp_guide_train_step(rp_guide *guide, float lr, float *loss, void *stream);

/* RP_ERR_TIMEOUT if a guide kernel's tensor-core wait gave up (synchronises
 * the device). */
rp_status rp_guide_status(rp_guide *guide);

/* Self-test of the timeout path of the tensor-core kernels (the paper has no
 * counterpart).  Runs one 128-row tile of the inference kernel with its
 * tensor-core completion signal withheld and its barrier wait bounded by
 * limit_ns (0 < limit_ns <= 2e9): nothing arrives at the barrier, the wait
 * runs out, the kernel records the timeout, releases its tensor memory and
 * returns, leaving the context usable.  Synchronous (device-wide).
 * Returns RP_ERR_TIMEOUT when the wait ran out, which is the expected
 * result, and clears the guide's timeout flag afterwards; RP_OK would mean
 * that the wait did not give up.  RP_ERR_TIMEOUT without running anything
 * when an earlier guide kernel's wait had already timed out (see
 * rp_guide_status).  Allocates two small scratch buffers. */
rp_status rp_guide_wait_selftest(rp_guide *guide, uint64_t limit_ns);

/* Attach a guide to a scene's technique (3) for the renders that follow
 * (NULL detaches).  The guide must outlive its attachment.  The
 * one-thread-per-root entry point (rp_render_residual_f32_noalloc) never
 * uses it. */
rp_status rp_scene_set_guide(rp_scene *scene, rp_guide *guide);

/* ------------------------------------------------------------------------
 * Batches of edits (animation frames) of one scene, each with its own image
 * size, sample count, seed and output, run as one CUDA graph: every wave of
 * every item is captured once; items are spread over `streams` concurrent
 * branches (longest first to the least loaded), each with its own
 * wavefront buffers, so that the tail of one item's waves overlaps another
 * item's.  Not in the paper (which names rendering many frames as future
 * work); each item's result equals rp_render_residual of that item. */
typedef struct {
    const rp_edit_handle *edit;  /* an edit of the batch's scene */
    uint32_t width, height;      /* image size; 0, 0: the scene's */
    uint32_t spp;
    uint64_t seed;               /* replaced by rp_batch_set_seeds */
    uint32_t tech_mask;
    double *d_out;               /* [height][width][3] device image, accumulated into; caller-owned,
                                    valid for the batch's lifetime */
} rp_batch_item;

typedef struct {
    uint32_t wave_roots;         /* roots per wave (0: min(largest item, 2^22)) */
    uint32_t streams;            /* graph mode: concurrent branches, 1..8 (0: 1);
                                    persistent mode: waves per round, 1..128 (0: 8) */
    uint32_t blocks_per_sm;      /* graph mode: grid of the queue kernels per SM, 1..128 (0: one
                                    block per 256 roots of a wave, 16..128 per SM);
                                    persistent mode: at most this many resident blocks per
                                    SM (0: as many as fit) */
    uint32_t persistent;         /* 0: a graph of per-wave kernel launches over `streams`
                                    branches; 1: rounds of `streams` waves (jobs: one wave of
                                    one item's technique and frame, each with its own wave
                                    buffers), each round one cooperative launch of a
                                    persistent kernel whose warps pull (job, chunk) work
                                    items of every stage from a device counter, with a
                                    grid barrier between stages */
} rp_batch_config;

typedef struct rp_batch_s rp_batch;

/* Capture the batch (allocates the branches' wavefront buffers; config NULL:
 * defaults).  The edits must outlive the batch; the scene's guide is not
 * used.  Synchronous.  Errors: RP_ERR_INVALID_ARG, RP_ERR_OOM, RP_ERR_CUDA. */
rp_status rp_batch_create(rp_scene *scene, const rp_batch_item *items, uint32_t n,
                          const rp_batch_config *config, rp_batch **out);
/* Frees a batch, its CUDA graph and its wave buffers (NULL: no-op). */
void rp_batch_destroy(rp_batch *batch);
/* One graph launch on `stream`: every item's residual added to its image. */
rp_status rp_batch_launch(rp_batch *batch, void *stream);
/* Stream-ordered upload of new per-item seeds (n values) for later launches. */
rp_status rp_batch_set_seeds(rp_batch *batch, const uint64_t *seeds, void *stream);
/* Synchronises the device and returns RP_ERR_TIMEOUT if a grid barrier of
 * the persistent kernel gave up (after about 2 s of waiting; the launch then
 * ended early and the images are incomplete), else RP_OK. */
rp_status rp_batch_status(rp_batch *batch);
/* The configuration in use and the number of graph nodes. */
rp_status rp_batch_info(rp_batch *batch, rp_batch_config *config, uint64_t *graph_nodes);
/* Autotuner: times candidate configurations on a proxy of the batch (each
 * item's spp divided by spp_divisor, outputs into a scratch image) by
 * coordinate descent in each batch mode: the graph mode over wave_roots
 * (2^20 .. 2^23), streams (1, 2, 4) and blocks_per_sm (0, 16, 32, 64, 128); the
 * persistent mode over wave_roots (2^18 .. 2^21), waves per round (4 .. 32,
 * at most 2^23 roots in flight) and resident blocks per SM (all, 4, 2).
 * Writes the fastest of both modes and its proxy time in ms.  Synchronous;
 * leaves the items' images untouched. */
rp_status rp_batch_autotune(rp_scene *scene, const rp_batch_item *items, uint32_t n,
                            uint32_t spp_divisor, rp_batch_config *best, double *best_ms);

/* Path mapping (Sec. 5) for the renders of a scene that follow:
 *   RP_MAPPING_CAMERA (2, default): paths whose first edge is dynamic (x_1 on
 *     the object, or the camera ray to x_1 crossing the ghost) keep their
 *     camera direction (Sec. 5, "Mapping between the dynamic and ghost pair")
 *     and map their light side as technique (2) does; all others move their
 *     dynamic vertex with the object;
 *   RP_MAPPING_OBJECT (1): the object transform for every path;
 *   RP_MAPPING_OFF (0): no mapping; a base path of frame g adds
 *     s_g f_g(x) / (N P_g(x)), so each frame's dynamic paths are estimated by
 *     that frame's sampling alone (the "without path mapping" comparison).
 * All three are unbiased.  Edits without motion are unaffected. */
#define RP_MAPPING_OFF 0
#define RP_MAPPING_OBJECT 1
#define RP_MAPPING_CAMERA 2
rp_status rp_scene_set_mapping(rp_scene *scene, int mode);

/* Thread-local message describing the last error (empty string if none). */
const char *rp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RP_H */
