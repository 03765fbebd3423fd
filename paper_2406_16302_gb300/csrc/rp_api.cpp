// C ABI of librp (include/rp.h): scene and edit management, argument
// checking and the stream-ordered launches of the path kernels.
#include "../../include/rp.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bvh_build.h"
#include "rp_internal.h"

using namespace rp;

namespace {

thread_local std::string g_err;

rp_status fail(rp_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

rp_status cuda_fail(cudaError_t e, const char *what) {
    return fail(RP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RP_CUDA(call, what)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

rp_status need_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(RP_ERR_CUDA, "no usable CUDA device (librp has no CPU fallback)");
    return RP_OK;
}

template <class T>
rp_status upload(const std::vector<T> &h, T **d) {
    *d = nullptr;
    if (h.empty()) return RP_OK;
    cudaError_t e = cudaMalloc((void **)d, sizeof(T) * h.size());
    if (e == cudaErrorMemoryAllocation) return fail(RP_ERR_OOM, "device allocation failed");
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    RP_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice), "upload");
    return RP_OK;
}

}  // namespace

struct rp_guide_s {
    float box[6] = {0, 0, 0, 1, 1, 1};
    uint32_t cap = 0;                  // training samples per step (both frames)
    std::vector<void *> allocs;
    // float network, Adam state, gradient, loss, activation maxima
    float *Wm = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    float *wsum = nullptr, *d_box = nullptr;
    unsigned int *amax = nullptr;
    int *err = nullptr;
    __nv_bfloat16 *Wbf = nullptr, *Wq = nullptr;
    // samples gathered by guided renders and the training batch built from them
    GuideSamples smp{};
    __nv_bfloat16 *X = nullptr;
    float *omega = nullptr, *wt = nullptr;
    // scratch of rp_guide_loss_grad
    __nv_bfloat16 *Xs = nullptr;
    size_t xs_rows = 0;
    // integer network used by renders
    bool has_int = false;
    int shift[4] = {0, 0, 0, 0};
    int out_exp = 0;
    int adam_t = 0;
    ~rp_guide_s() {
        for (void *p : allocs) cudaFree(p);
        if (Xs) cudaFree(Xs);
    }
};

// roots per wave of a render (the wave buffers scale with it, about 64 GB
// for an edit with motion at depth 8; ray tags hold 24 bits of wave-local
// root, so this is the largest wave).  A 64 spp render of the 1024^2 terrain
// edit takes 1966 ms with waves of 2^22 roots, 1815 ms with 2^23 and 1742 ms
// with 2^24 (fewer launches, fuller late bounces).
#ifndef RP_WAVE_ROOTS
#define RP_WAVE_ROOTS (1u << 24)
#endif

struct rp_scene_s {
    DevScene S{};
    std::vector<DevObject> objects;   // 0: the dynamic mesh; k >= 1: static triangle ranges
    std::vector<std::vector<double>> obj_tri_area;   // per object: triangle areas (double)
    std::vector<double> obj_area;     // per object: total area (double)
    double cam_hh = 0.0;              // tan(vfov / 2)
    std::vector<void *> allocs;
    int bvh_depth_static = 0, bvh_depth_dyn = 0;
    unsigned long long *d_stats = nullptr;
    bool stats_on = false;
    double *d_scratch = nullptr;   // FP64 image for the f32 and host entry points
    cudaStream_t last_stream = nullptr;
    // wavefront buffers (allocated on first use, grown on demand)
    WaveBuf W{};
    std::vector<void *> wave_allocs;
    bool wave_tasks = false;
    uint32_t wave_cap = RP_WAVE_ROOTS;  // roots per wave
    KernelTimer timer;
    bool timing_on = false;
    int map_mode = 2;                 // path mapping mode (rp_scene_set_mapping)
    // renders of few roots: their technique-and-frame waves run concurrently
    // on these streams, each with wave buffers of its own
    struct Lane {
        WaveBuf W{};
        std::vector<void *> allocs;
        bool tasks = false;
        cudaStream_t s = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<Lane> lanes;
    cudaEvent_t lanes_fork = nullptr;
    // learned proposal of technique (3) and its per-root buffers
    rp_guide *guide = nullptr;
    int8_t *gin = nullptr;
    float *gout = nullptr, *gratio = nullptr;
    uint32_t guide_R = 0;
    void free_guide_buffers() {
        if (gin) cudaFree(gin);
        if (gout) cudaFree(gout);
        if (gratio) cudaFree(gratio);
        gin = nullptr; gout = nullptr; gratio = nullptr;
        guide_R = 0;
    }
    void free_wave() {
        for (void *p : wave_allocs) cudaFree(p);
        wave_allocs.clear();
        W = WaveBuf{};
        wave_tasks = false;
        free_guide_buffers();
    }
    ~rp_scene_s() {
        for (void *p : allocs) cudaFree(p);
        if (d_stats) cudaFree(d_stats);
        if (d_scratch) cudaFree(d_scratch);
        free_wave();
        for (Lane &l : lanes) {
            for (void *p : l.allocs) cudaFree(p);
            if (l.s) cudaStreamDestroy(l.s);
            if (l.done) cudaEventDestroy(l.done);
        }
        if (lanes_fork) cudaEventDestroy(lanes_fork);
        for (int i = 0; i < timer.pool_n; ++i) cudaEventDestroy(timer.pool[i]);
        delete[] timer.pool;
        delete[] timer.entries;
    }
};

struct rp_edit_s {
    DevEdit E{};
    std::vector<void *> allocs;       // several objects: the area CDF and static skip bits
    ~rp_edit_s() {
        for (void *p : allocs) cudaFree(p);
    }
};

extern "C" const char *rp_last_error(void) { return g_err.c_str(); }

static bool material_ok(const float *m) {
    for (int i = 0; i < 11; ++i)
        if (!std::isfinite(m[i])) return false;
    int type = (int)m[0];
    if (!(m[0] == 0.f || m[0] == 1.f)) return false;
    if (type == 1 && !(m[4] > 0.f)) return false;
    return true;
}

// conservative bounding sphere of a triangle table (vertices in .xyz)
static float4 bounding_sphere(const std::vector<float4> &t) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (const float4 &v : t) {
        const double p[3] = {v.x, v.y, v.z};
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
    }
    const double c[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
    double r2 = 0.0;
    for (const float4 &v : t) {
        const double d[3] = {v.x - c[0], v.y - c[1], v.z - c[2]};
        r2 = std::max(r2, d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    const double r = std::sqrt(r2);
    return make_float4((float)c[0], (float)c[1], (float)c[2], (float)(r * 1.001 + 1e-5));
}

extern "C" rp_status rp_scene_create(const rp_scene_desc *d, rp_scene **out) {
    if (!d || !out) return fail(RP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (rp_status s = need_device()) return s;
    if (!d->static_vertices || !d->static_triangles || !d->static_material || !d->dyn_vertices ||
        !d->dyn_triangles || !d->materials)
        return fail(RP_ERR_INVALID_ARG, "null array in scene description");
    if (d->n_static_triangles == 0 || d->n_dyn_triangles == 0 || d->n_materials == 0)
        return fail(RP_ERR_INVALID_ARG, "empty static geometry, dynamic object or material table");
    if (d->width == 0 || d->height == 0 || (uint64_t)d->width * d->height > (1u << 26))
        return fail(RP_ERR_INVALID_ARG, "image size out of range");
    if (d->max_depth < 2 || d->max_depth > (uint32_t)kMaxDepth)
        return fail(RP_ERR_INVALID_ARG, "max_depth must be in [2, 10]");
    if (d->n_static_triangles + (uint64_t)d->n_dyn_triangles >= (1u << 30))
        return fail(RP_ERR_INVALID_ARG, "too many triangles");
    for (uint32_t i = 0; i < 3 * d->n_static_triangles; ++i)
        if (d->static_triangles[i] >= d->n_static_vertices)
            return fail(RP_ERR_INVALID_ARG, "static triangle index out of range");
    for (uint32_t i = 0; i < d->n_static_triangles; ++i)
        if (d->static_material[i] >= d->n_materials)
            return fail(RP_ERR_INVALID_ARG, "static material index out of range");
    for (uint32_t i = 0; i < 3 * d->n_dyn_triangles; ++i)
        if (d->dyn_triangles[i] >= d->n_dyn_vertices)
            return fail(RP_ERR_INVALID_ARG, "dynamic triangle index out of range");
    for (uint32_t i = 0; i < d->n_materials; ++i)
        if (!material_ok(d->materials + 12 * i))
            return fail(RP_ERR_INVALID_ARG, "invalid material row");
    if (d->n_objects && !d->object_ranges) return fail(RP_ERR_INVALID_ARG, "null object_ranges");
    for (uint32_t k = 0; k < d->n_objects; ++k) {
        const uint64_t first = d->object_ranges[2 * k], count = d->object_ranges[2 * k + 1];
        if (count == 0 || first + count > d->n_static_triangles)
            return fail(RP_ERR_INVALID_ARG, "object range outside the static triangles");
        for (uint64_t i = first; i < first + count; ++i) {
            const float *m = d->materials + 12 * d->static_material[i];
            if (m[8] != 0.f || m[9] != 0.f || m[10] != 0.f)
                return fail(RP_ERR_UNSUPPORTED, "a movable object may not be emissive");
        }
    }

    const int ns = (int)d->n_static_triangles, nd = (int)d->n_dyn_triangles;
    rp_scene *sc = new rp_scene_s();
    DevScene &S = sc->S;
    auto keep = [&](void *p) { if (p) sc->allocs.push_back(p); };

    BuiltBVH bs = build_bvh(d->static_vertices, d->static_triangles, ns, 0);
    BuiltBVH bd = build_bvh(d->dyn_vertices, d->dyn_triangles, nd, ns);
    sc->bvh_depth_static = bs.depth;
    sc->bvh_depth_dyn = bd.depth;
    if (bs.depth >= kStackDepth || bd.depth >= kStackDepth) {
        delete sc;
        return fail(RP_ERR_UNSUPPORTED, "BVH deeper than the traversal stack");
    }
    // triangles by id: three vertices, and in their .w slots the unit normal
    // computed in double precision
    std::vector<float4> st(3 * (size_t)ns), dt(3 * (size_t)nd);
    auto fill = [](const float *verts, const uint32_t *tri, float4 *out) {
        const float *p[3] = {verts + 3 * tri[0], verts + 3 * tri[1], verts + 3 * tri[2]};
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)p[1][a] - p[0][a];
            e2[a] = (double)p[2][a] - p[0][a];
        }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int a = 0; a < 3; ++a) n[a] = l > 0.0 ? n[a] / l : 0.0;
        for (int k = 0; k < 3; ++k) out[k] = make_float4(p[k][0], p[k][1], p[k][2], (float)n[k]);
    };
    for (int i = 0; i < ns; ++i) fill(d->static_vertices, d->static_triangles + 3 * i, &st[3 * (size_t)i]);
    for (int i = 0; i < nd; ++i) fill(d->dyn_vertices, d->dyn_triangles + 3 * i, &dt[3 * (size_t)i]);
    auto area = [](const float4 *t) {
        double e1[3] = {(double)t[1].x - t[0].x, (double)t[1].y - t[0].y, (double)t[1].z - t[0].z};
        double e2[3] = {(double)t[2].x - t[0].x, (double)t[2].y - t[0].y, (double)t[2].z - t[0].z};
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        return 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    };
    // area CDFs: p(x_D) = 1 / A_dyn and p(x_L) = 1 / A_emit
    // thresholds on the 2^-24 grid of the uniforms: u = k / 2^24 < CDF_i
    // exactly when k < ceil(CDF_i * 2^24)
    auto threshold = [](double cdf) -> uint32_t {
        double t = std::ceil(cdf * 16777216.0);
        return t >= 16777216.0 ? 16777216u : (uint32_t)t;
    };
    std::vector<uint32_t> dcdf(nd);
    double acc = 0.0;
    std::vector<double> dacc(nd);
    for (int i = 0; i < nd; ++i) { acc += area(&dt[3 * (size_t)i]); dacc[i] = acc; }
    const double dyn_area = acc;
    for (int i = 0; i < nd; ++i) dcdf[i] = threshold(dacc[i] / dyn_area);
    dcdf[nd - 1] = 16777216u;
    std::vector<int> eids;
    std::vector<double> eacc;
    acc = 0.0;
    for (int i = 0; i < ns; ++i) {
        const float *m = d->materials + 12 * d->static_material[i];
        if (m[8] == 0.f && m[9] == 0.f && m[10] == 0.f) continue;
        acc += area(&st[3 * (size_t)i]);
        eids.push_back(i);
        eacc.push_back(acc);
    }
    if (eids.empty() || !(acc > 0.0) || !(dyn_area > 0.0)) {
        delete sc;
        return fail(RP_ERR_INVALID_ARG, "scene needs an emitter and a dynamic object of non-zero area");
    }
    std::vector<uint32_t> ecdf(eids.size());
    for (size_t i = 0; i < eids.size(); ++i) ecdf[i] = threshold(eacc[i] / acc);
    ecdf.back() = 16777216u;
    // (cos, sin) tables for angles 2 pi k / 2^24 by angle addition
    std::vector<double2> cs_hi(4096), cs_lo(4096);
    for (int i = 0; i < 4096; ++i) {
        const double two_pi = 6.283185307179586476925286766559;
        cs_hi[i] = make_double2(std::cos(two_pi * i / 4096.0), std::sin(two_pi * i / 4096.0));
        cs_lo[i] = make_double2(std::cos(two_pi * i / 16777216.0), std::sin(two_pi * i / 16777216.0));
    }

    std::vector<uint32_t> smat(d->static_material, d->static_material + ns);
    std::vector<float> mats(d->materials, d->materials + 12 * (size_t)d->n_materials);
    rp_status s = RP_OK;
    float4 *p4;
    float *pf;
    uint32_t *pu;
    int *pi;
#define UP(vec, ptr, dst)                         \
    if ((s = upload(vec, &ptr)) != RP_OK) {       \
        delete sc;                                \
        return s;                                 \
    }                                             \
    keep(ptr);                                    \
    dst = ptr;
    UP(bs.nodes, p4, S.stat.nodes);
    UP(bs.tris, p4, S.stat.tris);
    DevObject o0{};
    UP(bd.nodes, p4, o0.bvh.nodes);
    UP(bd.tris, p4, o0.bvh.tris);
    UP(st, p4, S.stat_tri);
    UP(dt, p4, o0.tri);
    UP(smat, pu, S.stat_mat);
    UP(mats, pf, S.mats);
    UP(dcdf, pu, o0.cdf);
    UP(ecdf, pu, S.emit_cdf);
    double2 *pd2;
    UP(cs_hi, pd2, S.cs_hi);
    UP(cs_lo, pd2, S.cs_lo);
    UP(eids, pi, S.emit_ids);
#undef UP
    S.stat.n_nodes = (int)(bs.nodes.size() / 4);
    S.stat.n_tris = ns;
    o0.bvh.n_nodes = (int)(bd.nodes.size() / 4);
    o0.bvh.n_tris = nd;
    S.n_static = ns;
    S.n_emit = (int)eids.size();
    S.n_mats = (int)d->n_materials;
    S.emit_area = (float)acc;
    {
        o0.n = nd;
        o0.area = (float)dyn_area;
        o0.bs = bounding_sphere(dt);
        sc->objects.push_back(o0);
        std::vector<double> ta(nd);
        for (int i = 0; i < nd; ++i) ta[i] = area(&dt[3 * (size_t)i]);
        sc->obj_tri_area.push_back(std::move(ta));
        sc->obj_area.push_back(dyn_area);
    }
    // movable objects: a BVH in object space (their given coordinates), the
    // triangles by id and the area sampling table, as for the dynamic mesh
    for (uint32_t k = 0; k < d->n_objects; ++k) {
        const int first = (int)d->object_ranges[2 * k], count = (int)d->object_ranges[2 * k + 1];
        const uint32_t *tri = d->static_triangles + 3 * (size_t)first;
        BuiltBVH bo = build_bvh(d->static_vertices, tri, count, ns);
        if (bo.depth >= kStackDepth) {
            delete sc;
            return fail(RP_ERR_UNSUPPORTED, "BVH deeper than the traversal stack");
        }
        std::vector<float4> ot(3 * (size_t)count);
        for (int i = 0; i < count; ++i) fill(d->static_vertices, tri + 3 * i, &ot[3 * (size_t)i]);
        std::vector<double> oacc(count);
        double oa = 0.0;
        for (int i = 0; i < count; ++i) { oa += area(&ot[3 * (size_t)i]); oacc[i] = oa; }
        if (!(oa > 0.0)) {
            delete sc;
            return fail(RP_ERR_INVALID_ARG, "movable object of zero area");
        }
        std::vector<uint32_t> ocdf(count);
        for (int i = 0; i < count; ++i) ocdf[i] = threshold(oacc[i] / oa);
        ocdf[count - 1] = 16777216u;
        DevObject o{};
        float4 *q4;
        uint32_t *qu;
        if ((s = upload(bo.nodes, &q4)) != RP_OK) { delete sc; return s; }
        keep(q4); o.bvh.nodes = q4;
        if ((s = upload(bo.tris, &q4)) != RP_OK) { delete sc; return s; }
        keep(q4); o.bvh.tris = q4;
        if ((s = upload(ot, &q4)) != RP_OK) { delete sc; return s; }
        keep(q4); o.tri = q4;
        if ((s = upload(ocdf, &qu)) != RP_OK) { delete sc; return s; }
        keep(qu); o.cdf = qu;
        o.bvh.n_nodes = (int)(bo.nodes.size() / 4);
        o.bvh.n_tris = count;
        o.n = count;
        o.area = (float)oa;
        o.bs = bounding_sphere(ot);
        o.skip_lo = first;
        o.skip_n = count;
        sc->objects.push_back(o);
        std::vector<double> ta(count);
        for (int i = 0; i < count; ++i) ta[i] = area(&ot[3 * (size_t)i]);
        sc->obj_tri_area.push_back(std::move(ta));
        sc->obj_area.push_back(oa);
    }
    // camera basis in double, stored as float
    const float *c = d->camera;
    double pos[3] = {c[0], c[1], c[2]}, look[3] = {c[3], c[4], c[5]}, up[3] = {c[6], c[7], c[8]};
    double f[3] = {look[0] - pos[0], look[1] - pos[1], look[2] - pos[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double &v : f) v /= fl;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(fl > 0.0) || !(rl > 0.0) || !(c[9] > 0.f && c[9] < 180.f)) {
        delete sc;
        return fail(RP_ERR_INVALID_ARG, "degenerate camera");
    }
    for (double &v : r) v /= rl;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    S.cam_pos = make_float3((float)pos[0], (float)pos[1], (float)pos[2]);
    S.cam_fwd = make_float3((float)f[0], (float)f[1], (float)f[2]);
    S.cam_right = make_float3((float)r[0], (float)r[1], (float)r[2]);
    S.cam_up = make_float3((float)u[0], (float)u[1], (float)u[2]);
    double hh = std::tan(0.5 * (double)c[9] * 3.14159265358979323846 / 180.0);
    sc->cam_hh = hh;
    double hw = hh * d->width / d->height;
    S.hh = (float)hh;
    S.hw = (float)hw;
    S.pix_area = (float)((2.0 * hw / d->width) * (2.0 * hh / d->height));
    S.film_area = (float)(4.0 * hw * hh);
    S.W = (int)d->width;
    S.H = (int)d->height;
    S.max_depth = (int)d->max_depth;
    S.alpha_min = d->alpha_min;
    S.d_min = d->d_min;
    S.jac_max = d->jacobian_max;
    S.eps = 1e-5f;
    cudaError_t e = cudaMalloc((void **)&sc->d_stats, sizeof(unsigned long long) * ST_COUNT);
    if (e != cudaSuccess) {
        delete sc;
        return cuda_fail(e, "cudaMalloc stats");
    }
    cudaMemset(sc->d_stats, 0, sizeof(unsigned long long) * ST_COUNT);
    *out = sc;
    return RP_OK;
}

extern "C" void rp_scene_destroy(rp_scene *scene) { delete scene; }

static void invert_rigid(const float *M, float *Mi) {
    // inverse of [R | t] is [R^T | -R^T t], in double
    double R[9], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[3 * i + j] = M[4 * i + j];
        t[i] = M[4 * i + 3];
    }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) {
            Mi[4 * i + j] = (float)R[3 * j + i];
            acc += R[3 * j + i] * t[j];
        }
        Mi[4 * i + 3] = (float)(-acc);
    }
}

static bool rigid(const float *M) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(M[i])) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += (double)M[4 * i + k] * M[4 * j + k];
            if (std::fabs(acc - (i == j ? 1.0 : 0.0)) > 1e-4) return false;
        }
    double det = (double)M[0] * (M[5] * M[10] - M[6] * M[9]) -
                 (double)M[1] * (M[4] * M[10] - M[6] * M[8]) +
                 (double)M[2] * (M[4] * M[9] - M[5] * M[8]);
    return det > 0.0;
}

// device tables of an edit of several objects (uploaded by rp_edit_multi)
struct EditTables {
    std::vector<uint32_t> cdf;        // area CDF thresholds over all objects' triangles
    std::vector<uint32_t> skip_bits;  // static triangles of the moved base poses
};

// an edit of n objects (1 <= n <= kMaxInst); `tab` receives the tables that
// several objects need (none for one object)
static rp_status fill_edit_multi(const rp_scene *sc, const rp_edit_desc *d, uint32_t n, DevEdit &E,
                                 EditTables *tab) {
    if (n < 1 || n > (uint32_t)kMaxInst)
        return fail(RP_ERR_INVALID_ARG, "an edit moves between 1 and 8 objects");
    std::memset(&E, 0, sizeof E);
    E.n_inst = (int)n;
    int lo = 0x7fffffff, hi = 0, covered = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const rp_edit_desc *e = d + k;
        if (e->object >= sc->objects.size())
            return fail(RP_ERR_INVALID_ARG, "edit object index out of range");
        for (uint32_t j = 0; j < k; ++j)
            if (d[j].object == e->object) return fail(RP_ERR_INVALID_ARG, "an object is edited twice");
        if (!rigid(e->M1) || !rigid(e->M2))
            return fail(RP_ERR_UNSUPPORTED, "edit transforms must be rigid (rotation + translation)");
        if (!material_ok(e->mat1) || !material_ok(e->mat2))
            return fail(RP_ERR_INVALID_ARG, "invalid edit material");
        for (int i = 8; i < 11; ++i)
            if (e->mat1[i] != 0.f || e->mat2[i] != 0.f)
                return fail(RP_ERR_UNSUPPORTED, "the edited object may not be emissive");
        std::memcpy(E.M_[k][0], e->M1, sizeof(float) * 12);
        std::memcpy(E.M_[k][1], e->M2, sizeof(float) * 12);
        invert_rigid(e->M1, E.Minv_[k][0]);
        invert_rigid(e->M2, E.Minv_[k][1]);
        std::memcpy(E.mat_[k][0], e->mat1, sizeof(float) * 12);
        std::memcpy(E.mat_[k][1], e->mat2, sizeof(float) * 12);
        if (std::memcmp(e->M1, e->M2, sizeof(float) * 12) != 0) E.motion = 1;
        E.object[k] = (int)e->object;
        const DevObject &o = sc->objects[e->object];
        if (o.skip_n > 0) {
            lo = std::min(lo, o.skip_lo);
            hi = std::max(hi, o.skip_lo + o.skip_n);
            covered += o.skip_n;
        }
    }
    if (hi > 0) {
        E.skip_lo = lo;
        E.skip_n = hi - lo;
        if (covered != hi - lo) {     // the base poses are not one contiguous range
            if (!tab) return fail(RP_ERR_INVALID_ARG, "several-object edits need rp_edit_multi");
            tab->skip_bits.assign(((size_t)(hi - lo) + 31) / 32, 0u);
            for (uint32_t k = 0; k < n; ++k) {
                const DevObject &o = sc->objects[d[k].object];
                for (int i = o.skip_lo - lo; i < o.skip_lo - lo + o.skip_n && o.skip_n > 0; ++i)
                    tab->skip_bits[(size_t)i >> 5] |= 1u << (i & 31);
            }
        }
    }
    if (n > 1) {
        if (!tab) return fail(RP_ERR_INVALID_ARG, "several-object edits need rp_edit_multi");
        // p(x_D) = 1 / (total area): thresholds of the CDF over the objects'
        // triangles in edit order, as for one object
        double tot = 0.0;
        for (uint32_t k = 0; k < n; ++k) tot += sc->obj_area[d[k].object];
        double acc = 0.0;
        for (uint32_t k = 0; k < n; ++k)
            for (double a : sc->obj_tri_area[d[k].object]) {
                acc += a;
                const double t = std::ceil(acc / tot * 16777216.0);
                tab->cdf.push_back(t >= 16777216.0 ? 16777216u : (uint32_t)t);
            }
        tab->cdf.back() = 16777216u;
    }
    return RP_OK;
}

static rp_status fill_edit(const rp_scene *sc, const rp_edit_desc *d, DevEdit &E) {
    return fill_edit_multi(sc, d, 1, E, nullptr);
}

// the scene as seen by an edit: its objects as the dynamic set, their
// dynamic triangle ids in edit order
static DevScene scene_for_edit(const rp_scene *sc, const DevEdit &E) {
    DevScene S = sc->S;
    S.n_inst = E.n_inst;
    int base = 0;
    double area = 0.0;
    for (int k = 0; k < E.n_inst; ++k) {
        const DevObject &o = sc->objects[E.object[k]];
        S.inst[k] = DevInst{o.bvh, o.tri, base, o.n, o.bs};
        base += o.n;
        area += sc->obj_area[E.object[k]];
    }
    S.n_dyn = base;
    S.dyn_area = E.n_inst == 1 ? sc->objects[E.object[0]].area : (float)area;
    S.dyn_cdf = E.n_inst == 1 ? sc->objects[E.object[0]].cdf : E.cdf;
    return S;
}

// the camera for an image of W x H pixels (same position, basis and
// vertical field of view)
static void set_resolution(const rp_scene *sc, DevScene &S, int W, int H) {
    const double hh = sc->cam_hh, hw = hh * W / H;
    S.hh = (float)hh;
    S.hw = (float)hw;
    S.pix_area = (float)((2.0 * hw / W) * (2.0 * hh / H));
    S.film_area = (float)(4.0 * hw * hh);
    S.W = W;
    S.H = H;
}

extern "C" rp_status rp_edit(rp_scene *scene, const rp_edit_desc *desc, rp_edit_handle **out) {
    return rp_edit_multi(scene, desc, 1, out);
}

extern "C" rp_status rp_edit_multi(rp_scene *scene, const rp_edit_desc *descs, uint32_t n,
                                   rp_edit_handle **out) {
    if (!scene || !descs || !out) return fail(RP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    rp_edit_handle *e = new rp_edit_s();
    EditTables tab;
    rp_status s = fill_edit_multi(scene, descs, n, e->E, &tab);
    if (s != RP_OK) {
        delete e;
        return s;
    }
    auto up = [&](const std::vector<uint32_t> &v, const uint32_t **dst) -> rp_status {
        if (v.empty()) return RP_OK;
        void *p = nullptr;
        cudaError_t ce = cudaMalloc(&p, v.size() * sizeof(uint32_t));
        if (ce == cudaErrorMemoryAllocation) return fail(RP_ERR_OOM, "edit table allocation failed");
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMalloc edit table");
        e->allocs.push_back(p);
        ce = cudaMemcpy(p, v.data(), v.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) return cuda_fail(ce, "upload edit table");
        *dst = (const uint32_t *)p;
        return RP_OK;
    };
    if ((s = up(tab.cdf, &e->E.cdf)) != RP_OK || (s = up(tab.skip_bits, &e->E.skip_bits)) != RP_OK) {
        delete e;
        return s;
    }
    *out = e;
    return RP_OK;
}

extern "C" void rp_edit_destroy(rp_edit_handle *edit) { delete edit; }

static LaunchArgs base_args(rp_scene *sc, const DevEdit &E, uint32_t spp, uint64_t seed,
                            uint32_t mask) {
    LaunchArgs a{};
    a.S = scene_for_edit(sc, E);
    a.E = E;
    a.seed = seed;
    a.invN = (float)(1.0 / ((double)spp * sc->S.W * sc->S.H));
    a.tech_mask = (int)mask;
    a.stats = sc->stats_on ? sc->d_stats : nullptr;
    a.residual = 1;
    a.map_mode = sc->map_mode;
    a.timer = sc->timing_on ? &sc->timer : nullptr;
    if (rp_guide *gd = sc->guide) {
        a.G.on = 1;
        a.G.use_net = gd->has_int ? 1 : 0;
        a.G.net.Wq = gd->Wq;
        for (int l = 0; l < 4; ++l) a.G.net.hid_scale[l] = std::ldexp(1.0f, -gd->shift[l]);
        a.G.net.out_scale = std::ldexp(1.0f, -gd->out_exp);
        for (int i = 0; i < 6; ++i) a.G.net.box[i] = gd->box[i];
        a.G.smp = gd->smp;
        a.G.half = gd->cap / 2;
        a.G.err = gd->err;
        a.G.gin = sc->gin;
        a.G.gout = sc->gout;
        a.G.gratio = sc->gratio;
    }
    return a;
}

static rp_status check_render(rp_scene *sc, uint32_t spp, uint32_t mask) {
    if (!sc) return fail(RP_ERR_INVALID_ARG, "null scene");
    if (spp == 0) return fail(RP_ERR_INVALID_ARG, "spp must be positive");
    if ((uint64_t)spp * sc->S.W * sc->S.H > 0xffffffffull)
        return fail(RP_ERR_INVALID_ARG, "spp * width * height must fit in 32 bits");
    if (mask == 0 || (mask & ~RP_TECH_SEVEN)) return fail(RP_ERR_INVALID_ARG, "bad technique mask");
    return RP_OK;
}

// wavefront buffers for waves of up to R roots; `tasks` adds the mapping
// task queue needed by edits with motion
// the learned proposal's per-root buffers (features, outputs, p_cos / q)
// for waves of up to R roots
static rp_status ensure_guide_buffers(rp_scene *sc, uint32_t R_need) {
    if (!sc->guide || sc->guide_R >= R_need) return RP_OK;
    sc->free_guide_buffers();
    const size_t R = R_need;
    cudaError_t e = cudaMalloc((void **)&sc->gin, R * kGIn);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sc->gout, R * kGOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sc->gratio, R * sizeof(float));
    if (e != cudaSuccess) {
        sc->free_guide_buffers();
        return e == cudaErrorMemoryAllocation ? fail(RP_ERR_OOM, "guide buffer allocation failed")
                                              : cuda_fail(e, "cudaMalloc guide buffers");
    }
    sc->guide_R = R_need;
    return RP_OK;
}

// wavefront buffers for waves of up to R roots of paths with at most D
// edges; `tasks` adds the mapping task queue needed by edits with motion
static rp_status alloc_wavebuf(WaveBuf &W, std::vector<void *> &allocs, uint32_t R, int D, bool tasks) {
    W = WaveBuf{};
    W.R = R;
    W.S = slot_count(D);
    W.qc = 2 * R;
    W.qa = 3 * R;
    const int t3 = (D - 3) * (D - 2) / 2;
    W.qt = tasks ? (uint32_t)std::min<uint64_t>((uint64_t)R * (uint64_t)std::max(D + 1, t3),
                                                 0x7ffffffeull)
                 : 0u;
    W.qv = tasks ? std::max(W.qa, W.qt) : 0u;
    auto free_all = [&]() {
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        W = WaveBuf{};
    };
    auto alloc = [&](void **p, size_t bytes) -> rp_status {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation) return fail(RP_ERR_OOM, "wavefront buffer allocation failed");
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc wavefront");
        allocs.push_back(*p);
        return RP_OK;
    };
    const size_t SR = (size_t)W.S * R;
#define A_(ptr, bytes) if (rp_status s_ = alloc((void **)&(ptr), (bytes))) { free_all(); return s_; }
    A_(W.px, SR * 4) A_(W.py, SR * 4) A_(W.pz, SR * 4) A_(W.nx, SR * 4) A_(W.ny, SR * 4)
    A_(W.nz, SR * 4) A_(W.b1, SR * 4) A_(W.b2, SR * 4) A_(W.prim, SR * 4)
    A_(W.len_eye, R * 4ull) A_(W.len_light, R * 4ull) A_(W.flags, R * 4ull)
    A_(W.cam_ok, R * 4ull) A_(W.nee_ok, R * 4ull) A_(W.ghost_w, R * 4ull) A_(W.ghost_n, R * 4ull)
    for (int b = 0; b < 2; ++b) {
        A_(W.c_o[b], W.qc * 12ull) A_(W.c_d[b], W.qc * 12ull) A_(W.c_ex[b], W.qc * 4ull)
        A_(W.c_tag[b], W.qc * 4ull)
    }
    A_(W.h_prim, W.qc * 4ull) A_(W.h_b1, W.qc * 4ull) A_(W.h_b2, W.qc * 4ull)
    A_(W.h_p, W.qc * 12ull)
    A_(W.a_o, W.qa * 12ull) A_(W.a_d, W.qa * 12ull) A_(W.a_tmax, W.qa * 4ull)
    A_(W.a_ex0, W.qa * 4ull) A_(W.a_ex1, W.qa * 4ull) A_(W.a_tag, W.qa * 4ull)
    if (tasks) {
        A_(W.tasks, W.qt * 16ull)
        A_(W.v_o, W.qv * 12ull) A_(W.v_d, W.qv * 12ull) A_(W.v_tmax, W.qv * 4ull)
        A_(W.v_ex0, W.qv * 4ull) A_(W.v_ex1, W.qv * 4ull) A_(W.v_task, W.qv * 4ull)
        A_(W.m_pix, W.qt * 8ull) A_(W.m_val, W.qt * 36ull) A_(W.m_w, W.qt * 12ull)
        A_(W.m_vis, W.qt * 4ull) A_(W.pend, W.qt * 4ull)
        // wavefront mapping: state per task, a pool of replayed vertices
        // (tasks that find it full map in one thread), replay queues
        W.yc = (uint32_t)std::min<uint64_t>((uint64_t)R * 12u, 0x7ffffffeull);
        W.qr = (uint32_t)std::min<uint64_t>((uint64_t)R * 4u, W.qt);
        A_(W.ms_info, W.qt * 4ull) A_(W.ms_J, W.qt * 4ull) A_(W.ms_base, W.qt * 4ull)
        A_(W.fin, W.qt * 4ull)
        A_(W.y_p, W.yc * 12ull) A_(W.y_n, W.yc * 12ull) A_(W.y_b, W.yc * 8ull)
        A_(W.y_prim, W.yc * 4ull)
        for (int b = 0; b < 2; ++b) {
            A_(W.r_o[b], W.qr * 12ull) A_(W.r_d[b], W.qr * 12ull) A_(W.r_ex[b], W.qr * 4ull)
            A_(W.r_task[b], W.qr * 4ull)
        }
        A_(W.rh_prim, W.qr * 4ull) A_(W.rh_b1, W.qr * 4ull) A_(W.rh_b2, W.qr * 4ull)
        A_(W.rh_p, W.qr * 12ull)
    }
    A_(W.counts, kCountSlots * 4ull)
#undef A_
    return RP_OK;
}

static rp_status ensure_wave(rp_scene *sc, uint32_t R, bool tasks) {
    const int D = sc->S.max_depth;
    if (sc->W.R >= R && (!tasks || sc->wave_tasks)) return ensure_guide_buffers(sc, sc->W.R);
    R = std::max(R, sc->W.R);
    tasks = tasks || sc->wave_tasks;
    sc->free_wave();
    if (rp_status s = alloc_wavebuf(sc->W, sc->wave_allocs, R, D, tasks)) return s;
    sc->wave_tasks = tasks;
    return ensure_guide_buffers(sc, sc->W.R);
}

// run roots [r0, r1) of technique `tech` (0: primal) in frame a.frame as waves
static rp_status run_waves(rp_scene *sc, LaunchArgs a, int tech, uint32_t r0, uint32_t r1,
                           cudaStream_t st) {
    const bool tasks = a.residual && a.E.motion;
    const uint32_t n = r1 - r0;
    if (n == 0) return RP_OK;
    if (rp_status s = ensure_wave(sc, std::min(n, sc->wave_cap), tasks)) return s;
    a.W = sc->W;
    a.G.gin = sc->gin;
    a.G.gout = sc->gout;
    a.G.gratio = sc->gratio;
    for (uint32_t b = r0; b < r1; b += sc->W.R) {
        a.root_begin = b;
        a.root_end = std::min(r1, b + sc->W.R);
        RP_CUDA(launch_wave(tech, a, st), "wavefront launch");
    }
    return RP_OK;
}

// the learned proposal encodes x_D in the one edited object's space
static rp_status guide_fits(const rp_scene *sc, const DevEdit &E) {
    if (sc->guide && E.n_inst > 1)
        return fail(RP_ERR_UNSUPPORTED, "the learned proposal needs an edit of one object");
    return RP_OK;
}

// A render of at most kLaneRoots roots per technique and frame is one wave
// per technique and frame, too small to fill the GPU alone: its waves run on
// kLanes streams at once, each stream with wave buffers of its own, forked
// from and joined back into the caller's stream.  The waves are independent
// (their own counters and queues), so the image is the sum of the same
// samples as in sequence.
#ifndef RP_LANES
#define RP_LANES 4
#endif
constexpr uint32_t kLaneRoots = 1u << 20;
constexpr int kLanes = RP_LANES;

static rp_status render_lanes(rp_scene *sc, LaunchArgs a, uint32_t N, uint32_t mask, cudaStream_t st) {
    const bool tasks = a.residual && a.E.motion;
    if (sc->lanes.empty()) {
        sc->lanes.resize(kLanes);
        for (rp_scene::Lane &l : sc->lanes)
            if (cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess)
                return fail(RP_ERR_CUDA, "stream creation failed");
        if (cudaEventCreateWithFlags(&sc->lanes_fork, cudaEventDisableTiming) != cudaSuccess)
            return fail(RP_ERR_CUDA, "event creation failed");
    }
    const int D = sc->S.max_depth;
    for (rp_scene::Lane &l : sc->lanes) {
        if (l.W.R >= N && (!tasks || l.tasks)) continue;
        // a lane's buffers are only reallocated once its stream is idle
        RP_CUDA(cudaStreamSynchronize(l.s), "lane sync");
        for (void *p : l.allocs) cudaFree(p);
        l.allocs.clear();
        l.tasks = tasks || l.tasks;
        if (rp_status s = alloc_wavebuf(l.W, l.allocs, std::max(N, l.W.R), D, l.tasks)) return s;
    }
    // with the learned proposal, technique (3)'s two waves share the scene's
    // guide buffers, so they run one after the other on one lane
    const bool guided = sc->guide && (mask & RP_TECH_DYNAMIC_TWO_ENDS);
    if (guided) {
        if (rp_status s = ensure_guide_buffers(sc, N)) return s;
        a.G.gin = sc->gin;
        a.G.gout = sc->gout;
        a.G.gratio = sc->gratio;
    }
    RP_CUDA(cudaEventRecord(sc->lanes_fork, st), "fork");
    for (rp_scene::Lane &l : sc->lanes) RP_CUDA(cudaStreamWaitEvent(l.s, sc->lanes_fork, 0), "fork");
    const int techs[7] = {1, 2, 3, 7, 4, 5, 6};
    int k = 0, t3_lane = -1;
    a.root_begin = 0;
    a.root_end = N;
    for (int t = 0; t < 7; ++t)
        for (int g = 1; g <= 2; ++g) {
            if (!(mask & (1u << t)) || (t >= 4 && !a.E.motion)) continue;
            int li = k++ % kLanes;
            if (guided && techs[t] == 3) {
                if (t3_lane < 0) t3_lane = li;
                li = t3_lane;
            }
            rp_scene::Lane &l = sc->lanes[li];
            a.frame = g;
            a.W = l.W;
            RP_CUDA(launch_wave(techs[t], a, l.s), "wavefront launch");
        }
    for (rp_scene::Lane &l : sc->lanes) {
        RP_CUDA(cudaEventRecord(l.done, l.s), "join");
        RP_CUDA(cudaStreamWaitEvent(st, l.done, 0), "join");
    }
    return RP_OK;
}

static rp_status render_into(rp_scene *sc, const DevEdit &E, uint32_t spp, uint64_t seed,
                             uint32_t mask, double *d_out, cudaStream_t st) {
    if (rp_status s = guide_fits(sc, E)) return s;
    LaunchArgs a = base_args(sc, E, spp, seed, mask);
    a.img = d_out;
    a.residual = 1;
    const uint32_t N = spp * (uint32_t)(sc->S.W * sc->S.H);
    if (sc->stats_on)
        RP_CUDA(cudaMemsetAsync(sc->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, st), "memset");
    if (sc->guide && (mask & RP_TECH_DYNAMIC_TWO_ENDS))
        RP_CUDA(cudaMemsetAsync(sc->guide->smp.wt, 0, sizeof(float) * sc->guide->cap, st),
                "memset guide weights");
    // mask bits 0..6: techniques (1), (2), (3), path tracing, (4), (5), (6);
    // the ghost techniques need motion (without it there is no ghost)
    const int techs[7] = {1, 2, 3, 7, 4, 5, 6};
    int jobs = 0;
    for (int t = 0; t < 7; ++t)
        if ((mask & (1u << t)) && !(t >= 4 && !E.motion)) jobs += 2;
    if (N <= kLaneRoots && jobs >= 2) {
        if (rp_status s = render_lanes(sc, a, N, mask, st)) return s;
        sc->last_stream = st;
        return RP_OK;
    }
    for (int g = 1; g <= 2; ++g)
        for (int t = 0; t < 7; ++t) {
            if (!(mask & (1u << t)) || (t >= 4 && !E.motion)) continue;
            a.frame = g;
            if (rp_status s = run_waves(sc, a, techs[t], 0, N, st)) return s;
        }
    sc->last_stream = st;
    return RP_OK;
}

// the same render with the one-thread-per-root kernels, which need no
// scratch memory besides the image
static rp_status render_into_direct(rp_scene *sc, const DevEdit &E, uint32_t spp, uint64_t seed,
                                    uint32_t mask, double *d_out, cudaStream_t st) {
    if (mask & RP_TECH_GHOSTS)
        return fail(RP_ERR_UNSUPPORTED, "the one-thread-per-root kernels have no ghost techniques");
    LaunchArgs a = base_args(sc, E, spp, seed, mask);
    a.G = GuideLaunch{};           // the one-thread-per-root kernels run without the proposal
    a.img = d_out;
    a.root_begin = 0;
    a.root_end = spp * (uint32_t)(sc->S.W * sc->S.H);
    if (sc->stats_on)
        RP_CUDA(cudaMemsetAsync(sc->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, st), "memset");
    const int techs[4] = {1, 2, 3, 7};
    for (int g = 1; g <= 2; ++g)
        for (int t = 0; t < 4; ++t) {
            if (!(mask & (1u << t))) continue;
            a.frame = g;
            RP_CUDA(launch_residual(techs[t], a, st), "residual launch");
        }
    sc->last_stream = st;
    return RP_OK;
}

extern "C" rp_status rp_render_residual(rp_scene *scene, const rp_edit_handle *edit, uint32_t spp,
                                        uint64_t seed, uint32_t tech_mask, double *d_out,
                                        void *stream) {
    if (rp_status s = check_render(scene, spp, tech_mask)) return s;
    if (!edit || !d_out) return fail(RP_ERR_INVALID_ARG, "null edit or image");
    return render_into(scene, edit->E, spp, seed, tech_mask, d_out, (cudaStream_t)stream);
}

static rp_status ensure_scratch(rp_scene *sc) {
    if (sc->d_scratch) return RP_OK;
    size_t n = (size_t)sc->S.W * sc->S.H * 3;
    cudaError_t e = cudaMalloc((void **)&sc->d_scratch, n * sizeof(double));
    if (e == cudaErrorMemoryAllocation) return fail(RP_ERR_OOM, "scratch image allocation failed");
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc scratch");
    return RP_OK;
}

extern "C" rp_status rp_render_residual_f32(rp_scene *scene, const rp_edit_handle *edit,
                                            uint32_t spp, uint64_t seed, uint32_t tech_mask,
                                            float *d_out, void *stream) {
    if (rp_status s = check_render(scene, spp, tech_mask)) return s;
    if (!edit || !d_out) return fail(RP_ERR_INVALID_ARG, "null edit or image");
    if (rp_status s = ensure_scratch(scene)) return s;
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)scene->S.W * scene->S.H * 3;
    RP_CUDA(cudaMemsetAsync(scene->d_scratch, 0, n * sizeof(double), st), "memset scratch");
    if (rp_status s = render_into(scene, edit->E, spp, seed, tech_mask, scene->d_scratch, st))
        return s;
    RP_CUDA(launch_add_f64_to_f32(scene->d_scratch, d_out, n, st), "resolve launch");
    return RP_OK;
}

extern "C" rp_status rp_render_residual_host(rp_scene *scene, const rp_edit_desc *edit,
                                             uint32_t spp, uint64_t seed, uint32_t tech_mask,
                                             double *host_out, void *stream) {
    if (rp_status s = check_render(scene, spp, tech_mask)) return s;
    if (!edit || !host_out) return fail(RP_ERR_INVALID_ARG, "null edit or image");
    DevEdit E;
    if (rp_status s = fill_edit(scene, edit, E)) return s;
    if (rp_status s = ensure_scratch(scene)) return s;
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)scene->S.W * scene->S.H * 3;
    RP_CUDA(cudaMemsetAsync(scene->d_scratch, 0, n * sizeof(double), st), "memset scratch");
    if (rp_status s = render_into(scene, E, spp, seed, tech_mask, scene->d_scratch, st)) return s;
    RP_CUDA(cudaMemcpyAsync(host_out, scene->d_scratch, n * sizeof(double), cudaMemcpyDeviceToHost,
                            st),
            "copy image to host");
    RP_CUDA(cudaStreamSynchronize(st), "render");
    return RP_OK;
}

extern "C" rp_status rp_render_primal(rp_scene *scene, const rp_edit_handle *edit, int frame,
                                      uint32_t spp, uint64_t seed, double *d_out, void *stream) {
    if (rp_status s = check_render(scene, spp, RP_TECH_ALL)) return s;
    if (!edit || !d_out) return fail(RP_ERR_INVALID_ARG, "null edit or image");
    if (frame != 1 && frame != 2) return fail(RP_ERR_INVALID_ARG, "frame must be 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    LaunchArgs a = base_args(scene, edit->E, spp, seed, RP_TECH_ALL);
    a.img = d_out;
    a.frame = frame;
    a.residual = 0;
    if (scene->stats_on)
        RP_CUDA(cudaMemsetAsync(scene->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, st),
                "memset");
    if (rp_status s = run_waves(scene, a, 0, 0, spp * (uint32_t)(scene->S.W * scene->S.H), st))
        return s;
    scene->last_stream = st;
    return RP_OK;
}

extern "C" rp_status rp_dump_samples(rp_scene *scene, const rp_edit_handle *edit, int tech,
                                     int frame, uint32_t spp, uint64_t seed, uint32_t root_begin,
                                     uint32_t root_end, uint32_t tech_mask, rp_record *d_records,
                                     uint64_t capacity, unsigned long long *d_count, void *stream) {
    if (rp_status s = check_render(scene, spp, tech_mask)) return s;
    if (!edit || !d_count || (!d_records && capacity)) return fail(RP_ERR_INVALID_ARG, "null buffer");
    if (tech < 1 || tech > 7)
        return fail(RP_ERR_INVALID_ARG, "tech must be in 1..7");
    if (frame != 1 && frame != 2) return fail(RP_ERR_INVALID_ARG, "frame must be 1 or 2");
    if (rp_status s = guide_fits(scene, edit->E)) return s;
    if (root_end < root_begin || root_end > spp * (uint32_t)(scene->S.W * scene->S.H))
        return fail(RP_ERR_INVALID_ARG, "root range out of bounds");
    static_assert(sizeof(rp_record) == sizeof(Record), "record layout");
    cudaStream_t st = (cudaStream_t)stream;
    RP_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st), "memset count");
    LaunchArgs a = base_args(scene, edit->E, spp, seed, tech_mask);
    a.frame = frame;
    a.residual = 1;
    a.rec = reinterpret_cast<Record *>(d_records);
    a.rec_cap = capacity;
    a.rec_count = d_count;
    return run_waves(scene, a, tech, root_begin, root_end, st);
}

extern "C" rp_status rp_trace_closest(rp_scene *scene, const rp_edit_handle *edit, int frame,
                                      uint32_t n, const float *d_origins, const float *d_dirs,
                                      float *d_t, int32_t *d_prim, float *d_b1, float *d_b2,
                                      void *stream) {
    if (!scene || !edit) return fail(RP_ERR_INVALID_ARG, "null scene or edit");
    if (frame != 1 && frame != 2) return fail(RP_ERR_INVALID_ARG, "frame must be 1 or 2");
    if (n && (!d_origins || !d_dirs || !d_t || !d_prim || !d_b1 || !d_b2))
        return fail(RP_ERR_INVALID_ARG, "null ray buffer");
    if (scene->stats_on)
        RP_CUDA(cudaMemsetAsync(scene->d_stats, 0, sizeof(unsigned long long) * ST_COUNT,
                                (cudaStream_t)stream), "memset");
    RP_CUDA(launch_trace(scene_for_edit(scene, edit->E), edit->E, frame, n, d_origins, d_dirs, d_t, d_prim, d_b1, d_b2,
                         scene->stats_on ? scene->d_stats : nullptr, (cudaStream_t)stream),
            "trace launch");
    return RP_OK;
}

extern "C" rp_status rp_bvh_build_host(const float *verts, uint32_t n_verts, const uint32_t *tris,
                                       uint32_t n_tris, float *nodes_out, uint32_t node_cap,
                                       float *tris_out, uint32_t *n_nodes, int *depth) {
    if (!verts || !tris || !n_nodes || !depth || n_tris == 0)
        return fail(RP_ERR_INVALID_ARG, "null argument or no triangles");
    if (n_tris > (1u << 30)) return fail(RP_ERR_INVALID_ARG, "too many triangles");
    for (uint64_t i = 0; i < 3ull * n_tris; ++i)
        if (tris[i] >= n_verts) return fail(RP_ERR_INVALID_ARG, "vertex index out of range");
    BuiltBVH b = build_bvh(verts, tris, (int)n_tris, 0);
    *n_nodes = (uint32_t)(b.nodes.size() / 4);
    *depth = b.depth;
    if (nodes_out) {
        if (node_cap < *n_nodes) return fail(RP_ERR_INVALID_ARG, "node buffer too small");
        std::memcpy(nodes_out, b.nodes.data(), b.nodes.size() * sizeof(float4));
    }
    if (tris_out) std::memcpy(tris_out, b.tris.data(), b.tris.size() * sizeof(float4));
    return RP_OK;
}

extern "C" rp_status rp_philox(uint32_t n, const uint32_t *d_counters, const uint32_t *d_keys,
                               uint32_t *d_out, void *stream) {
    if (rp_status s = need_device()) return s;
    if (n && (!d_counters || !d_keys || !d_out)) return fail(RP_ERR_INVALID_ARG, "null buffer");
    RP_CUDA(launch_philox(n, d_counters, d_keys, d_out, (cudaStream_t)stream), "philox launch");
    return RP_OK;
}

extern "C" rp_status rp_enable_stats(rp_scene *scene, int on) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    scene->stats_on = on != 0;
    return RP_OK;
}

extern "C" rp_status rp_sync_status(rp_scene *scene) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    RP_CUDA(cudaStreamSynchronize(scene->last_stream), "sync");
    RP_CUDA(cudaGetLastError(), "device status");
    return RP_OK;
}

extern "C" rp_status rp_get_stats(rp_scene *scene, rp_stats *out) {
    if (!scene || !out) return fail(RP_ERR_INVALID_ARG, "null argument");
    unsigned long long h[ST_COUNT];
    RP_CUDA(cudaStreamSynchronize(scene->last_stream), "sync");
    RP_CUDA(cudaMemcpy(h, scene->d_stats, sizeof h, cudaMemcpyDeviceToHost), "stats copy");
    out->roots = h[ST_ROOTS];
    out->paths = h[ST_PATHS];
    out->rays_closest = h[ST_RAYS_CLOSEST];
    out->rays_shadow = h[ST_RAYS_SHADOW];
    out->nodes_visited = h[ST_NODES];
    out->tris_tested = h[ST_TRIS];
    out->accepted = h[ST_ACCEPTED];
    out->rejected = h[ST_REJECTED];
    out->nodes_closest = h[ST_NODES_C];
    out->tris_closest = h[ST_TRIS_C];
    out->nodes_shadow = h[ST_NODES_S];
    out->tris_shadow = h[ST_TRIS_S];
    return RP_OK;
}

extern "C" rp_status rp_enable_timing(rp_scene *scene, int on) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    scene->timing_on = on != 0;
    scene->timer.only[0] = 0;
    return RP_OK;
}

extern "C" rp_status rp_enable_timing_of(rp_scene *scene, const char *kernel) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    if (kernel && std::strlen(kernel) >= sizeof scene->timer.only)
        return fail(RP_ERR_INVALID_ARG, "kernel name too long");
    scene->timing_on = true;
    if (kernel) std::strcpy(scene->timer.only, kernel);
    else scene->timer.only[0] = 0;
    return RP_OK;
}

extern "C" rp_status rp_get_kernel_times(rp_scene *scene, rp_kernel_time *out, int capacity,
                                         int *count) {
    if (!scene || !count || (capacity > 0 && !out)) return fail(RP_ERR_INVALID_ARG, "null argument");
    KernelTimer &t = scene->timer;
    RP_CUDA(cudaStreamSynchronize(scene->last_stream), "sync");
    std::vector<rp_kernel_time> agg;
    for (int i = 0; i < t.n; ++i) {
        float ms = 0.f;
        RP_CUDA(cudaEventElapsedTime(&ms, t.entries[i].start, t.entries[i].stop), "event time");
        size_t j = 0;
        while (j < agg.size() && std::strcmp(agg[j].name, t.entries[i].name) != 0) ++j;
        if (j == agg.size()) {
            rp_kernel_time k{};
            std::strncpy(k.name, t.entries[i].name, sizeof(k.name) - 1);
            agg.push_back(k);
        }
        agg[j].launches += 1;
        agg[j].ms += ms;
    }
    t.n = 0;
    t.pool_used = 0;
    *count = (int)agg.size();
    for (int i = 0; i < (int)agg.size() && i < capacity; ++i) out[i] = agg[i];
    return RP_OK;
}

// ---------------------------------------------------------------------------
// helpers for entry points defined in other translation units
// ---------------------------------------------------------------------------

namespace rp {

rp_status set_last_error(rp_status s, const char *msg) { return fail(s, msg); }

rp_status scene_image_size(const rp_scene *scene, int *w, int *h) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    *w = scene->S.W;
    *h = scene->S.H;
    return RP_OK;
}

// validated residual render into a caller-supplied FP64 image (no allocation)
rp_status render_residual_into(rp_scene *scene, const rp_edit_handle *edit, uint32_t spp,
                               uint64_t seed, uint32_t tech_mask, double *d_img,
                               cudaStream_t stream) {
    if (rp_status s = check_render(scene, spp, tech_mask)) return s;
    if (!edit || !d_img) return fail(RP_ERR_INVALID_ARG, "null edit or image");
    return render_into_direct(scene, edit->E, spp, seed, tech_mask, d_img, stream);
}

}  // namespace rp

// ---------------------------------------------------------------------------
// learned proposal of technique (3)
// ---------------------------------------------------------------------------

namespace {

// splitmix64 and Box-Muller: the seeded He initialisation of the float network
uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unit_open(uint64_t &s) { return ((double)(splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

rp_status guide_alloc(rp_guide *g, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) return fail(RP_ERR_OOM, "guide allocation failed");
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc guide");
    g->allocs.push_back(*p);
    return cudaMemset(*p, 0, bytes) == cudaSuccess ? RP_OK : fail(RP_ERR_CUDA, "memset guide");
}

rp_status upload_float_weights(rp_guide *g, const float *h) {
    RP_CUDA(cudaMemcpy(g->Wm, h, sizeof(float) * kGWeights, cudaMemcpyHostToDevice), "upload weights");
    RP_CUDA(cudaMemset(g->m, 0, sizeof(float) * kGWeights), "reset adam");
    RP_CUDA(cudaMemset(g->v, 0, sizeof(float) * kGWeights), "reset adam");
    RP_CUDA(launch_f32_to_bf16(g->Wm, g->Wbf, kGWeights, 0), "convert weights");
    RP_CUDA(cudaDeviceSynchronize(), "convert weights");
    g->adam_t = 0;
    return RP_OK;
}

rp_status upload_int_network(rp_guide *g, const int8_t *W, const int32_t *shift, int32_t out_exp) {
    for (int l = 0; l < 4; ++l)
        if (shift[l] < 0 || shift[l] > 24) return fail(RP_ERR_INVALID_ARG, "shift must be in [0, 24]");
    if (out_exp < -30 || out_exp > 60) return fail(RP_ERR_INVALID_ARG, "out_exp must be in [-30, 60]");
    std::vector<float> f(kGWeights);
    for (int i = 0; i < kGWeights; ++i) {
        if (W[i] < -127) return fail(RP_ERR_INVALID_ARG, "integer weights must be in [-127, 127]");
        f[i] = (float)W[i];
    }
    float *tmp = nullptr;
    RP_CUDA(cudaMalloc((void **)&tmp, sizeof(float) * kGWeights), "cudaMalloc");
    cudaError_t e = cudaMemcpy(tmp, f.data(), sizeof(float) * kGWeights, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_f32_to_bf16(tmp, g->Wq, kGWeights, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "upload integer network");
    for (int l = 0; l < 4; ++l) g->shift[l] = shift[l];
    g->out_exp = out_exp;
    g->has_int = true;
    return RP_OK;
}

// integer network from the float one: per layer the largest power-of-two
// weight scale with |W| 2^s <= 127, activation scales 2^t with the largest
// recorded activation <= 255 (2^7 for the inputs), requantisation shifts
// t_l + s_l - t_{l+1} (never negative)
rp_status quantize(rp_guide *g, const float *W, const float *amax) {
    std::vector<int8_t> q(kGWeights);
    int s[kGLayers], t[kGLayers];
    t[0] = 7;
    for (int l = 0; l < kGLayers; ++l) {
        float mx = 0.f;
        for (int i = guide_off(l); i < guide_off(l + 1); ++i) mx = std::max(mx, std::fabs(W[i]));
        s[l] = mx > 0.f ? (int)std::floor(std::log2(127.0 / mx)) : 0;
        s[l] = std::max(-20, std::min(30, s[l]));
        for (int i = guide_off(l); i < guide_off(l + 1); ++i) {
            double v = std::nearbyint(std::ldexp((double)W[i], s[l]));
            q[i] = (int8_t)std::max(-127.0, std::min(127.0, v));
        }
    }
    int32_t shift[4];
    for (int l = 0; l < 4; ++l) {
        int tn = amax[l] > 0.f ? (int)std::floor(std::log2(255.0 / amax[l])) : t[l] + s[l];
        int sh = t[l] + s[l] - tn;
        if (sh < 0) { sh = 0; tn = t[l] + s[l]; }
        if (sh > 24) { sh = 24; tn = t[l] + s[l] - 24; }
        shift[l] = sh;
        t[l + 1] = tn;
    }
    int32_t out_exp = std::max(-30, std::min(60, t[4] + s[4]));
    return upload_int_network(g, q.data(), shift, out_exp);
}

}  // namespace

extern "C" rp_status rp_guide_create(const float *box, uint32_t batch, uint64_t seed, rp_guide **out) {
    if (!box || !out) return fail(RP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (batch < 256 || (batch & 1u) || batch > (1u << 24))
        return fail(RP_ERR_INVALID_ARG, "batch must be even and in [256, 2^24]");
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(box[i])) return fail(RP_ERR_INVALID_ARG, "box must be finite");
    if (rp_status s = need_device()) return s;
    rp_guide *g = new rp_guide_s();
    for (int i = 0; i < 6; ++i) g->box[i] = box[i];
    g->cap = batch;
    const size_t C = batch;
    rp_status st = RP_OK;
#define GA_(ptr, bytes) if (st == RP_OK) st = guide_alloc(g, (void **)&(ptr), (bytes));
    GA_(g->Wm, sizeof(float) * kGWeights) GA_(g->m, sizeof(float) * kGWeights)
    GA_(g->v, sizeof(float) * kGWeights) GA_(g->grad, sizeof(float) * kGWeights)
    GA_(g->loss, sizeof(float)) GA_(g->wsum, sizeof(float)) GA_(g->d_box, sizeof(float) * 6)
    GA_(g->amax, sizeof(unsigned int) * 4) GA_(g->err, sizeof(int))
    GA_(g->Wbf, sizeof(__nv_bfloat16) * kGWeights) GA_(g->Wq, sizeof(__nv_bfloat16) * kGWeights)
    GA_(g->smp.p, sizeof(float) * 3 * C) GA_(g->smp.n, sizeof(float) * 3 * C)
    GA_(g->smp.w, sizeof(float) * 3 * C) GA_(g->smp.wt, sizeof(float) * C)
    GA_(g->X, sizeof(__nv_bfloat16) * kGIn * C) GA_(g->omega, sizeof(float) * 3 * C)
    GA_(g->wt, sizeof(float) * C)
#undef GA_
    g->smp.cap = batch;
    if (st == RP_OK && cudaMemcpy(g->d_box, box, sizeof(float) * 6, cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(RP_ERR_CUDA, "upload box");
    if (st == RP_OK) {
        std::vector<float> W(kGWeights);
        uint64_t rs = seed;
        for (int l = 0; l < kGLayers; ++l) {
            const double sd = std::sqrt(2.0 / guide_in(l));
            for (int i = guide_off(l); i < guide_off(l + 1); ++i) {
                const double a = unit_open(rs), b = unit_open(rs);
                W[i] = (float)(sd * std::sqrt(-2.0 * std::log(a)) * std::cos(6.283185307179586 * b));
            }
        }
        st = upload_float_weights(g, W.data());
    }
    if (st != RP_OK) {
        delete g;
        return st;
    }
    *out = g;
    return RP_OK;
}

extern "C" void rp_guide_destroy(rp_guide *guide) { delete guide; }

extern "C" rp_status rp_guide_set_weights(rp_guide *g, const float *W) {
    if (!g || !W) return fail(RP_ERR_INVALID_ARG, "null argument");
    for (int i = 0; i < kGWeights; ++i)
        if (!std::isfinite(W[i])) return fail(RP_ERR_INVALID_ARG, "weights must be finite");
    return upload_float_weights(g, W);
}

extern "C" rp_status rp_guide_get_weights(rp_guide *g, float *W) {
    if (!g || !W) return fail(RP_ERR_INVALID_ARG, "null argument");
    RP_CUDA(cudaDeviceSynchronize(), "sync");
    RP_CUDA(cudaMemcpy(W, g->Wm, sizeof(float) * kGWeights, cudaMemcpyDeviceToHost), "download");
    return RP_OK;
}

extern "C" rp_status rp_guide_set_int(rp_guide *g, const int8_t *W, const int32_t *shift,
                                      int32_t out_exp) {
    if (!g || !W || !shift) return fail(RP_ERR_INVALID_ARG, "null argument");
    return upload_int_network(g, W, shift, out_exp);
}

extern "C" rp_status rp_guide_get_int(rp_guide *g, int8_t *W, int32_t *shift, int32_t *out_exp) {
    if (!g || !W || !shift || !out_exp) return fail(RP_ERR_INVALID_ARG, "null argument");
    if (!g->has_int) return fail(RP_ERR_INVALID_ARG, "the guide has no integer network yet");
    std::vector<__nv_bfloat16> q(kGWeights);
    RP_CUDA(cudaDeviceSynchronize(), "sync");
    RP_CUDA(cudaMemcpy(q.data(), g->Wq, sizeof(__nv_bfloat16) * kGWeights, cudaMemcpyDeviceToHost),
            "download");
    for (int i = 0; i < kGWeights; ++i) W[i] = (int8_t)(int)__bfloat162float(q[i]);
    for (int l = 0; l < 4; ++l) shift[l] = g->shift[l];
    *out_exp = g->out_exp;
    return RP_OK;
}

extern "C" rp_status rp_guide_infer(rp_guide *g, const int8_t *d_in, uint32_t n, float *d_out,
                                    void *stream) {
    if (!g || (n && (!d_in || !d_out))) return fail(RP_ERR_INVALID_ARG, "null argument");
    if (!g->has_int) return fail(RP_ERR_INVALID_ARG, "the guide has no integer network yet");
    GuideNet net{};
    net.Wq = g->Wq;
    for (int l = 0; l < 4; ++l) net.hid_scale[l] = std::ldexp(1.0f, -g->shift[l]);
    net.out_scale = std::ldexp(1.0f, -g->out_exp);
    for (int i = 0; i < 6; ++i) net.box[i] = g->box[i];
    RP_CUDA(launch_guide_infer(net, d_in, n, d_out, g->err, (cudaStream_t)stream), "guide inference");
    return RP_OK;
}

extern "C" rp_status rp_guide_encode(rp_guide *g, const double *d_p, const float *d_n, uint32_t n,
                                    int8_t *d_out, void *stream) {
    if (!g || (n && (!d_p || !d_n || !d_out))) return fail(RP_ERR_INVALID_ARG, "null argument");
    RP_CUDA(launch_guide_encode(g->box, d_p, d_n, n, d_out, (cudaStream_t)stream), "guide encoding");
    return RP_OK;
}

extern "C" rp_status rp_guide_loss_grad(rp_guide *g, const float *d_x, const float *d_omega,
                                        const float *d_wt, uint32_t n, float *d_grad, float *d_loss,
                                        void *stream) {
    if (!g || !d_grad || !d_loss || (n && (!d_x || !d_omega || !d_wt)))
        return fail(RP_ERR_INVALID_ARG, "null argument");
    if (n == 0) return RP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->xs_rows < n) {
        if (g->Xs) cudaFree(g->Xs);
        g->Xs = nullptr;
        g->xs_rows = 0;
        cudaError_t e = cudaMalloc((void **)&g->Xs, sizeof(__nv_bfloat16) * kGIn * (size_t)n);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc features");
        g->xs_rows = n;
    }
    RP_CUDA(launch_f32_to_bf16(d_x, g->Xs, (size_t)kGIn * n, st), "convert features");
    GuideTrain T{};
    T.W = g->Wbf;
    T.X = g->Xs;
    T.omega = d_omega;
    T.wt = d_wt;
    T.n = n;
    T.inv_n = 1.0f / (float)n;
    T.wsum = nullptr;
    T.grad = d_grad;
    T.loss = d_loss;
    T.amax = g->amax;
    T.err = g->err;
    RP_CUDA(launch_guide_train(T, st), "guide training kernel");
    return RP_OK;
}

extern "C" rp_status rp_guide_train_step(rp_guide *g, float lr, float *loss_out, void *stream) {
    if (!g) return fail(RP_ERR_INVALID_ARG, "null guide");
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(RP_ERR_INVALID_ARG, "lr must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t n = g->cap;
    RP_CUDA(launch_guide_features(g->smp, g->d_box, n, g->X, g->omega, g->wt, g->wsum, st),
            "guide features");
    RP_CUDA(cudaMemsetAsync(g->grad, 0, sizeof(float) * kGWeights, st), "memset");
    RP_CUDA(cudaMemsetAsync(g->loss, 0, sizeof(float), st), "memset");
    RP_CUDA(cudaMemsetAsync(g->amax, 0, sizeof(unsigned int) * 4, st), "memset");
    GuideTrain T{};
    T.W = g->Wbf;
    T.X = g->X;
    T.omega = g->omega;
    T.wt = g->wt;
    T.n = n;
    T.inv_n = 1.0f / (float)n;
    T.wsum = g->wsum;          // the loss is the weighted mean -sum wt log q / sum wt
    T.grad = g->grad;
    T.loss = g->loss;
    T.amax = g->amax;
    T.err = g->err;
    RP_CUDA(launch_guide_train(T, st), "guide training kernel");
    g->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.99f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)g->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)g->adam_t));
    RP_CUDA(launch_guide_adam(g->Wm, g->m, g->v, g->grad, g->Wbf, kGWeights, lr, b1, b2, 1e-8f, c1, c2, st),
            "adam");
    RP_CUDA(cudaStreamSynchronize(st), "training step");
    int err = 0;
    float loss = 0.f, amax[4];
    unsigned int ab[4];
    RP_CUDA(cudaMemcpy(&err, g->err, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (err) return fail(RP_ERR_TIMEOUT, "a tensor-core wait of the guide kernels timed out");
    RP_CUDA(cudaMemcpy(&loss, g->loss, sizeof(float), cudaMemcpyDeviceToHost), "read loss");
    RP_CUDA(cudaMemcpy(ab, g->amax, sizeof ab, cudaMemcpyDeviceToHost), "read maxima");
    for (int l = 0; l < 4; ++l) std::memcpy(&amax[l], &ab[l], sizeof(float));
    if (loss_out) *loss_out = loss;
    std::vector<float> W(kGWeights);
    RP_CUDA(cudaMemcpy(W.data(), g->Wm, sizeof(float) * kGWeights, cudaMemcpyDeviceToHost), "download");
    return quantize(g, W.data(), amax);
}

extern "C" rp_status rp_guide_wait_selftest(rp_guide *g, uint64_t limit_ns) {
    if (!g) return fail(RP_ERR_INVALID_ARG, "null guide");
    if (limit_ns == 0 || limit_ns > 2000000000ull)
        return fail(RP_ERR_INVALID_ARG, "limit_ns must be in (0, 2e9]");
    RP_CUDA(cudaDeviceSynchronize(), "sync");
    int prev = 0;
    RP_CUDA(cudaMemcpy(&prev, g->err, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (prev) return fail(RP_ERR_TIMEOUT, "a tensor-core wait of the guide kernels timed out earlier");
    int8_t *in = nullptr;
    float *out = nullptr;
    cudaError_t e = cudaMalloc((void **)&in, 128 * kGIn);
    if (e == cudaSuccess) e = cudaMalloc((void **)&out, 128 * kGOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(in, 0, 128 * kGIn);
    GuideNet net{};
    net.Wq = g->Wq;
    for (int l = 0; l < 4; ++l) net.hid_scale[l] = 1.0f;
    net.out_scale = 1.0f;
    if (e == cudaSuccess) e = launch_guide_wait_selftest(net, in, out, g->err, limit_ns, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, g->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err) e = cudaMemset(g->err, 0, sizeof(int));   // the expected timeout
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "guide wait self-test");
    return err ? fail(RP_ERR_TIMEOUT, "the withheld tensor-core wait ran out (expected)") : RP_OK;
}

extern "C" rp_status rp_guide_status(rp_guide *g) {
    if (!g) return fail(RP_ERR_INVALID_ARG, "null guide");
    int err = 0;
    RP_CUDA(cudaDeviceSynchronize(), "sync");
    RP_CUDA(cudaMemcpy(&err, g->err, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    return err ? fail(RP_ERR_TIMEOUT, "a tensor-core wait of the guide kernels timed out") : RP_OK;
}

extern "C" rp_status rp_scene_set_guide(rp_scene *scene, rp_guide *guide) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    scene->guide = guide;
    if (!guide) scene->free_guide_buffers();
    return RP_OK;
}

// ---------------------------------------------------------------------------
// batches of edits: every wave of every item captured in one CUDA graph
// ---------------------------------------------------------------------------

struct rp_batch_s {
    struct Item {
        DevEdit E;
        int W, H;
        uint32_t spp, mask;
        double *out;
        uint64_t cost;
        int branch;
    };
    struct Branch {
        WaveBuf W{};
        std::vector<void *> allocs;
        cudaStream_t s = nullptr;
        cudaEvent_t join = nullptr;
    };
    rp_scene *sc = nullptr;
    std::vector<Item> items;
    rp_batch_config cfg{};
    unsigned long long *d_seeds = nullptr;
    std::vector<Branch> br;          // graph mode: branches; persistent mode: job slots
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    // persistent mode: the jobs' launch arguments, the rounds' work counters
    // and barrier, the timeout flag
    LaunchArgs *d_jobs = nullptr;
    unsigned int *d_ctrl = nullptr;
    int *d_err = nullptr;
    size_t jobs = 0, rounds = 0;
    ~rp_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (fork) cudaEventDestroy(fork);
        if (d_jobs) cudaFree(d_jobs);
        if (d_ctrl) cudaFree(d_ctrl);
        if (d_err) cudaFree(d_err);
        for (Branch &b : br) {
            for (void *p : b.allocs) cudaFree(p);
            if (b.s) cudaStreamDestroy(b.s);
            if (b.join) cudaEventDestroy(b.join);
        }
        if (d_seeds) cudaFree(d_seeds);
    }
};

namespace {

int popcount4(uint32_t m) { return __builtin_popcount(m & 127u); }

rp_status check_items(rp_scene *sc, const rp_batch_item *items, uint32_t n) {
    if (!sc || !items || n == 0) return fail(RP_ERR_INVALID_ARG, "null scene, null items or no items");
    for (uint32_t i = 0; i < n; ++i) {
        const rp_batch_item &it = items[i];
        if (!it.edit || !it.d_out) return fail(RP_ERR_INVALID_ARG, "batch item without edit or output");
        const uint64_t W = it.width ? it.width : (uint32_t)sc->S.W, H = it.height ? it.height : (uint32_t)sc->S.H;
        if (W == 0 || H == 0 || W * H > (1u << 26)) return fail(RP_ERR_INVALID_ARG, "item image size out of range");
        if (it.spp == 0 || (uint64_t)it.spp * W * H > 0xffffffffull)
            return fail(RP_ERR_INVALID_ARG, "item spp must be positive and spp * width * height fit in 32 bits");
        if (it.tech_mask == 0 || (it.tech_mask & ~RP_TECH_SEVEN)) return fail(RP_ERR_INVALID_ARG, "bad technique mask");
        if (rp_status s = guide_fits(sc, it.edit->E)) return s;
    }
    return RP_OK;
}

// Persistent mode: every wave of every item's techniques and frames is a job
// (launch arguments of its own, the wave buffers of a slot); jobs of the same
// technique, frame and edit kind form rounds of up to cfg.streams jobs, and
// each round is one cooperative launch of the persistent batch kernel
// (k_batch.cuh) in the captured graph, after a reset of its work counters.
rp_status batch_build_persistent(rp_batch *b, const rp_batch_item *items, bool motion) {
    rp_scene *sc = b->sc;
    const rp_batch_config &c = b->cfg;
    const int D = sc->S.max_depth;
    b->br.resize(c.streams);
    for (rp_batch_s::Branch &sl : b->br)
        if (rp_status s = alloc_wavebuf(sl.W, sl.allocs, c.wave_roots, D, motion)) return s;
    struct Job {
        LaunchArgs a;
        int tech;
    };
    // jobs grouped by (frame, technique, mapped), in that order
    std::map<std::tuple<int, int, int>, std::vector<Job>> groups;
    const int techs[7] = {1, 2, 3, 7, 4, 5, 6};
    for (size_t i = 0; i < b->items.size(); ++i) {
        const rp_batch_s::Item &it = b->items[i];
        LaunchArgs a = base_args(sc, it.E, it.spp, items[i].seed, it.mask);
        a.G = GuideLaunch{};
        a.stats = nullptr;
        a.timer = nullptr;
        set_resolution(sc, a.S, it.W, it.H);
        a.invN = (float)(1.0 / ((double)it.spp * it.W * it.H));
        a.img = it.out;
        a.residual = 1;
        a.seed_dev = b->d_seeds + i;
        const uint32_t N = it.spp * (uint32_t)(it.W * it.H);
        for (int g = 1; g <= 2; ++g)
            for (int t = 0; t < 7; ++t) {
                if (!(it.mask & (1u << t)) || (t >= 4 && !it.E.motion)) continue;
                const int mapped = (t >= 4 || it.E.motion) ? 1 : 0;
                a.frame = g;
                for (uint32_t r0 = 0; r0 < N; r0 += c.wave_roots) {
                    a.root_begin = r0;
                    a.root_end = std::min(N, r0 + c.wave_roots);
                    groups[std::make_tuple(g, t, mapped)].push_back(Job{a, techs[t]});
                }
            }
    }
    // rounds: consecutive jobs of a group, job k of a round in slot k
    std::vector<LaunchArgs> all;
    struct Round {
        size_t first;
        int n, tech, mapped;
    };
    std::vector<Round> rounds;
    for (auto &kv : groups) {
        std::vector<Job> &js = kv.second;
        for (size_t j0 = 0; j0 < js.size(); j0 += c.streams) {
            const int nj = (int)std::min<size_t>(c.streams, js.size() - j0);
            rounds.push_back(Round{all.size(), nj, js[j0].tech, std::get<2>(kv.first)});
            for (int k = 0; k < nj; ++k) {
                LaunchArgs a = js[j0 + k].a;
                a.W = b->br[k].W;
                all.push_back(a);
            }
        }
    }
    b->jobs = all.size();
    b->rounds = rounds.size();
    cudaError_t e = cudaMalloc((void **)&b->d_jobs, sizeof(LaunchArgs) * std::max<size_t>(all.size(), 1));
    if (e == cudaSuccess && !all.empty())
        e = cudaMemcpy(b->d_jobs, all.data(), sizeof(LaunchArgs) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ctrl, sizeof(unsigned int) * (kMaxBatchStages + 2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "batch job tables");
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return fail(RP_ERR_CUDA, "stream creation failed");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (const Round &r : rounds) {
        if (e != cudaSuccess) break;
        BatchRound R{};
        R.jobs = b->d_jobs + r.first;
        R.n_jobs = r.n;
        R.n_stages = batch_stages(r.tech, D, r.mapped != 0, R.stages);
        R.work = b->d_ctrl;
        R.bar = b->d_ctrl + kMaxBatchStages;
        R.err = b->d_err;
        R.chunk = 128;             // elements per work item of one warp
        e = cudaMemsetAsync(b->d_ctrl, 0, sizeof(unsigned int) * (kMaxBatchStages + 2), cs);
        if (e == cudaSuccess) e = launch_batch_round(r.tech, R, (int)c.blocks_per_sm, cs);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(cs);
    b->graph = graph;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture of the persistent batch");
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return fail(RP_ERR_CUDA, "graph instantiation failed");
    cudaGraphGetNodes(b->graph, nullptr, &b->nodes);
    return RP_OK;
}

rp_status batch_build(rp_scene *sc, const rp_batch_item *items, uint32_t n, const rp_batch_config *cfg_in,
                      rp_batch **out) {
    if (rp_status s = check_items(sc, items, n)) return s;
    rp_batch *b = new rp_batch_s();
    b->sc = sc;
    uint64_t max_roots = 1;
    bool motion = false;
    for (uint32_t i = 0; i < n; ++i) {
        rp_batch_s::Item it{};
        it.E = items[i].edit->E;
        it.W = items[i].width ? (int)items[i].width : sc->S.W;
        it.H = items[i].height ? (int)items[i].height : sc->S.H;
        it.spp = items[i].spp;
        it.mask = items[i].tech_mask;
        it.out = items[i].d_out;
        const uint64_t roots = (uint64_t)it.spp * it.W * it.H;
        it.cost = roots * (uint64_t)popcount4(it.mask) * (it.E.motion ? 2 : 1);
        max_roots = std::max(max_roots, roots);
        motion = motion || it.E.motion;
        b->items.push_back(it);
    }
    rp_batch_config c = cfg_in ? *cfg_in : rp_batch_config{};
    if (c.wave_roots == 0) c.wave_roots = (uint32_t)std::min<uint64_t>(max_roots, sc->wave_cap);
    if (c.wave_roots > (1u << 24)) c.wave_roots = 1u << 24;
    c.wave_roots = std::max<uint32_t>(c.wave_roots, 256u);
    if (c.streams == 0) c.streams = 1;
    c.streams = std::min<uint32_t>(c.streams, std::min<uint32_t>(8u, n));
    c.blocks_per_sm = std::min<uint32_t>(c.blocks_per_sm, 128u);     // 0: by the wave's roots
    c.persistent = c.persistent ? 1u : 0u;
    if (c.persistent) {
        // jobs per round (one wave buffer each): at most kMaxBatchJobs
        c.streams = std::min<uint32_t>(std::max<uint32_t>(cfg_in && cfg_in->streams ? cfg_in->streams : 8u, 1u),
                                       (uint32_t)kMaxBatchJobs);
        if (!cfg_in || cfg_in->blocks_per_sm == 0) c.blocks_per_sm = 0;      // as many as fit
    }
    b->cfg = c;
    auto bail = [&](rp_status s) { delete b; return s; };
    cudaError_t e = cudaMalloc((void **)&b->d_seeds, sizeof(unsigned long long) * n);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc seeds"));
    std::vector<unsigned long long> seeds(n);
    for (uint32_t i = 0; i < n; ++i) seeds[i] = items[i].seed;
    e = cudaMemcpy(b->d_seeds, seeds.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "upload seeds"));
    if (c.persistent) {
        if (rp_status s = batch_build_persistent(b, items, motion)) return bail(s);
        *out = b;
        return RP_OK;
    }
    // longest items first, each to the least loaded branch
    b->br.resize(c.streams);
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return b->items[x].cost > b->items[y].cost; });
    std::vector<uint64_t> load(c.streams, 0);
    for (uint32_t i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->items[i].branch = k;
        load[k] += b->items[i].cost;
    }
    for (rp_batch_s::Branch &br : b->br) {
        if (rp_status s = alloc_wavebuf(br.W, br.allocs, c.wave_roots, sc->S.max_depth, motion)) return bail(s);
        if (cudaStreamCreateWithFlags(&br.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&br.join, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(RP_ERR_CUDA, "stream creation failed"));
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(RP_ERR_CUDA, "event creation failed"));
    // capture: fork to the branches, every wave of every item, join
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(RP_ERR_CUDA, "stream creation failed"));
    rp_status st = RP_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, cs);
    for (rp_batch_s::Branch &br : b->br)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(br.s, b->fork, 0);
    const int techs[7] = {1, 2, 3, 7, 4, 5, 6};
    const int grid_q = (int)c.blocks_per_sm * device_sm_count();
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
        const rp_batch_s::Item &it = b->items[i];
        rp_batch_s::Branch &br = b->br[it.branch];
        LaunchArgs a = base_args(sc, it.E, it.spp, items[i].seed, it.mask);
        a.G = GuideLaunch{};
        a.stats = nullptr;
        a.timer = nullptr;
        set_resolution(sc, a.S, it.W, it.H);
        a.invN = (float)(1.0 / ((double)it.spp * it.W * it.H));
        a.img = it.out;
        a.residual = 1;
        a.seed_dev = b->d_seeds + i;
        a.grid_q = grid_q;
        a.W = br.W;
        const uint32_t N = it.spp * (uint32_t)(it.W * it.H);
        for (int g = 1; g <= 2 && e == cudaSuccess; ++g)
            for (int t = 0; t < 7 && e == cudaSuccess; ++t) {
                if (!(it.mask & (1u << t)) || (t >= 4 && !it.E.motion)) continue;
                a.frame = g;
                for (uint32_t r0 = 0; r0 < N && e == cudaSuccess; r0 += c.wave_roots) {
                    a.root_begin = r0;
                    a.root_end = std::min(N, r0 + c.wave_roots);
                    e = launch_wave(techs[t], a, br.s);
                }
            }
    }
    for (rp_batch_s::Branch &br : b->br) {
        if (e == cudaSuccess) e = cudaEventRecord(br.join, br.s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, br.join, 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(cs);
    b->graph = graph;
    if (e != cudaSuccess) st = cuda_fail(e, "graph capture");
    if (st == RP_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        st = fail(RP_ERR_CUDA, "graph instantiation failed");
    if (st == RP_OK) cudaGraphGetNodes(b->graph, nullptr, &b->nodes);
    if (st != RP_OK) return bail(st);
    *out = b;
    return RP_OK;
}

}  // namespace

extern "C" rp_status rp_batch_create(rp_scene *scene, const rp_batch_item *items, uint32_t n,
                                     const rp_batch_config *config, rp_batch **out) {
    if (!out) return fail(RP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    return batch_build(scene, items, n, config, out);
}

extern "C" void rp_batch_destroy(rp_batch *batch) { delete batch; }

extern "C" rp_status rp_batch_launch(rp_batch *batch, void *stream) {
    if (!batch || !batch->exec) return fail(RP_ERR_INVALID_ARG, "null batch");
    RP_CUDA(cudaGraphLaunch(batch->exec, (cudaStream_t)stream), "graph launch");
    batch->sc->last_stream = (cudaStream_t)stream;
    return RP_OK;
}

extern "C" rp_status rp_batch_set_seeds(rp_batch *batch, const uint64_t *seeds, void *stream) {
    if (!batch || !seeds) return fail(RP_ERR_INVALID_ARG, "null argument");
    RP_CUDA(cudaMemcpyAsync(batch->d_seeds, seeds, sizeof(uint64_t) * batch->items.size(),
                            cudaMemcpyHostToDevice, (cudaStream_t)stream),
            "seed upload");
    return RP_OK;
}

extern "C" rp_status rp_batch_status(rp_batch *batch) {
    if (!batch) return fail(RP_ERR_INVALID_ARG, "null batch");
    RP_CUDA(cudaDeviceSynchronize(), "sync");
    if (!batch->d_err) return RP_OK;
    int err = 0;
    RP_CUDA(cudaMemcpy(&err, batch->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    return err ? fail(RP_ERR_TIMEOUT, "a grid barrier of the persistent batch kernel timed out") : RP_OK;
}

extern "C" rp_status rp_batch_info(rp_batch *batch, rp_batch_config *config, uint64_t *graph_nodes) {
    if (!batch) return fail(RP_ERR_INVALID_ARG, "null batch");
    if (config) *config = batch->cfg;
    if (graph_nodes) *graph_nodes = batch->nodes;
    return RP_OK;
}

extern "C" rp_status rp_batch_autotune(rp_scene *scene, const rp_batch_item *items, uint32_t n,
                                       uint32_t spp_divisor, rp_batch_config *best, double *best_ms) {
    if (!best) return fail(RP_ERR_INVALID_ARG, "null argument");
    if (rp_status s = check_items(scene, items, n)) return s;
    if (spp_divisor == 0) spp_divisor = 1;
    // proxy items: spp / spp_divisor, all outputs into one scratch image
    size_t px = 0;
    uint64_t max_roots = 1;
    std::vector<rp_batch_item> proxy(items, items + n);
    for (rp_batch_item &it : proxy) {
        it.spp = std::max(1u, it.spp / spp_divisor);
        const size_t W = it.width ? it.width : (uint32_t)scene->S.W, H = it.height ? it.height : (uint32_t)scene->S.H;
        px = std::max(px, W * H);
        max_roots = std::max<uint64_t>(max_roots, (uint64_t)it.spp * W * H);
    }
    double *scratch = nullptr;
    RP_CUDA(cudaMalloc((void **)&scratch, px * 3 * sizeof(double)), "cudaMalloc scratch");
    for (rp_batch_item &it : proxy) it.d_out = scratch;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto measure = [&](const rp_batch_config &c, double &ms) -> rp_status {
        rp_batch *b = nullptr;
        if (rp_status s = batch_build(scene, proxy.data(), n, &c, &b)) return s;
        float best_t = 1e30f;
        cudaError_t e = cudaGraphLaunch(b->exec, st);            // warm-up
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = cudaGraphLaunch(b->exec, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best_t = std::min(best_t, t);
        }
        delete b;
        if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
        ms = best_t;
        return RP_OK;
    };
    // coordinate descent from the defaults of each batch mode, then the
    // faster mode:
    //  - graph mode over the wave size (2^20 .. 2^23), the concurrent branches
    //    (1, 2, 4) and the blocks per SM of the queue kernels (by the wave's
    //    roots, 16, 32, 64, 128);
    //  - persistent mode over the wave size (2^18 .. 2^21) and the waves per
    //    round (4 .. 32) with at most 2^23 roots in flight, and the resident
    //    blocks per SM (all that fit, 4, 2)
    auto descend = [&](rp_batch_config cur, const std::vector<uint32_t> *vals, double &cur_ms,
                       bool persistent) -> rp_status {
        rp_status st2 = measure(cur, cur_ms);
        for (int dim = 0; dim < 3 && st2 == RP_OK; ++dim)
            for (uint32_t v : vals[dim]) {
                rp_batch_config c = cur;
                (dim == 0 ? c.wave_roots : dim == 1 ? c.streams : c.blocks_per_sm) = v;
                if (c.wave_roots == cur.wave_roots && c.streams == cur.streams &&
                    c.blocks_per_sm == cur.blocks_per_sm)
                    continue;
                if (persistent && (uint64_t)c.wave_roots * c.streams > (1ull << 23)) continue;
                double ms = 0.0;
                st2 = measure(c, ms);
                if (st2 != RP_OK) break;
                if (ms < cur_ms) { cur = c; cur_ms = ms; }
            }
        if (st2 == RP_OK) *best = cur;
        return st2;
    };
    std::vector<uint32_t> gw[3], pw[3];
    for (uint32_t w = 1u << 20; w <= (1u << 23); w <<= 1) {
        gw[0].push_back(w);
        if (w >= max_roots) break;
    }
    gw[1] = {1, 2, 4};
    gw[2] = {0, 16, 32, 64, 128};
    for (uint32_t w = 1u << 18; w <= (1u << 21); w <<= 1) {
        pw[0].push_back(w);
        if (w >= max_roots) break;
    }
    pw[1] = {4, 8, 16, 32};
    pw[2] = {0, 4, 2};
    rp_batch_config g0{};
    g0.wave_roots = (uint32_t)std::min<uint64_t>(max_roots, scene->wave_cap);
    g0.streams = 1;
    g0.blocks_per_sm = 0;
    rp_batch_config p0{};
    p0.wave_roots = (uint32_t)std::min<uint64_t>(max_roots, 1u << 20);
    p0.streams = 8;
    p0.blocks_per_sm = 0;
    p0.persistent = 1;
    double g_ms = 0.0, p_ms = 0.0, cur_ms = 0.0;
    rp_batch_config g_best{}, p_best{};
    rp_status s = descend(g0, gw, g_ms, false);
    if (s == RP_OK) g_best = *best;
    if (s == RP_OK) s = descend(p0, pw, p_ms, true);
    if (s == RP_OK) p_best = *best;
    rp_batch_config cur = p_ms < g_ms ? p_best : g_best;
    cur_ms = p_ms < g_ms ? p_ms : g_ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(scratch);
    if (s != RP_OK) return s;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return RP_OK;
}

extern "C" rp_status rp_scene_set_mapping(rp_scene *scene, int mode) {
    if (!scene) return fail(RP_ERR_INVALID_ARG, "null scene");
    if (mode < 0 || mode > 2) return fail(RP_ERR_INVALID_ARG, "mapping mode must be 0, 1 or 2");
    scene->map_mode = mode;
    return RP_OK;
}
