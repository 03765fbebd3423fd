/*
 * CPU oracle for the residual path integral estimator (arXiv 2406.16302).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * double-precision reference that the CUDA library is checked against.  Only
 * the test suite, the package smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code, header,
 * table or constant generator with the CUDA library: both read the same
 * float32 scene arrays and implement the same published definitions
 * independently.
 *
 * What it computes (paper sections in brackets):
 *   - the primal path integral I = int f dmu with f = W_e G0 prod rho G V L_e
 *     [Sec. 3.1, Eq. pathIntegral / pathcontribution], by camera path tracing
 *     with next-event estimation;
 *   - the residual I2 - I1 as one mapped integral of f2(p) - f1(T p)|T'(p)|
 *     [Sec. 3.2, Eq. shiftmapped], restricted to dynamic paths
 *     [Sec. 3.4, Eq. difference_integral], estimated with the dynamic-vertex
 *     techniques (1) "dynamic from emitter", (2) "dynamic from sensor",
 *     (3) "dynamic two ends" [Sec. 4.1] plus path tracing with static paths
 *     rejected [Sec. 4.3], optionally the ghost techniques (4) "ghost from
 *     emitter", (5) "ghost from sensor", (6) "ghost two ends" [Sec. 4.2],
 *     combined by the balance heuristic over all
 *     techniques that can produce a path [Sec. 4.3], with the path mapping
 *     operators of Sec. 5 (object transform, reconnection, random replay,
 *     rejection) and two-way mapping [Sec. 5, "Path rejection"];
 *   - optionally, technique (3) with its first light-side direction drawn
 *     from a learned von Mises-Fisher mixture mixed 50/50 with the cosine
 *     density (not in the paper; an integer network evaluated exactly), and
 *     the float network's loss and gradient used to train it.
 *
 * Readings of the paper where it is silent, ambiguous or garbled:
 *   R1 area measure everywhere: |J| of object transform and of reconnection
 *      is 1; a replayed vertex contributes the ratio of its area sampling
 *      densities in the two frames.
 *   R2 the mapping is a function of the path alone: it follows the walk order
 *      of the unique technique owning the path's one dynamic vertex, and a
 *      replayed step recovers its random numbers by inverting that step's
 *      sampling routine.
 *   R3 two-way estimator: a base path x of frame g with mapped path y adds
 *      s_g [f_g(x) - f_g'(y) J] / (N (P_g(x) + P_g'(y) J)), split between
 *      the pixels of x and y; a rejected or invalid pair adds
 *      s_g f_g(x) / (N P_g(x)); s_2 = +1, s_1 = -1.
 *   R4 acceptance is symmetric: the mapped path must have exactly one dynamic
 *      vertex, max(J, 1/J) <= jacobian_max, and every replayed step must be
 *      one that the inverse mapping would also replay.
 *   R5 without motion (material edit, identity edit) the mapping is the
 *      identity on every path and nothing is rejected.
 *   R6 paths have at most max_depth edges; emitters are reached by
 *      next-event estimation only (paths of two vertices, camera to emitter,
 *      come from the camera ray).
 *
 * Parity status: pinned.  Philox by published known answers; intersection by
 * brute force; BSDF and pdfs by quadrature; primal by the white furnace and
 * the closed-form polygon irradiance; residual by exact zero for identity
 * edits, the closed-form moving-quad residual, agreement with the difference
 * of independent primal renders, mapping bijectivity and finite-difference
 * Jacobians; the balance heuristic's terms by brute-force counts of dynamic
 * vertices and ghost crossings; each of techniques (1)-(3) alone by path
 * tracing restricted to its domain.  Learned proposal: vMF density and sampler by quadrature and the
 * closed-form cosine CDF, encoding by known angles, integer network by
 * hand-built networks, float gradient by finite differences, guided
 * estimator by agreement with correlated path tracing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* vectors                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct { double x, y, z; } vec3;

static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 add(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 sub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 scale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static vec3 mul(vec3 a, vec3 b) { return v3(a.x * b.x, a.y * b.y, a.z * b.z); }
static double dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 cross(vec3 a, vec3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double length(vec3 a) { return sqrt(dot(a, a)); }
static vec3 normalize(vec3 a) { return scale(a, 1.0 / length(a)); }
static int is_zero3(vec3 a) { return a.x == 0.0 && a.y == 0.0 && a.z == 0.0; }
static int same_point(vec3 a, vec3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:    */
/* ten rounds of two 32x32->64 multiplies with key bumps by the Weyl          */
/* constants.                                                                */
/* ------------------------------------------------------------------------- */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* technique codes and random-number stream layout */
enum { TECH_PT = 0, TECH_T1 = 1, TECH_T2 = 2, TECH_T3 = 3, TECH_T4 = 4, TECH_T5 = 5, TECH_T6 = 6,
       TECH_T7 = 7 };
enum { SIDE_ROOT = 0, SIDE_EYE = 1, SIDE_LIGHT = 2, SIDE_NEE = 3 };

typedef struct { double u[4]; } rnd4;

static rnd4 draw(uint64_t seed, uint32_t root, int tech, int frame, int side, int step) {
    uint32_t ctr[4] = {root, ((uint32_t)tech << 24) | ((uint32_t)frame << 20) |
                                 ((uint32_t)side << 16) | (uint32_t)step, 0u, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    rnd4 o;
    for (int i = 0; i < 4; ++i) o.u[i] = (double)(r[i] >> 8) * (1.0 / 16777216.0);
    return o;
}

/* ------------------------------------------------------------------------- */
/* scene                                                                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int type;            /* 0 Lambert, 1 GGX */
    vec3 albedo;
    double alpha;
    vec3 f0;
    vec3 emission;
} material;

typedef struct { vec3 v0, v1, v2; } tri;

typedef struct {
    double lo[3], hi[3];
    int left, right;     /* children; leaf if left < 0 */
    int first, count;    /* leaf primitive range into the index array */
} bvh_node;

typedef struct {
    bvh_node *nodes;
    int n_nodes;
    int *index;          /* primitive ids */
    const tri *tris;     /* indexed by primitive id */
    int id_offset;       /* global id = id_offset + local id */
} bvh;

#define MAX_INST 8

typedef struct {
    /* static geometry (world) and dynamic object (object space) */
    int n_static, n_dyn;
    tri *stat;           /* world-space static triangles */
    int *stat_mat;
    tri *dyn_obj;        /* object-space dynamic triangles */
    material *mats;
    int n_mats;
    /* per-frame world copies of the dynamic object, index 1 and 2.  The
     * dynamic mesh may be several objects moved together (an edit of several
     * objects, Sec. 6): triangle i belongs to instance dyn_inst[i], which has
     * its own transforms and materials */
    tri *dyn_world[3];
    int n_inst;
    int *dyn_inst;       /* [n_dyn] instance of each dynamic triangle */
    double M[3][MAX_INST][12];
    material dyn_mat[3][MAX_INST];
    int motion;          /* some instance has M1 != M2 */
    int has_edit;
    /* acceleration */
    bvh stat_bvh;
    bvh dyn_bvh[3];
    int brute_force;
    int map_mode;        /* 0: no mapping, 1: object transform only, 2: camera replay (default) */
    /* sampling tables */
    double *dyn_cdf;     /* over dyn_obj areas */
    double dyn_area;
    int n_emit;
    int *emit_ids;       /* static triangle ids */
    double *emit_cdf;
    double emit_area;
    /* camera */
    vec3 cam_pos, cam_fwd, cam_right, cam_up;
    double hw, hh, pix_area;
    int W, H;
    /* parameters */
    int max_depth;
    double alpha_min, d_min, jac_max;
    double eps;
    struct oguide_s *guide;   /* learned proposal of technique (3), or NULL */
} oscene;

static double tri_area(const tri *t) {
    return 0.5 * length(cross(sub(t->v1, t->v0), sub(t->v2, t->v0)));
}

static vec3 tri_normal(const tri *t) {
    return normalize(cross(sub(t->v1, t->v0), sub(t->v2, t->v0)));
}

static vec3 apply_M(const double *M, vec3 p) {
    return v3(M[0] * p.x + M[1] * p.y + M[2] * p.z + M[3],
              M[4] * p.x + M[5] * p.y + M[6] * p.z + M[7],
              M[8] * p.x + M[9] * p.y + M[10] * p.z + M[11]);
}

/* --- BVH (median split over centroids, leaves of up to 4 triangles) ----- */

typedef struct { const tri *tris; double *cent; int axis; } sort_ctx;
static sort_ctx g_sort;
static int cmp_axis(const void *a, const void *b) {
    int ia = *(const int *)a, ib = *(const int *)b;
    double ca = g_sort.cent[3 * ia + g_sort.axis], cb = g_sort.cent[3 * ib + g_sort.axis];
    return (ca < cb) ? -1 : (ca > cb) ? 1 : (ia - ib);
}

static void tri_bounds(const tri *t, double lo[3], double hi[3]) {
    const vec3 *v[3] = {&t->v0, &t->v1, &t->v2};
    for (int k = 0; k < 3; ++k) {
        double a[3] = {v[k]->x, v[k]->y, v[k]->z};
        for (int d = 0; d < 3; ++d) {
            if (a[d] < lo[d]) lo[d] = a[d];
            if (a[d] > hi[d]) hi[d] = a[d];
        }
    }
}

static int bvh_build_rec(bvh *b, double *cent, int first, int count) {
    int id = b->n_nodes++;
    bvh_node *nd = &b->nodes[id];
    for (int d = 0; d < 3; ++d) { nd->lo[d] = 1e300; nd->hi[d] = -1e300; }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int i = first; i < first + count; ++i) {
        int p = b->index[i];
        tri_bounds(&b->tris[p], nd->lo, nd->hi);
        for (int d = 0; d < 3; ++d) {
            double c = cent[3 * p + d];
            if (c < clo[d]) clo[d] = c;
            if (c > chi[d]) chi[d] = c;
        }
    }
    if (count <= 4) {
        nd->left = nd->right = -1; nd->first = first; nd->count = count;
        return id;
    }
    int axis = 0;
    for (int d = 1; d < 3; ++d)
        if (chi[d] - clo[d] > chi[axis] - clo[axis]) axis = d;
    g_sort.cent = cent; g_sort.axis = axis;
    qsort(b->index + first, (size_t)count, sizeof(int), cmp_axis);
    int half = count / 2;
    int l = bvh_build_rec(b, cent, first, half);
    int r = bvh_build_rec(b, cent, first + half, count - half);
    b->nodes[id].left = l; b->nodes[id].right = r;
    b->nodes[id].first = 0; b->nodes[id].count = 0;
    return id;
}

static void bvh_build(bvh *b, const tri *tris, int n, int id_offset) {
    b->tris = tris; b->id_offset = id_offset; b->n_nodes = 0;
    b->nodes = (bvh_node *)malloc(sizeof(bvh_node) * (size_t)(2 * (n > 0 ? n : 1)));
    b->index = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (n <= 0) return;
    double *cent = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        b->index[i] = i;
        vec3 c = scale(add(add(tris[i].v0, tris[i].v1), tris[i].v2), 1.0 / 3.0);
        cent[3 * i] = c.x; cent[3 * i + 1] = c.y; cent[3 * i + 2] = c.z;
    }
    bvh_build_rec(b, cent, 0, n);
    free(cent);
}

static void bvh_free(bvh *b) { free(b->nodes); free(b->index); b->nodes = NULL; b->index = NULL; }

/* --- ray / triangle (Moller-Trumbore, both faces) ------------------------ */

static int ray_tri(vec3 o, vec3 d, const tri *t, double *tt, double *bu, double *bv) {
    vec3 e1 = sub(t->v1, t->v0), e2 = sub(t->v2, t->v0);
    vec3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    vec3 s = sub(o, t->v0);
    double u = dot(s, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    vec3 q = cross(s, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *tt = dot(e2, q) * inv;
    *bu = u; *bv = v;
    return 1;
}

static int ray_box(vec3 o, vec3 d, const double lo[3], const double hi[3], double tmin, double tmax) {
    double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0) {
            if (oo[a] < lo[a] || oo[a] > hi[a]) return 0;
            continue;
        }
        double t0 = (lo[a] - oo[a]) / dd[a], t1 = (hi[a] - oo[a]) / dd[a];
        if (t0 > t1) { double tmp = t0; t0 = t1; t1 = tmp; }
        if (t0 > tmin) tmin = t0;
        if (t1 < tmax) tmax = t1;
        if (tmin > tmax) return 0;
    }
    return 1;
}

typedef struct { double t, b1, b2; int prim; } hitrec;

/* closest hit (any=0) or first found (any=1) with t in (tmin, tmax),
 * skipping primitives ex0 and ex1 */
static int bvh_trace(const bvh *b, vec3 o, vec3 d, double tmin, double tmax, int ex0, int ex1,
                     int any, hitrec *h) {
    if (b->n_nodes == 0) return 0;
    int stack[128];
    int sp = 0, found = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bvh_node *nd = &b->nodes[stack[--sp]];
        if (!ray_box(o, d, nd->lo, nd->hi, tmin, tmax)) continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; ++i) {
                int lp = b->index[i];
                int gid = b->id_offset + lp;
                if (gid == ex0 || gid == ex1) continue;
                double t, u, v;
                if (ray_tri(o, d, &b->tris[lp], &t, &u, &v) && t > tmin && t < tmax) {
                    tmax = t; found = 1;
                    h->t = t; h->b1 = u; h->b2 = v; h->prim = gid;
                    if (any) return 1;
                }
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return found;
}

static int brute_trace(const tri *tris, int n, int off, vec3 o, vec3 d, double tmin, double tmax,
                       int ex0, int ex1, int any, hitrec *h) {
    int found = 0;
    for (int i = 0; i < n; ++i) {
        int gid = off + i;
        if (gid == ex0 || gid == ex1) continue;
        double t, u, v;
        if (ray_tri(o, d, &tris[i], &t, &u, &v) && t > tmin && t < tmax) {
            tmax = t; found = 1;
            h->t = t; h->b1 = u; h->b2 = v; h->prim = gid;
            if (any) return 1;
        }
    }
    return found;
}

/* scene query in frame g over static + dynamic (dyn_only restricts to the
 * dynamic object at its frame-g pose) */
static int scene_trace(const oscene *s, int g, vec3 o, vec3 d, double tmin, double tmax, int ex0,
                       int ex1, int any, int dyn_only, hitrec *h) {
    int found = 0;
    hitrec hh;
    if (!dyn_only) {
        int ok = s->brute_force
                     ? brute_trace(s->stat, s->n_static, 0, o, d, tmin, tmax, ex0, ex1, any, &hh)
                     : bvh_trace(&s->stat_bvh, o, d, tmin, tmax, ex0, ex1, any, &hh);
        if (ok) {
            *h = hh; found = 1; tmax = hh.t;
            if (any) return 1;
        }
    }
    if (s->n_dyn > 0) {
        int ok = s->brute_force
                     ? brute_trace(s->dyn_world[g], s->n_dyn, s->n_static, o, d, tmin, tmax, ex0,
                                   ex1, any, &hh)
                     : bvh_trace(&s->dyn_bvh[g], o, d, tmin, tmax, ex0, ex1, any, &hh);
        if (ok) { *h = hh; found = 1; }
    }
    return found;
}

/* ------------------------------------------------------------------------- */
/* path vertices                                                             */
/* ------------------------------------------------------------------------- */

enum { VK_CAMERA = 0, VK_SURFACE = 1 };

typedef struct {
    vec3 p, n;
    int kind;
    int prim;            /* global triangle id */
    int dyn;             /* on the dynamic object */
    double b1, b2;       /* barycentrics on prim */
    const material *mat;
} vtx;

static const tri *prim_tri(const oscene *s, int g, int prim) {
    return prim < s->n_static ? &s->stat[prim] : &s->dyn_world[g][prim - s->n_static];
}

static const material *prim_mat(const oscene *s, int g, int prim) {
    return prim < s->n_static ? &s->mats[s->stat_mat[prim]]
                              : &s->dyn_mat[g][s->dyn_inst[prim - s->n_static]];
}

/* the surface point with barycentrics (b1, b2) on prim, in frame g */
static vtx make_vertex(const oscene *s, int g, int prim, double b1, double b2) {
    const tri *t = prim_tri(s, g, prim);
    vtx v;
    double b0 = 1.0 - b1 - b2;
    v.p = add(add(scale(t->v0, b0), scale(t->v1, b1)), scale(t->v2, b2));
    v.n = tri_normal(t);
    v.kind = VK_SURFACE;
    v.prim = prim;
    v.dyn = prim >= s->n_static;
    v.b1 = b1; v.b2 = b2;
    v.mat = prim_mat(s, g, prim);
    return v;
}

static vtx camera_vertex(const oscene *s) {
    vtx v;
    memset(&v, 0, sizeof v);
    v.p = s->cam_pos;
    v.kind = VK_CAMERA;
    v.prim = -1;
    return v;
}

static int is_black(const material *m) {
    return m->type == 0 ? is_zero3(m->albedo) : is_zero3(m->f0);
}

static double roughness(const material *m) { return m->type == 0 ? INFINITY : m->alpha; }

/* ------------------------------------------------------------------------- */
/* tangent frame: Duff et al. 2017 branchless basis, built in a fixed generic */
/* rotation so that no axis-aligned normal sits on its discontinuity          */
/* ------------------------------------------------------------------------- */

static const double QROT[3][3] = {
    {0.727128712871287, -0.16910891089108918, 0.6653465346534656},
    {0.44356435643564374, 0.85544554455445543, -0.26732673267326734},
    {-0.52396039603960409, 0.48950495049504961, 0.69702970297029698}};

static void tangent_frame(vec3 n, vec3 *t, vec3 *b) {
    vec3 m = v3(QROT[0][0] * n.x + QROT[0][1] * n.y + QROT[0][2] * n.z,
                QROT[1][0] * n.x + QROT[1][1] * n.y + QROT[1][2] * n.z,
                QROT[2][0] * n.x + QROT[2][1] * n.y + QROT[2][2] * n.z);
    double sign = m.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + m.z);
    double c = m.x * m.y * a;
    vec3 tl = v3(1.0 + sign * m.x * m.x * a, sign * c, -sign * m.x);
    vec3 bl = v3(c, sign + m.y * m.y * a, -m.y);
    /* rotate back with the transpose */
    *t = v3(QROT[0][0] * tl.x + QROT[1][0] * tl.y + QROT[2][0] * tl.z,
            QROT[0][1] * tl.x + QROT[1][1] * tl.y + QROT[2][1] * tl.z,
            QROT[0][2] * tl.x + QROT[1][2] * tl.y + QROT[2][2] * tl.z);
    *b = v3(QROT[0][0] * bl.x + QROT[1][0] * bl.y + QROT[2][0] * bl.z,
            QROT[0][1] * bl.x + QROT[1][1] * bl.y + QROT[2][1] * bl.z,
            QROT[0][2] * bl.x + QROT[1][2] * bl.y + QROT[2][2] * bl.z);
}

/* ------------------------------------------------------------------------- */
/* BSDFs (Lambert; GGX microfacet reflection of Walter et al. 2007 with       */
/* separable Smith masking and Schlick Fresnel)                               */
/* ------------------------------------------------------------------------- */

static double ggx_D(double a2, double cos_h) {
    double k = cos_h * cos_h * (a2 - 1.0) + 1.0;
    return a2 / (PI * k * k);
}

static double ggx_G1(double a2, double c) {
    return 2.0 * c / (c + sqrt(a2 + (1.0 - a2) * c * c));
}

/* rho(wi, wo) with wi, wo unit vectors leaving the surface point */
static vec3 bsdf_eval(const material *m, vec3 n, vec3 wi, vec3 wo) {
    double ci = dot(n, wi), co = dot(n, wo);
    if (ci <= 0.0 || co <= 0.0) return v3(0, 0, 0);
    if (m->type == 0) return scale(m->albedo, 1.0 / PI);
    double a2 = m->alpha * m->alpha;
    vec3 h = normalize(add(wi, wo));
    double ch = dot(n, h), ih = dot(wi, h);
    if (ch <= 0.0 || ih <= 0.0) return v3(0, 0, 0);
    double fw = pow(1.0 - ih, 5.0);
    vec3 F = v3(m->f0.x + (1.0 - m->f0.x) * fw, m->f0.y + (1.0 - m->f0.y) * fw,
                m->f0.z + (1.0 - m->f0.z) * fw);
    double s = ggx_D(a2, ch) * ggx_G1(a2, ci) * ggx_G1(a2, co) / (4.0 * ci * co);
    return scale(F, s);
}

/* solid-angle density of sampling wo given the conditioning direction wc */
static double bsdf_pdf(const material *m, vec3 n, vec3 wc, vec3 wo) {
    double cc = dot(n, wc), co = dot(n, wo);
    if (cc <= 0.0 || co <= 0.0) return 0.0;
    if (m->type == 0) return co / PI;
    double a2 = m->alpha * m->alpha;
    vec3 h = normalize(add(wc, wo));
    double ch = dot(n, h), oh = dot(wo, h);
    if (ch <= 0.0 || oh <= 0.0) return 0.0;
    return ggx_D(a2, ch) * ch / (4.0 * oh);
}

static double cosine_pdf(vec3 n, vec3 wo) {
    double c = dot(n, wo);
    return c > 0.0 ? c / PI : 0.0;
}

static vec3 cosine_dir(vec3 n, double u1, double u2) {
    vec3 t, b;
    tangent_frame(n, &t, &b);
    double r = sqrt(u1), phi = 2.0 * PI * u2;
    double z = sqrt(fmax(0.0, 1.0 - u1));
    return add(add(scale(t, r * cos(phi)), scale(b, r * sin(phi))), scale(n, z));
}

static void cosine_inverse(vec3 n, vec3 w, double *u1, double *u2) {
    vec3 t, b;
    tangent_frame(n, &t, &b);
    double x = dot(w, t), y = dot(w, b);
    *u1 = x * x + y * y;
    double a = atan2(y, x) / (2.0 * PI);
    *u2 = a < 0.0 ? a + 1.0 : a;
}

/* sample wo at a surface with conditioning direction wc; 0 on failure */
static int bsdf_sample(const material *m, vec3 n, vec3 wc, double u1, double u2, vec3 *wo) {
    if (dot(n, wc) <= 0.0) return 0;
    if (m->type == 0) {
        *wo = cosine_dir(n, u1, u2);
        return dot(n, *wo) > 0.0;
    }
    double a2 = m->alpha * m->alpha;
    double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
    double ct = sqrt(c2), st = sqrt(fmax(0.0, 1.0 - c2)), phi = 2.0 * PI * u2;
    vec3 t, b;
    tangent_frame(n, &t, &b);
    vec3 h = add(add(scale(t, st * cos(phi)), scale(b, st * sin(phi))), scale(n, ct));
    double d = dot(wc, h);
    if (d <= 0.0) return 0;
    *wo = sub(scale(h, 2.0 * d), wc);
    return dot(n, *wo) > 0.0;
}

/* the random numbers (u1, u2) that make bsdf_sample produce wo */
static void bsdf_inverse(const material *m, vec3 n, vec3 wc, vec3 wo, double *u1, double *u2) {
    if (m->type == 0) { cosine_inverse(n, wo, u1, u2); return; }
    double a2 = m->alpha * m->alpha;
    vec3 h = normalize(add(wc, wo));
    vec3 t, b;
    tangent_frame(n, &t, &b);
    double hx = dot(h, t), hy = dot(h, b), hz = dot(h, n);
    double c2 = hz * hz;
    *u1 = (1.0 - c2) / (1.0 + c2 * (a2 - 1.0));
    double a = atan2(hy, hx) / (2.0 * PI);
    *u2 = a < 0.0 ? a + 1.0 : a;
}

/* ------------------------------------------------------------------------- */
/* camera                                                                    */
/* ------------------------------------------------------------------------- */

static vec3 camera_dir(const oscene *s, int px, int py, double jx, double jy) {
    double sx = (2.0 * (px + jx) / s->W - 1.0) * s->hw;
    double sy = (1.0 - 2.0 * (py + jy) / s->H) * s->hh;
    return normalize(add(add(s->cam_fwd, scale(s->cam_right, sx)), scale(s->cam_up, sy)));
}

/* pixel index of the projection of p, or -1; *cos_c = cosine to the axis */
static int camera_project(const oscene *s, vec3 p, double *cos_c) {
    vec3 v = sub(p, s->cam_pos);
    double z = dot(v, s->cam_fwd);
    if (z <= 0.0) return -1;
    double sx = dot(v, s->cam_right) / z, sy = dot(v, s->cam_up) / z;
    double fx = (sx / s->hw + 1.0) * 0.5 * s->W;
    double fy = (1.0 - sy / s->hh) * 0.5 * s->H;
    if (!(fx >= 0.0 && fx < s->W && fy >= 0.0 && fy < s->H)) return -1;
    int px = (int)floor(fx), py = (int)floor(fy);
    if (px >= s->W) px = s->W - 1;
    if (py >= s->H) py = s->H - 1;
    *cos_c = z / length(v);
    return py * s->W + px;
}

/* ------------------------------------------------------------------------- */
/* path contribution f (Eq. pathcontribution with the camera importance of   */
/* a pinhole with a box pixel filter), visibility excluded                    */
/* ------------------------------------------------------------------------- */

static vec3 path_throughput(const oscene *s, const vtx *x, int k, int *pix) {
    double cc;
    *pix = camera_project(s, x[1].p, &cc);
    if (*pix < 0) return v3(0, 0, 0);
    vec3 d01 = sub(x[0].p, x[1].p);
    double r2 = dot(d01, d01);
    double c1 = dot(x[1].n, d01) / sqrt(r2);
    if (c1 <= 0.0) return v3(0, 0, 0);
    double We = 1.0 / (s->pix_area * cc * cc * cc);
    vec3 f = v3(We * c1 / r2, We * c1 / r2, We * c1 / r2);
    for (int j = 1; j <= k - 2; ++j) {
        vec3 wi = normalize(sub(x[j - 1].p, x[j].p));
        vec3 e = sub(x[j + 1].p, x[j].p);
        double r2e = dot(e, e);
        vec3 wo = scale(e, 1.0 / sqrt(r2e));
        vec3 rho = bsdf_eval(x[j].mat, x[j].n, wi, wo);
        if (is_zero3(rho)) return v3(0, 0, 0);
        double ca = dot(x[j].n, wo), cb = -dot(x[j + 1].n, wo);
        if (ca <= 0.0 || cb <= 0.0) return v3(0, 0, 0);
        f = scale(mul(f, rho), ca * cb / r2e);
    }
    const material *em = x[k - 1].mat;
    f = mul(f, em->emission);
    return f;
}

/* ------------------------------------------------------------------------- */
/* technique densities and the balance-heuristic denominator (Sec. 4.3):     */
/* forward products along the camera-to-light direction (pE) and backward    */
/* products along the light-to-camera direction (pL)                          */
/* ------------------------------------------------------------------------- */

static double area_from_dir(double pdf_w, vec3 from, const vtx *to) {
    vec3 e = sub(to->p, from);
    double r2 = dot(e, e);
    double c = -dot(to->n, e) / sqrt(r2);
    if (c <= 0.0) return 0.0;
    return pdf_w * c / r2;
}

static double pdf_camera_area(const oscene *s, const vtx *x1) {
    double cc;
    if (camera_project(s, x1->p, &cc) < 0) return 0.0;
    vec3 d = sub(s->cam_pos, x1->p);
    double r2 = dot(d, d);
    double c1 = dot(x1->n, d) / sqrt(r2);
    if (c1 <= 0.0) return 0.0;
    double film_area = s->pix_area * s->W * s->H;
    return c1 / r2 / (film_area * cc * cc * cc);
}

/* area density of x[to] when sampled from x[at] conditioned on x[cond] */
static double step_pdf(const vtx *x, int cond, int at, int to) {
    vec3 wc = normalize(sub(x[cond].p, x[at].p));
    vec3 wo = normalize(sub(x[to].p, x[at].p));
    return area_from_dir(bsdf_pdf(x[at].mat, x[at].n, wc, wo), x[at].p, &x[to]);
}

typedef struct { int t1, t2, t3, t7, t4, t5, t6; } techmask;

/* ------------------------------------------------------------------------- */
/* ghost crossings (Sec. 3.3, 4.2): where an edge of a frame-g path passes   */
/* through the edited object's pose in the other frame                        */
/* ------------------------------------------------------------------------- */

typedef struct { vec3 p, n; } gcross;

/* every crossing of the open segment a-b of frame g with the ghost (the
 * dynamic object at its pose of the other frame), up to max */
static int ghost_crossings(const oscene *s, int g, vec3 a, vec3 b, gcross *out, int max) {
    if (!s->motion || s->n_dyn == 0) return 0;
    const int go = 3 - g;
    vec3 e = sub(b, a);
    double dist = length(e);
    vec3 d = scale(e, 1.0 / dist);
    const double tmin = s->eps, tmax = dist - s->eps;
    const bvh *bv = &s->dyn_bvh[go];
    int n = 0;
    int stack[128];
    int sp = 0;
    if (bv->n_nodes == 0) return 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bvh_node *nd = &bv->nodes[stack[--sp]];
        if (!ray_box(a, d, nd->lo, nd->hi, tmin, tmax)) continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; ++i) {
                int lp = bv->index[i];
                double t, u, v;
                const tri *tr = &s->dyn_world[go][lp];
                if (ray_tri(a, d, tr, &t, &u, &v) && t > tmin && t < tmax && n < max) {
                    out[n].p = add(a, scale(d, t));
                    out[n].n = tri_normal(tr);
                    ++n;
                }
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return n;
}

/* area density of x1 reached by the ray from o through the ghost point c,
 * c sampled by area with density pD (Eq. vertex1pdf) */
static double ghost_ray_pdf(double pD, vec3 o, const gcross *c, const vtx *x1) {
    vec3 w = normalize(sub(x1->p, o));
    double cg = fabs(dot(c->n, w)), c1 = fabs(dot(x1->n, w));
    vec3 og = sub(c->p, o), o1 = sub(x1->p, o);
    if (cg <= 0.0) return 0.0;
    return pD * dot(og, og) / cg * c1 / dot(o1, o1);
}

/* the terms of the balance-heuristic denominator, summed in order and, when
 * terms != NULL, recorded one by one (technique id and density) */
typedef struct {
    double sum;
    int n, cap;
    double *terms;
    int *tech;
} termacc;

static void add_term(termacc *a, int tech, double p) {
    a->sum += p;
    if (a->terms && a->n < a->cap) {
        a->terms[a->n] = p;
        a->tech[a->n] = tech;
    }
    a->n++;
}

/* sum over the enabled techniques that produce x of their per-root densities */
static double mis_terms(const oscene *s, int g, const vtx *x, int k, techmask tm, termacc *acc);

static double mis_denominator(const oscene *s, int g, const vtx *x, int k, techmask tm) {
    termacc acc = {0.0, 0, 0, NULL, NULL};
    return mis_terms(s, g, x, k, tm, &acc);
}

static double mis_terms(const oscene *s, int g, const vtx *x, int k, techmask tm, termacc *acc) {
    double pE[16], pL[16];
    double pD = 1.0 / s->dyn_area, pLi = 1.0 / s->emit_area;
    if (k == 2) {
        if (tm.t7) add_term(acc, 7, pdf_camera_area(s, &x[1]));
        return acc->sum;
    }
    pE[1] = pdf_camera_area(s, &x[1]);
    for (int j = 2; j <= k - 2; ++j) pE[j] = step_pdf(x, j - 2, j - 1, j);
    for (int j = 1; j <= k - 3; ++j) pL[j] = step_pdf(x, j + 2, j + 1, j);
    if (tm.t7) {
        double p = pLi;
        for (int j = 1; j <= k - 2; ++j) p *= pE[j];
        add_term(acc, 7, p);
    }
    for (int i = 1; i <= k - 2; ++i) {
        if (!x[i].dyn) continue;
        if (i == k - 2) {                     /* (1) dynamic from emitter */
            if (!tm.t1) continue;
            double p = pD * pLi;
            for (int j = 1; j <= k - 3; ++j) p *= pL[j];
            add_term(acc, 1, p);
        } else if (i == 1) {                  /* (2) dynamic from sensor */
            if (!tm.t2) continue;
            double p = pD * pLi;
            for (int j = 2; j <= k - 2; ++j) p *= pE[j];
            add_term(acc, 2, p);
        } else {                              /* (3) dynamic two ends */
            if (!tm.t3) continue;
            vec3 w = normalize(sub(x[i + 1].p, x[i].p));
            double p = pD * pLi * area_from_dir(cosine_pdf(x[i].n, w), x[i].p, &x[i + 1]);
            for (int j = i + 2; j <= k - 2; ++j) p *= pE[j];
            for (int j = 1; j <= i - 1; ++j) p *= pL[j];
            add_term(acc, 3, p);
        }
    }
    /* (4)-(6): one term per ghost crossing of an edge; (5) on the first edge,
     * (4) on the last, (6) in between (Sec. 4.2, Eq. vertex1pdf and the
     * two-ends geometric term with a uniform direction density 1 / (4 pi)) */
    if ((tm.t4 || tm.t5 || tm.t6) && s->motion && k >= 3) {
        for (int j = 0; j <= k - 2; ++j) {
            const int kind = (j == 0) ? 5 : (j == k - 2) ? 4 : 6;
            if ((kind == 4 && !tm.t4) || (kind == 5 && !tm.t5) || (kind == 6 && !tm.t6)) continue;
            gcross cr[8];
            int nc = ghost_crossings(s, g, x[j].p, x[j + 1].p, cr, 8);
            for (int c = 0; c < nc; ++c) {
                double p;
                if (kind == 4) {
                    p = pLi * ghost_ray_pdf(pD, x[k - 1].p, &cr[c], &x[k - 2]);
                    for (int m = 1; m <= k - 3; ++m) p *= pL[m];
                } else if (kind == 5) {
                    p = pLi * ghost_ray_pdf(pD, x[0].p, &cr[c], &x[1]);
                    for (int m = 2; m <= k - 2; ++m) p *= pE[m];
                } else {
                    vec3 w = normalize(sub(x[j + 1].p, x[j].p));
                    vec3 e = sub(x[j + 1].p, x[j].p);
                    double cg = fabs(dot(cr[c].n, w));
                    if (cg <= 0.0) continue;
                    p = pD * pLi * fabs(dot(x[j].n, w)) * fabs(dot(x[j + 1].n, w)) / (cg * dot(e, e)) /
                        (4.0 * PI);
                    for (int m = 1; m <= j - 1; ++m) p *= pL[m];
                    for (int m = j + 2; m <= k - 2; ++m) p *= pE[m];
                }
                add_term(acc, kind, p);
            }
        }
    }
    return acc->sum;
}

/* ------------------------------------------------------------------------- */
/* visibility                                                                */
/* ------------------------------------------------------------------------- */

static int segment_clear(const oscene *s, int g, const vtx *a, const vtx *b, int dyn_only) {
    vec3 e = sub(b->p, a->p);
    double dist = length(e);
    vec3 d = scale(e, 1.0 / dist);
    hitrec h;
    return !scene_trace(s, g, a->p, d, s->eps, dist - s->eps, a->prim, b->prim, 1, dyn_only, &h);
}

/* closest surface hit from vertex a along d in frame g */
static int trace_next(const oscene *s, int g, const vtx *a, vec3 d, vtx *out) {
    hitrec h;
    if (!scene_trace(s, g, a->p, d, s->eps, INFINITY, a->prim, -1, 0, 0, &h)) return 0;
    *out = make_vertex(s, g, h.prim, h.b1, h.b2);
    return 1;
}

/* a path of frame g is static when it has no dynamic vertex and no edge
 * passes through the object's pose in the other frame (Sec. 3.3) */
static int path_is_static(const oscene *s, int g, const vtx *x, int k) {
    for (int i = 0; i < k; ++i)
        if (x[i].dyn) return 0;
    if (!s->motion) return 1;
    int go = 3 - g;
    for (int j = 0; j + 1 < k; ++j)
        if (!segment_clear(s, go, &x[j], &x[j + 1], 1)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* path mapping (Sec. 5)                                                     */
/* ------------------------------------------------------------------------- */

enum {
    MAP_ACCEPT = 0,
    MAP_INVALID = 1,        /* mapped path has zero contribution */
    MAP_REJECT_NODYN = 2,   /* only dynamic edges: the identity image is blocked */
    MAP_REJECT_MULTI = 3,   /* more than one dynamic vertex */
    MAP_REJECT_INVERT = 4,  /* the inverse mapping would not replay this step */
    MAP_REJECT_JAC = 5,
    MAP_OFF = 6             /* path mapping switched off: each frame estimates its own paths */
};

static int reconnect_ok(const oscene *s, const vtx *a, const vtx *ap, const vtx *b) {
    if (b->dyn) return 0;
    double r = fmin(fmin(roughness(a->mat), roughness(ap->mat)), roughness(b->mat));
    if (!(r >= s->alpha_min)) return 0;
    double d = fmin(length(sub(ap->p, b->p)), length(sub(a->p, b->p)));
    return d >= s->d_min;
}

typedef struct {
    int status;
    double J;
    int replayed[16];       /* y[j] produced by replay */
} mapinfo;

/* one walk step of the mapping: x[b] was reached from x[a]; the sampling at
 * x[a] was conditioned on x[c] (c < 0: cosine sampling).  Fills y[b]. */
static int map_step(const oscene *s, int g2, const vtx *x, vtx *y, int a, int b, int c,
                    mapinfo *mi) {
    if (same_point(y[a].p, x[a].p)) {           /* predecessor unchanged */
        y[b] = x[b];
        return MAP_ACCEPT;
    }
    if (reconnect_ok(s, &x[a], &y[a], &x[b])) { /* keep vertex the same */
        y[b] = x[b];
        return MAP_ACCEPT;
    }
    /* random-seed replay: recover the step's random numbers, reuse them */
    vec3 wo = normalize(sub(x[b].p, x[a].p));
    double u1, u2;
    vec3 w2;
    if (c < 0) {
        cosine_inverse(x[a].n, wo, &u1, &u2);
        w2 = cosine_dir(y[a].n, u1, u2);
        if (dot(y[a].n, w2) <= 0.0) return MAP_INVALID;
    } else {
        vec3 wc = normalize(sub(x[c].p, x[a].p));
        bsdf_inverse(x[a].mat, x[a].n, wc, wo, &u1, &u2);
        vec3 wc2 = normalize(sub(y[c].p, y[a].p));
        if (!bsdf_sample(y[a].mat, y[a].n, wc2, u1, u2, &w2)) return MAP_INVALID;
    }
    vtx nb;
    if (!trace_next(s, g2, &y[a], w2, &nb)) return MAP_INVALID;
    if (dot(nb.n, w2) >= 0.0) return MAP_INVALID;  /* back face */
    if (nb.dyn) return MAP_REJECT_MULTI;
    if (reconnect_ok(s, &y[a], &x[a], &nb)) return MAP_REJECT_INVERT;
    y[b] = nb;
    mi->replayed[b] = 1;
    /* area-measure Jacobian of the replayed vertex (reading R1) */
    double px, py;
    if (c < 0) {
        px = area_from_dir(cosine_pdf(x[a].n, wo), x[a].p, &x[b]);
        py = area_from_dir(cosine_pdf(y[a].n, w2), y[a].p, &y[b]);
    } else {
        px = step_pdf(x, c, a, b);
        py = step_pdf(y, c, a, b);
    }
    if (!(px > 0.0) || !(py > 0.0)) return MAP_INVALID;
    mi->J *= px / py;
    return MAP_ACCEPT;
}

/* the first edge of a frame-g path is dynamic: x_1 lies on the object or the
 * camera ray to x_1 crosses the ghost (the object at its other-frame pose) */
static int first_edge_dynamic(const oscene *s, int g, const vtx *x, int k) {
    if (k < 2 || !s->motion) return 0;
    if (x[1].dyn) return 1;
    return !segment_clear(s, 3 - g, &x[0], &x[1], 1);
}

/* camera replay (Sec. 5, "Mapping between the dynamic and ghost pair": the
 * same camera direction in both frames): y_1 is the first hit of the camera
 * ray through x_1 in frame g2 (area Jacobian: the ratio of the camera
 * densities), then the light side walks as for technique (2).  The class of
 * paths with a dynamic first edge is closed under this map. */
static void map_camera(const oscene *s, int g, int g2, const vtx *x, int k, vtx *y, mapinfo *mi) {
    for (int j = 2; j <= k - 2; ++j)
        if (x[j].dyn) { mi->status = MAP_REJECT_MULTI; return; }
    vec3 w = normalize(sub(x[1].p, x[0].p));
    vtx y1;
    if (!trace_next(s, g2, &y[0], w, &y1) || dot(y1.n, w) >= 0.0) { mi->status = MAP_INVALID; return; }
    y[1] = y1;
    mi->replayed[1] = 1;
    double px = pdf_camera_area(s, &x[1]), py = pdf_camera_area(s, &y[1]);
    if (!(px > 0.0) || !(py > 0.0)) { mi->status = MAP_INVALID; return; }
    mi->J *= px / py;
    for (int b = 2; b <= k - 2; ++b) {
        int st = map_step(s, g2, x, y, b - 1, b, b - 2, mi);
        if (st != MAP_ACCEPT) { mi->status = st; return; }
    }
    if (!first_edge_dynamic(s, g2, y, k)) { mi->status = MAP_REJECT_INVERT; return; }
    (void)g;
    if (!(mi->J <= s->jac_max && 1.0 / mi->J <= s->jac_max)) { mi->status = MAP_REJECT_JAC; return; }
    mi->status = MAP_ACCEPT;
}

/* map the frame-g path x (k vertices) into frame g2 */
static void map_path(const oscene *s, int g, int g2, const vtx *x, int k, vtx *y, mapinfo *mi) {
    mi->J = 1.0;
    for (int j = 0; j < k; ++j) mi->replayed[j] = 0;
    for (int j = 0; j < k; ++j) y[j] = x[j];
    if (s->map_mode == 2 && first_edge_dynamic(s, g, x, k)) {
        map_camera(s, g, g2, x, k, y, mi);
        return;
    }
    int nd = 0, i = -1;
    for (int j = 1; j <= k - 2; ++j)
        if (x[j].dyn) { ++nd; i = j; }
    if (nd == 0) { mi->status = MAP_REJECT_NODYN; return; }
    if (nd > 1) { mi->status = MAP_REJECT_MULTI; return; }
    /* transform with object movement: same point of the object in frame g2 */
    y[i] = make_vertex(s, g2, x[i].prim, x[i].b1, x[i].b2);
    int st;
    if (i == k - 2) {
        /* (1): the light end is fixed; walk the eye side from x_D, first step
         * conditioned on the emitter vertex */
        for (int b = i - 1; b >= 1; --b) {
            int c = (b == i - 1) ? k - 1 : b + 2;
            st = map_step(s, g2, x, y, b + 1, b, c, mi);
            if (st != MAP_ACCEPT) { mi->status = st; return; }
        }
    } else if (i == 1) {
        /* (2): the eye end is the camera; walk the light side, first step
         * conditioned on the camera */
        for (int b = 2; b <= k - 2; ++b) {
            st = map_step(s, g2, x, y, b - 1, b, b - 2, mi);
            if (st != MAP_ACCEPT) { mi->status = st; return; }
        }
    } else {
        /* (3): light side first (cosine step), then the eye side conditioned on
         * the first light-side vertex */
        for (int b = i + 1; b <= k - 2; ++b) {
            int c = (b == i + 1) ? -1 : b - 2;
            st = map_step(s, g2, x, y, b - 1, b, c, mi);
            if (st != MAP_ACCEPT) { mi->status = st; return; }
        }
        for (int b = i - 1; b >= 1; --b) {
            st = map_step(s, g2, x, y, b + 1, b, b + 2, mi);
            if (st != MAP_ACCEPT) { mi->status = st; return; }
        }
    }
    if (!(mi->J <= s->jac_max && 1.0 / mi->J <= s->jac_max)) {
        mi->status = MAP_REJECT_JAC;
        return;
    }
    /* the image must stay outside the camera-replay class, else the inverse
     * map would differ */
    if (s->map_mode == 2 && first_edge_dynamic(s, g2, y, k)) {
        mi->status = MAP_REJECT_INVERT;
        return;
    }
    mi->status = MAP_ACCEPT;
}

/* visibility of the mapped path in frame g2: an edge traced by a replay step
 * is visible by construction (closest hit); an edge whose two ends are
 * unchanged is re-checked against the dynamic object only (the static scene
 * is the same in both frames); every other edge gets a full check */
static int mapped_visible(const oscene *s, int g2, const vtx *x, const vtx *y, int k,
                          const mapinfo *mi) {
    int i = -1;
    for (int j = 1; j <= k - 2; ++j)
        if (y[j].dyn) i = j;
    for (int j = 0; j + 1 < k; ++j) {
        /* the end of edge (j, j+1) farther from the dynamic vertex */
        int far = (j + 1 <= i) ? j : j + 1;
        if (mi->replayed[far]) continue;
        int unchanged = same_point(x[j].p, y[j].p) && same_point(x[j + 1].p, y[j + 1].p);
        if (!segment_clear(s, g2, &y[j], &y[j + 1], unchanged)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* evaluation of one base path: two-way mapped, MIS-weighted contribution    */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t root;
    int32_t tech, frame, sa, sb;     /* strategy: (t', s') or path length */
    int32_t pix_a, pix_b;
    double va[3], vb[3];
    int32_t status;
    double Pg, Py, J;
} orecord;

typedef struct {
    const oscene *s;
    double *img;            /* H*W*3 accumulation, may be NULL */
    orecord *rec;           /* records, may be NULL */
    int64_t max_rec;
    int64_t *n_rec;
    double N;               /* roots per technique per frame */
    techmask tm;
    int residual;           /* 0: primal (plain path tracing, no MIS) */
    int64_t counters[8];
    double vscale;          /* 0: none; else every emitted value is multiplied by it */
    int domain;             /* primal only: 0 all paths; else bit t-1 keeps the paths with a
                               dynamic vertex where technique t (1, 2, 3) would sample it */
} sink;

/* whether the path has a dynamic vertex at a position of a technique in
 * `domain` (Sec. 4.1: (1) next to the emitter, (2) next to the sensor,
 * (3) in between) */
static int in_domain(const vtx *x, int n, int domain) {
    for (int i = 1; i <= n - 2; ++i) {
        if (!x[i].dyn) continue;
        const int t = (i == n - 2) ? 1 : (i == 1) ? 2 : 3;
        if ((domain >> (t - 1)) & 1) return 1;
    }
    return 0;
}

static void emit(sink *k, uint32_t root, int tech, int g, int sa, int sb, int pa, vec3 va, int pb,
                 vec3 vb, int status, double Pg, double Py, double J) {
    if (k->vscale != 0.0) { va = scale(va, k->vscale); vb = scale(vb, k->vscale); }
    if (k->img) {
        if (pa >= 0) {
            k->img[3 * pa] += va.x; k->img[3 * pa + 1] += va.y; k->img[3 * pa + 2] += va.z;
        }
        if (pb >= 0) {
            k->img[3 * pb] += vb.x; k->img[3 * pb + 1] += vb.y; k->img[3 * pb + 2] += vb.z;
        }
    }
    if (k->rec && *k->n_rec < k->max_rec) {
        orecord *r = &k->rec[*k->n_rec];
        r->root = root; r->tech = tech; r->frame = g; r->sa = sa; r->sb = sb;
        r->pix_a = pa; r->pix_b = pb;
        r->va[0] = va.x; r->va[1] = va.y; r->va[2] = va.z;
        r->vb[0] = vb.x; r->vb[1] = vb.y; r->vb[2] = vb.z;
        r->status = status; r->Pg = Pg; r->Py = Py; r->J = J;
    }
    if (k->n_rec) ++*k->n_rec;
}

static int g_check_mode = 0;
static void mc_evaluate(sink *k, int g, const vtx *x, int n);

static void evaluate_path(sink *k, int g, const vtx *x, int n, uint32_t root, int tech, int sa,
                          int sb) {
    const oscene *s = k->s;
    if (g_check_mode) { mc_evaluate(k, g, x, n); return; }
    int pa;
    vec3 fx = path_throughput(s, x, n, &pa);
    if (is_zero3(fx)) return;
    if (!k->residual) {
        /* primal path tracing: a single technique, no MIS */
        if (k->domain && !in_domain(x, n, k->domain)) return;
        techmask only7 = {0, 0, 0, 1, 0, 0, 0};
        double p = mis_denominator(s, g, x, n, only7);
        emit(k, root, tech, g, sa, sb, pa, scale(fx, 1.0 / (k->N * p)), -1, v3(0, 0, 0), 0, p, 0,
             1);
        return;
    }
    if (tech == TECH_T7 && path_is_static(s, g, x, n)) { k->counters[0]++; return; }
    double Pg = mis_denominator(s, g, x, n, k->tm);
    double sign = (g == 2) ? 1.0 : -1.0;
    int g2 = 3 - g;
    vtx y[16];
    mapinfo mi;
    vec3 fy = v3(0, 0, 0);
    int pb = -1;
    double Py = 0.0;
    if (!s->motion) {
        for (int j = 0; j < n; ++j) {
            y[j] = x[j];
            if (y[j].kind == VK_SURFACE) y[j].mat = prim_mat(s, g2, y[j].prim);
        }
        mi.status = MAP_ACCEPT; mi.J = 1.0;
    } else if (s->map_mode == 0) {
        mi.status = MAP_OFF; mi.J = 0.0;
    } else {
        map_path(s, g, g2, x, n, y, &mi);
    }
    if (mi.status == MAP_ACCEPT) {
        if (s->motion && !mapped_visible(s, g2, x, y, n, &mi)) {
            mi.status = MAP_INVALID;
        } else {
            fy = path_throughput(s, y, n, &pb);
            if (is_zero3(fy)) mi.status = MAP_INVALID;
            else Py = mis_denominator(s, g2, y, n, k->tm);
            if (!(Py > 0.0)) mi.status = MAP_INVALID;
        }
    }
    k->counters[1 + (mi.status < 6 ? mi.status : 6)]++;
    if (mi.status == MAP_ACCEPT) {
        double J = mi.J;
        double den = k->N * (Pg + Py * J);
        emit(k, root, tech, g, sa, sb, pa, scale(fx, sign / den), pb, scale(fy, -sign * J / den),
             mi.status, Pg, Py, J);
    } else {
        emit(k, root, tech, g, sa, sb, pa, scale(fx, sign / (k->N * Pg)), -1, v3(0, 0, 0),
             mi.status, Pg, 0.0, 0.0);
    }
}

/* ------------------------------------------------------------------------- */
/* root sampling                                                             */
/* ------------------------------------------------------------------------- */

static int cdf_pick(const double *cdf, int n, double u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (u < cdf[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void tri_sample(double u1, double u2, double *b1, double *b2) {
    double sq = sqrt(u1);
    *b1 = sq * (1.0 - u2);
    *b2 = sq * u2;
}

static vtx sample_dynamic(const oscene *s, int g, rnd4 r) {
    int t = cdf_pick(s->dyn_cdf, s->n_dyn, r.u[0]);
    double b1, b2;
    tri_sample(r.u[1], r.u[2], &b1, &b2);
    return make_vertex(s, g, s->n_static + t, b1, b2);
}

static vtx sample_emitter(const oscene *s, int g, rnd4 r) {
    int t = cdf_pick(s->emit_cdf, s->n_emit, r.u[0]);
    double b1, b2;
    tri_sample(r.u[1], r.u[2], &b1, &b2);
    return make_vertex(s, g, s->emit_ids[t], b1, b2);
}

static int faces(const vtx *v, vec3 towards) {
    return dot(v->n, sub(towards, v->p)) > 0.0;
}

/* connection of a surface vertex to the pinhole */
static int camera_visible(const oscene *s, int g, const vtx *z) {
    vtx c = camera_vertex(s);
    double cc;
    if (camera_project(s, z->p, &cc) < 0) return 0;
    if (!faces(z, c.p)) return 0;
    return segment_clear(s, g, z, &c, 0);
}

/* next-event estimation: emitter vertex connected to z */
static int nee(const oscene *s, int g, const vtx *z, rnd4 r, vtx *L) {
    *L = sample_emitter(s, g, r);
    if (!faces(z, L->p) || !faces(L, z->p)) return 0;
    return segment_clear(s, g, z, L, 0);
}

/* extend a walk from `at` (previous vertex `prev`) with random numbers r */
static int walk_step(const oscene *s, int g, const vtx *prev, const vtx *at, rnd4 r, vtx *out) {
    vec3 wc = normalize(sub(prev->p, at->p));
    vec3 wo;
    if (!bsdf_sample(at->mat, at->n, wc, r.u[0], r.u[1], &wo)) return 0;
    if (!trace_next(s, g, at, wo, out)) return 0;
    if (dot(out->n, wo) >= 0.0) return 0;      /* back face: one-sided surfaces */
    return 1;
}

/* (1) dynamic from emitter */
static void root_T1(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    int D = s->max_depth;
    vtx xD = sample_dynamic(s, g, draw(seed, root, TECH_T1, g, SIDE_ROOT, 0));
    vtx xL;
    if (!nee(s, g, &xD, draw(seed, root, TECH_T1, g, SIDE_NEE, 0), &xL)) return;
    if (is_black(xD.mat)) return;
    vtx z[16];                    /* z[0] = xD, z[1..] eye-side walk */
    z[0] = xD;
    vtx path[16];
    for (int t = 0; t <= D - 2; ++t) {
        if (t > 0) {
            const vtx *prev = (t == 1) ? &xL : &z[t - 2];
            if (!walk_step(s, g, prev, &z[t - 1], draw(seed, root, TECH_T1, g, SIDE_EYE, t),
                           &z[t]))
                break;
            if (is_black(z[t].mat)) break;
        }
        if (camera_visible(s, g, &z[t])) {
            int n = t + 3;
            path[0] = camera_vertex(s);
            for (int j = 0; j <= t; ++j) path[1 + j] = z[t - j];
            path[n - 1] = xL;
            evaluate_path(k, g, path, n, root, TECH_T1, t, 0);
        }
    }
}

/* (2) dynamic from sensor */
static void root_T2(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    int D = s->max_depth;
    vtx xD = sample_dynamic(s, g, draw(seed, root, TECH_T2, g, SIDE_ROOT, 0));
    if (is_black(xD.mat)) return;
    if (!camera_visible(s, g, &xD)) return;
    vtx cam = camera_vertex(s);
    vtx yv[16];                   /* yv[0] = xD, yv[1..] light-side walk */
    yv[0] = xD;
    vtx path[16];
    for (int t = 1; t <= D - 2; ++t) {
        const vtx *prev = (t == 1) ? &cam : &yv[t - 2];
        if (!walk_step(s, g, prev, &yv[t - 1], draw(seed, root, TECH_T2, g, SIDE_LIGHT, t),
                       &yv[t]))
            break;
        if (is_black(yv[t].mat)) break;
        vtx L;
        if (nee(s, g, &yv[t], draw(seed, root, TECH_T2, g, SIDE_NEE, t), &L)) {
            int n = t + 3;
            path[0] = cam;
            for (int j = 0; j <= t; ++j) path[1 + j] = yv[j];
            path[n - 1] = L;
            evaluate_path(k, g, path, n, root, TECH_T2, 0, t);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* learned proposal for the light-side direction of technique (3)            */
/*                                                                           */
/* Not in the paper (which lists better importance sampling as future work,  */
/* Sec. 7): a small network maps the object-space position and normal of x_D */
/* to an 8-lobe von Mises-Fisher mixture over directions; technique (3)      */
/* draws its first light-side direction from the defensive one-sample        */
/* mixture q = 1/2 p_cos + 1/2 sum_j pi_j vMF_j and multiplies the values of */
/* the root's paths by p_cos / q.  The balance-heuristic weights stay those  */
/* of the plain techniques, so any network leaves the estimator unbiased.    */
/*                                                                           */
/* Inference runs on integers: inputs in [-127, 127], weights in             */
/* [-127, 127], hidden activations in [0, 255] requantised by a right shift  */
/* with round-half-even; every sum stays below 2^24, so any summation order  */
/* gives the same result.                                                    */
/* ------------------------------------------------------------------------- */

enum { G_IN = 80, G_HID = 64, G_OUT = 48, G_LOBES = 8, G_LAYERS = 5 };
static const int G_DIM_IN[G_LAYERS] = {G_IN, G_HID, G_HID, G_HID, G_HID};
static const int G_DIM_OUT[G_LAYERS] = {G_HID, G_HID, G_HID, G_HID, G_OUT};
static const int G_OFF[G_LAYERS + 1] = {0, 5120, 9216, 13312, 17408, 20480};

typedef struct oguide_s {
    int32_t W[20480];            /* layer l: [out][in] at G_OFF[l] */
    int shift[4];                /* hidden requantisation right shifts */
    int out_exp;                 /* output = z * 2^-out_exp */
    double center[3], inv_half[3];
} oguide;

/* input features of (p, n), object space: for each coordinate c of
 * u = clamp((p - center) * inv_half, -1, 1), then of n, the pairs
 * sin(2^f pi c), cos(2^f pi c) for f = 0..5 (72 features), then u and n
 * (6 features), quantised to rint(128 e) clamped to [-127, 127]; feature 78
 * is the constant 127 and feature 79 is 0 */
static void guide_encode(const double center[3], const double inv_half[3], vec3 p, vec3 n,
                         int32_t m[G_IN]) {
    double u[3] = {(p.x - center[0]) * inv_half[0], (p.y - center[1]) * inv_half[1],
                   (p.z - center[2]) * inv_half[2]};
    double nn[3] = {n.x, n.y, n.z};
    double e[78];
    int i = 0;
    for (int c = 0; c < 3; ++c) u[c] = fmin(1.0, fmax(-1.0, u[c]));
    for (int v = 0; v < 2; ++v)
        for (int c = 0; c < 3; ++c)
            for (int f = 0; f < 6; ++f) {
                double a = ldexp(v == 0 ? u[c] : nn[c], f);
                e[i++] = sin(PI * a);
                e[i++] = cos(PI * a);
            }
    for (int c = 0; c < 3; ++c) e[i++] = u[c];
    for (int c = 0; c < 3; ++c) e[i++] = nn[c];
    for (int j = 0; j < 78; ++j) {
        double q = nearbyint(128.0 * e[j]);
        m[j] = (int32_t)fmin(127.0, fmax(-127.0, q));
    }
    m[78] = 127;
    m[79] = 0;
}

/* integer forward pass: 4 hidden layers with ReLU, then the output layer */
static void guide_forward(const oguide *gd, const int32_t m_in[G_IN], double out[G_OUT]) {
    int64_t a[G_IN], h[G_HID];
    for (int i = 0; i < G_IN; ++i) a[i] = m_in[i];
    for (int l = 0; l < G_LAYERS; ++l) {
        const int K = G_DIM_IN[l], N = G_DIM_OUT[l];
        const int32_t *W = gd->W + G_OFF[l];
        for (int o = 0; o < N; ++o) {
            int64_t z = 0;
            for (int i = 0; i < K; ++i) z += (int64_t)W[o * K + i] * a[i];
            if (l < G_LAYERS - 1) {
                double q = nearbyint(ldexp((double)z, -gd->shift[l]));
                h[o] = (int64_t)fmin(255.0, fmax(0.0, q));
            } else {
                out[o] = ldexp((double)z, -gd->out_exp);
            }
        }
        if (l < G_LAYERS - 1)
            for (int o = 0; o < N; ++o) a[o] = h[o];
    }
}

/* lobe j reads outputs 5j..5j+4: direction (3, normalised), log kappa
 * (clamped to [-4, 6.2]) and the mixture logit (softmax) */
static void guide_mixture(const double o[G_OUT], vec3 mu[G_LOBES], double kappa[G_LOBES],
                          double pi[G_LOBES]) {
    double mx = o[4];
    for (int j = 1; j < G_LOBES; ++j) mx = fmax(mx, o[5 * j + 4]);
    double sum = 0.0;
    for (int j = 0; j < G_LOBES; ++j) { pi[j] = exp(o[5 * j + 4] - mx); sum += pi[j]; }
    for (int j = 0; j < G_LOBES; ++j) {
        pi[j] /= sum;
        vec3 m = v3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
        double l = length(m);
        mu[j] = l > 1e-12 ? scale(m, 1.0 / l) : v3(0.0, 0.0, 1.0);
        kappa[j] = exp(fmin(6.2, fmax(-4.0, o[5 * j + 3])));
    }
}

/* von Mises-Fisher density on the unit sphere:
 * kappa / (2 pi (1 - exp(-2 kappa))) exp(kappa (mu.w - 1)) */
static double vmf_pdf(vec3 mu, double kappa, vec3 w) {
    return kappa / (2.0 * PI * -expm1(-2.0 * kappa)) * exp(kappa * (dot(mu, w) - 1.0));
}

/* inversion sampling (Jakob 2012, "Numerically stable sampling of the von
 * Mises Fisher distribution on S^2"): the cosine to mu is
 * 1 + log(u1 + (1 - u1) exp(-2 kappa)) / kappa, the azimuth 2 pi u2 in the
 * tangent frame of mu */
static vec3 vmf_sample(vec3 mu, double kappa, double u1, double u2) {
    double c = 1.0 + log(u1 + (1.0 - u1) * exp(-2.0 * kappa)) / kappa;
    c = fmin(1.0, fmax(-1.0, c));
    double s = sqrt(fmax(0.0, 1.0 - c * c)), phi = 2.0 * PI * u2;
    vec3 t, b;
    tangent_frame(mu, &t, &b);
    return add(add(scale(t, s * cos(phi)), scale(b, s * sin(phi))), scale(mu, c));
}

/* linear part of a 3x4 row-major transform and of its transpose */
static vec3 lin_M(const double *M, vec3 a) {
    return v3(M[0] * a.x + M[1] * a.y + M[2] * a.z, M[4] * a.x + M[5] * a.y + M[6] * a.z,
              M[8] * a.x + M[9] * a.y + M[10] * a.z);
}
static vec3 lin_MT(const double *M, vec3 a) {
    return v3(M[0] * a.x + M[4] * a.y + M[8] * a.z, M[1] * a.x + M[5] * a.y + M[9] * a.z,
              M[2] * a.x + M[6] * a.y + M[10] * a.z);
}

/* the first light-side direction of technique (3) at x_D in frame g, drawn
 * with the numbers r of that step: u[2] < 1/2 picks the cosine component,
 * else lobe j with (2 u[2] - 1) against the cumulative mixture weights;
 * *ratio receives p_cos(w) / q(w) */
static vec3 guided_direction(const oscene *s, int g, const vtx *xD, rnd4 r, double *ratio) {
    const oguide *gd = s->guide;
    const tri *t = &s->dyn_obj[xD->prim - s->n_static];
    const double *M = s->M[g][s->dyn_inst[xD->prim - s->n_static]];
    double b0 = 1.0 - xD->b1 - xD->b2;
    vec3 p_obj = add(add(scale(t->v0, b0), scale(t->v1, xD->b1)), scale(t->v2, xD->b2));
    vec3 nd = tri_normal(t);
    vec3 n_obj = v3((float)nd.x, (float)nd.y, (float)nd.z);   /* the normal as stored in float */
    int32_t m[G_IN];
    guide_encode(gd->center, gd->inv_half, p_obj, n_obj, m);
    double o[G_OUT];
    guide_forward(gd, m, o);
    vec3 mu[G_LOBES];
    double kappa[G_LOBES], pi[G_LOBES];
    guide_mixture(o, mu, kappa, pi);
    vec3 w, wl;
    if (r.u[2] < 0.5) {
        w = cosine_dir(xD->n, r.u[0], r.u[1]);
        wl = lin_MT(M, w);
    } else {
        double v = 2.0 * r.u[2] - 1.0, acc = 0.0;
        int j = G_LOBES - 1;
        for (int i = 0; i < G_LOBES; ++i) {
            acc += pi[i];
            if (v < acc) { j = i; break; }
        }
        wl = vmf_sample(mu[j], kappa[j], r.u[0], r.u[1]);
        w = lin_M(M, wl);
    }
    double pc = cosine_pdf(xD->n, w), pv = 0.0;
    for (int j = 0; j < G_LOBES; ++j) pv += pi[j] * vmf_pdf(mu[j], kappa[j], wl);
    *ratio = pc / (0.5 * pc + 0.5 * pv);
    return w;
}

/* the float network of the same shape for training: ReLU hidden layers, no
 * biases besides the constant input feature; out[n][48] */
static void mlp_forward_float(const double *W, const double *x, double *acts[G_LAYERS + 1]) {
    for (int i = 0; i < G_IN; ++i) acts[0][i] = x[i];
    for (int l = 0; l < G_LAYERS; ++l) {
        const int K = G_DIM_IN[l], N = G_DIM_OUT[l];
        for (int o = 0; o < N; ++o) {
            double z = 0.0;
            for (int i = 0; i < K; ++i) z += W[G_OFF[l] + o * K + i] * acts[l][i];
            acts[l + 1][o] = (l < G_LAYERS - 1) ? fmax(z, 0.0) : z;
        }
    }
}

/* loss of one sample, -wt log sum_j pi_j vMF_j(w), and its gradient with
 * respect to the 48 outputs (added into dout, scaled by `scale_`); the sum
 * is taken in log space, log pi_j + log vMF_j(w), so that no lobe
 * underflows */
static double mixture_nll(const double o[G_OUT], vec3 w, double wt, double scale_, double *dout) {
    vec3 mu[G_LOBES];
    double kappa[G_LOBES], pi[G_LOBES], lv[G_LOBES], lpi[G_LOBES];
    guide_mixture(o, mu, kappa, pi);
    double lmax = o[4];
    for (int j = 1; j < G_LOBES; ++j) lmax = fmax(lmax, o[5 * j + 4]);
    double ls = 0.0;
    for (int j = 0; j < G_LOBES; ++j) ls += exp(o[5 * j + 4] - lmax);
    double lse = lmax + log(ls);
    double mx = -INFINITY;
    for (int j = 0; j < G_LOBES; ++j) {
        double k = kappa[j];
        lpi[j] = o[5 * j + 4] - lse;
        lv[j] = lpi[j] + log(k) - log(2.0 * PI) - log(-expm1(-2.0 * k)) + k * (dot(mu[j], w) - 1.0);
        mx = fmax(mx, lv[j]);
    }
    double s = 0.0;
    for (int j = 0; j < G_LOBES; ++j) s += exp(lv[j] - mx);
    double logq = mx + log(s);
    if (dout) {
        for (int j = 0; j < G_LOBES; ++j) {
            double resp = exp(lv[j] - logq);
            double c = dot(mu[j], w);
            dout[5 * j + 4] += scale_ * -wt * (resp - exp(lpi[j]));
            double kr = o[5 * j + 3];
            if (kr > -4.0 && kr < 6.2) {
                double k = kappa[j];
                double dlogv = 1.0 / k - 2.0 * exp(-2.0 * k) / -expm1(-2.0 * k) + (c - 1.0);
                dout[5 * j + 3] += scale_ * -wt * resp * k * dlogv;
            }
            vec3 m = v3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
            double l = length(m);
            if (l > 1e-12) {
                vec3 gdir = scale(sub(w, scale(mu[j], c)), kappa[j] / l);
                dout[5 * j + 0] += scale_ * -wt * resp * gdir.x;
                dout[5 * j + 1] += scale_ * -wt * resp * gdir.y;
                dout[5 * j + 2] += scale_ * -wt * resp * gdir.z;
            }
        }
    }
    return -wt * logq;
}

/* (3) dynamic two ends */
static void root_T3(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    int D = s->max_depth;
    if (D < 4) return;
    vtx xD = sample_dynamic(s, g, draw(seed, root, TECH_T3, g, SIDE_ROOT, 0));
    if (is_black(xD.mat)) return;
    vtx yv[16], zv[16], Lv[16];
    int Lok[16], Cok[16];
    int ny = 0, nz = 0;
    yv[0] = xD; zv[0] = xD;
    /* light side: cosine direction about n(xD), then BSDF walk */
    {
        rnd4 r = draw(seed, root, TECH_T3, g, SIDE_LIGHT, 1);
        vec3 w;
        if (s->guide) {
            w = guided_direction(s, g, &xD, r, &k->vscale);
        } else {
            w = cosine_dir(xD.n, r.u[0], r.u[1]);
        }
        if (dot(xD.n, w) > 0.0 && trace_next(s, g, &xD, w, &yv[1]) && dot(yv[1].n, w) < 0.0 &&
            !is_black(yv[1].mat)) {
            ny = 1;
            for (int t = 2; t <= D - 3; ++t) {
                if (!walk_step(s, g, &yv[t - 2], &yv[t - 1],
                               draw(seed, root, TECH_T3, g, SIDE_LIGHT, t), &yv[t]))
                    break;
                if (is_black(yv[t].mat)) break;
                ny = t;
            }
        }
    }
    if (ny == 0) return;
    for (int t = 1; t <= ny; ++t)
        Lok[t] = nee(s, g, &yv[t], draw(seed, root, TECH_T3, g, SIDE_NEE, t), &Lv[t]);
    /* eye side: BSDF sample at xD conditioned on the light-side direction */
    for (int t = 1; t <= D - 3; ++t) {
        const vtx *prev = (t == 1) ? &yv[1] : &zv[t - 2];
        if (!walk_step(s, g, prev, &zv[t - 1], draw(seed, root, TECH_T3, g, SIDE_EYE, t), &zv[t]))
            break;
        if (is_black(zv[t].mat)) break;
        nz = t;
    }
    for (int t = 1; t <= nz; ++t) Cok[t] = camera_visible(s, g, &zv[t]);
    vtx path[16];
    for (int te = 1; te <= nz; ++te) {
        if (!Cok[te]) continue;
        for (int sl = 1; sl <= ny && te + sl <= D - 2; ++sl) {
            if (!Lok[sl]) continue;
            int n = te + sl + 3;
            path[0] = camera_vertex(s);
            for (int j = 0; j < te; ++j) path[1 + j] = zv[te - j];
            path[te + 1] = xD;
            for (int j = 1; j <= sl; ++j) path[te + 1 + j] = yv[j];
            path[n - 1] = Lv[sl];
            evaluate_path(k, g, path, n, root, TECH_T3, te, sl);
        }
    }
}

/* a point on the ghost: the dynamic object sampled by area at its pose of
 * the other frame */
static vtx sample_ghost(const oscene *s, int g, rnd4 r) {
    vtx v = sample_dynamic(s, 3 - g, r);
    v.prim = -1;                  /* not a surface of frame g */
    v.dyn = 0;
    return v;
}

/* (4) ghost from emitter: x_L by area, x_G on the ghost by area, the ray
 * from x_L through x_G finds the first vertex, which walks to the sensor */
static void root_T4(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    if (!s->motion) return;
    int D = s->max_depth;
    vtx xG = sample_ghost(s, g, draw(seed, root, TECH_T4, g, SIDE_ROOT, 0));
    vtx xL = sample_emitter(s, g, draw(seed, root, TECH_T4, g, SIDE_NEE, 0));
    vec3 e = sub(xG.p, xL.p);
    double dG = length(e);
    vec3 w = scale(e, 1.0 / dG);
    if (dot(xL.n, w) <= 0.0) return;
    vtx z[16];
    if (!trace_next(s, g, &xL, w, &z[0])) return;
    if (length(sub(z[0].p, xL.p)) <= dG || dot(z[0].n, w) >= 0.0) return;
    if (is_black(z[0].mat)) return;
    vtx path[16];
    for (int t = 0; t <= D - 2; ++t) {
        if (t > 0) {
            const vtx *prev = (t == 1) ? &xL : &z[t - 2];
            if (!walk_step(s, g, prev, &z[t - 1], draw(seed, root, TECH_T4, g, SIDE_EYE, t), &z[t]))
                break;
            if (is_black(z[t].mat)) break;
        }
        if (camera_visible(s, g, &z[t])) {
            int n = t + 3;
            path[0] = camera_vertex(s);
            for (int j = 0; j <= t; ++j) path[1 + j] = z[t - j];
            path[n - 1] = xL;
            evaluate_path(k, g, path, n, root, TECH_T4, t, 0);
        }
    }
}

/* (5) ghost from sensor: x_G on the ghost by area, the camera ray through
 * x_G finds x_1, then path tracing with next-event estimation */
static void root_T5(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    if (!s->motion) return;
    int D = s->max_depth;
    vtx xG = sample_ghost(s, g, draw(seed, root, TECH_T5, g, SIDE_ROOT, 0));
    double cc;
    if (camera_project(s, xG.p, &cc) < 0) return;
    vtx path[16];
    path[0] = camera_vertex(s);
    vec3 e = sub(xG.p, path[0].p);
    double dG = length(e);
    vec3 w = scale(e, 1.0 / dG);
    if (!trace_next(s, g, &path[0], w, &path[1])) return;
    if (length(sub(path[1].p, path[0].p)) <= dG || dot(path[1].n, w) >= 0.0) return;
    for (int j = 1; j <= D - 1; ++j) {
        if (is_black(path[j].mat)) break;
        vtx L;
        if (nee(s, g, &path[j], draw(seed, root, TECH_T5, g, SIDE_NEE, j), &L)) {
            path[j + 1] = L;
            evaluate_path(k, g, path, j + 2, root, TECH_T5, 0, j + 2);
        }
        if (j == D - 1) break;
        if (!walk_step(s, g, &path[j - 1], &path[j], draw(seed, root, TECH_T5, g, SIDE_LIGHT, j),
                       &path[j + 1]))
            break;
    }
}

/* (6) ghost two ends: x_G on the ghost by area and a uniform direction w;
 * the rays from x_G along +w and -w find the light-side vertex y_1 and the
 * eye-side vertex z_1 of an edge through x_G, then both sides walk */
static void root_T6(sink *k, int g, uint32_t root, uint64_t seed) {
    const oscene *s = k->s;
    if (!s->motion) return;
    int D = s->max_depth;
    if (D < 3) return;
    vtx xG = sample_ghost(s, g, draw(seed, root, TECH_T6, g, SIDE_ROOT, 0));
    rnd4 r = draw(seed, root, TECH_T6, g, SIDE_ROOT, 1);
    double zc = 1.0 - 2.0 * r.u[0], rs = sqrt(fmax(0.0, 1.0 - zc * zc)), phi = 2.0 * PI * r.u[1];
    vec3 w = v3(rs * cos(phi), rs * sin(phi), zc);
    vtx yv[16], zv[16], Lv[16];
    int Lok[16], Cok[16];
    if (!trace_next(s, g, &xG, w, &yv[1]) || dot(yv[1].n, w) >= 0.0 || is_black(yv[1].mat)) return;
    if (!trace_next(s, g, &xG, scale(w, -1.0), &zv[1]) || dot(zv[1].n, w) <= 0.0 ||
        is_black(zv[1].mat))
        return;
    int ny = 1, nz = 1;
    for (int t = 2; t <= D - 2; ++t) {
        const vtx *prev = (t == 2) ? &zv[1] : &yv[t - 2];
        if (!walk_step(s, g, prev, &yv[t - 1], draw(seed, root, TECH_T6, g, SIDE_LIGHT, t), &yv[t]))
            break;
        if (is_black(yv[t].mat)) break;
        ny = t;
    }
    for (int t = 1; t <= ny; ++t)
        Lok[t] = nee(s, g, &yv[t], draw(seed, root, TECH_T6, g, SIDE_NEE, t), &Lv[t]);
    for (int t = 2; t <= D - 2; ++t) {
        const vtx *prev = (t == 2) ? &yv[1] : &zv[t - 2];
        if (!walk_step(s, g, prev, &zv[t - 1], draw(seed, root, TECH_T6, g, SIDE_EYE, t), &zv[t]))
            break;
        if (is_black(zv[t].mat)) break;
        nz = t;
    }
    for (int t = 1; t <= nz; ++t) Cok[t] = camera_visible(s, g, &zv[t]);
    vtx path[16];
    for (int te = 1; te <= nz; ++te) {
        if (!Cok[te]) continue;
        for (int sl = 1; sl <= ny && te + sl <= D - 1; ++sl) {
            if (!Lok[sl]) continue;
            int n = te + sl + 2;
            path[0] = camera_vertex(s);
            for (int j = 0; j < te; ++j) path[1 + j] = zv[te - j];
            for (int j = 1; j <= sl; ++j) path[te + j] = yv[j];
            path[n - 1] = Lv[sl];
            evaluate_path(k, g, path, n, root, TECH_T6, te, sl);
        }
    }
}

/* path tracing with next-event estimation (technique PT / (7)) */
static void root_PT(sink *k, int g, uint32_t root, uint64_t seed, int tech) {
    const oscene *s = k->s;
    int D = s->max_depth;
    int npix = s->W * s->H;
    int pix = (int)(root % (uint32_t)npix);
    /* plain path tracing draws the same numbers in both frames (the frame
     * field of its counter is 0), so equal seeds give correlated path tracing;
     * technique (7) draws per frame like the other residual techniques */
    int rg = (tech == TECH_PT) ? 0 : g;
    rnd4 r = draw(seed, root, tech, rg, SIDE_ROOT, 0);
    vec3 d = camera_dir(s, pix % s->W, pix / s->W, r.u[0], r.u[1]);
    vtx path[16];
    path[0] = camera_vertex(s);
    if (!trace_next(s, g, &path[0], d, &path[1])) return;
    if (dot(path[1].n, d) >= 0.0) return;
    if (!is_zero3(path[1].mat->emission)) evaluate_path(k, g, path, 2, root, tech, 0, 2);
    for (int j = 1; j <= D - 1; ++j) {
        if (is_black(path[j].mat)) break;
        vtx L;
        if (nee(s, g, &path[j], draw(seed, root, tech, rg, SIDE_NEE, j), &L)) {
            path[j + 1] = L;
            evaluate_path(k, g, path, j + 2, root, tech, 0, j + 2);
        }
        if (j == D - 1) break;
        if (!walk_step(s, g, &path[j - 1], &path[j], draw(seed, root, tech, rg, SIDE_LIGHT, j),
                       &path[j + 1]))
            break;
    }
}

/* ------------------------------------------------------------------------- */
/* public entry points (ctypes)                                              */
/* ------------------------------------------------------------------------- */

static material read_material(const float *m) {
    material r;
    r.type = (int)m[0];
    r.albedo = v3(m[1], m[2], m[3]);
    r.alpha = m[4];
    r.f0 = v3(m[5], m[6], m[7]);
    r.emission = v3(m[8], m[9], m[10]);
    return r;
}

void *oracle_create(const float *sv, int n_sv, const uint32_t *st, const uint32_t *smat, int n_st,
                    const float *dv, int n_dv, const uint32_t *dt, int n_dt, const float *mats,
                    int n_mats, const float *cam /* pos, look, up, vfov */, int W, int H,
                    int max_depth, double alpha_min, double d_min, double jac_max) {
    (void)n_sv; (void)n_dv;
    oscene *s = (oscene *)calloc(1, sizeof(oscene));
    s->map_mode = 2;
    s->n_static = n_st;
    s->n_dyn = n_dt;
    s->stat = (tri *)malloc(sizeof(tri) * (size_t)(n_st > 0 ? n_st : 1));
    s->stat_mat = (int *)malloc(sizeof(int) * (size_t)(n_st > 0 ? n_st : 1));
    for (int i = 0; i < n_st; ++i) {
        const float *a = sv + 3 * st[3 * i], *b = sv + 3 * st[3 * i + 1], *c = sv + 3 * st[3 * i + 2];
        s->stat[i].v0 = v3(a[0], a[1], a[2]);
        s->stat[i].v1 = v3(b[0], b[1], b[2]);
        s->stat[i].v2 = v3(c[0], c[1], c[2]);
        s->stat_mat[i] = (int)smat[i];
    }
    s->dyn_obj = (tri *)malloc(sizeof(tri) * (size_t)(n_dt > 0 ? n_dt : 1));
    for (int i = 0; i < n_dt; ++i) {
        const float *a = dv + 3 * dt[3 * i], *b = dv + 3 * dt[3 * i + 1], *c = dv + 3 * dt[3 * i + 2];
        s->dyn_obj[i].v0 = v3(a[0], a[1], a[2]);
        s->dyn_obj[i].v1 = v3(b[0], b[1], b[2]);
        s->dyn_obj[i].v2 = v3(c[0], c[1], c[2]);
    }
    s->n_mats = n_mats;
    s->mats = (material *)malloc(sizeof(material) * (size_t)(n_mats > 0 ? n_mats : 1));
    for (int i = 0; i < n_mats; ++i) s->mats[i] = read_material(mats + 12 * i);
    bvh_build(&s->stat_bvh, s->stat, n_st, 0);
    /* sampling tables */
    s->dyn_cdf = (double *)malloc(sizeof(double) * (size_t)(n_dt > 0 ? n_dt : 1));
    double acc = 0.0;
    for (int i = 0; i < n_dt; ++i) { acc += tri_area(&s->dyn_obj[i]); s->dyn_cdf[i] = acc; }
    s->dyn_area = acc;
    for (int i = 0; i < n_dt; ++i) s->dyn_cdf[i] /= acc;
    if (n_dt > 0) s->dyn_cdf[n_dt - 1] = 1.0;
    s->n_emit = 0;
    s->emit_ids = (int *)malloc(sizeof(int) * (size_t)(n_st > 0 ? n_st : 1));
    s->emit_cdf = (double *)malloc(sizeof(double) * (size_t)(n_st > 0 ? n_st : 1));
    acc = 0.0;
    for (int i = 0; i < n_st; ++i) {
        if (is_zero3(s->mats[s->stat_mat[i]].emission)) continue;
        acc += tri_area(&s->stat[i]);
        s->emit_ids[s->n_emit] = i;
        s->emit_cdf[s->n_emit] = acc;
        s->n_emit++;
    }
    s->emit_area = acc;
    for (int i = 0; i < s->n_emit; ++i) s->emit_cdf[i] /= acc;
    if (s->n_emit > 0) s->emit_cdf[s->n_emit - 1] = 1.0;
    /* camera */
    s->cam_pos = v3(cam[0], cam[1], cam[2]);
    vec3 look = v3(cam[3], cam[4], cam[5]), up = v3(cam[6], cam[7], cam[8]);
    s->cam_fwd = normalize(sub(look, s->cam_pos));
    s->cam_right = normalize(cross(s->cam_fwd, up));
    s->cam_up = cross(s->cam_right, s->cam_fwd);
    s->hh = tan(0.5 * (double)cam[9] * PI / 180.0);
    s->W = W; s->H = H;
    s->hw = s->hh * (double)W / (double)H;
    s->pix_area = (2.0 * s->hw / W) * (2.0 * s->hh / H);
    s->max_depth = max_depth;
    s->alpha_min = alpha_min; s->d_min = d_min; s->jac_max = jac_max;
    s->eps = 1e-5;
    return s;
}

/* an edit of n objects moved (or re-materialed) together: dynamic triangle i
 * belongs to instance inst[i] (0..n-1), whose object-to-world transforms in
 * frames 1 and 2 are M1[12 k..], M2[12 k..] and whose materials are
 * mat1[12 k..], mat2[12 k..] */
int oracle_set_edit_multi(void *h, int n, const int *inst, const float *M1, const float *M2,
                          const float *mat1, const float *mat2) {
    oscene *s = (oscene *)h;
    if (n < 1 || n > MAX_INST) return -1;
    for (int i = 0; i < s->n_dyn; ++i)
        if (inst[i] < 0 || inst[i] >= n) return -1;
    s->n_inst = n;
    free(s->dyn_inst);
    s->dyn_inst = (int *)malloc(sizeof(int) * (size_t)(s->n_dyn > 0 ? s->n_dyn : 1));
    for (int i = 0; i < s->n_dyn; ++i) s->dyn_inst[i] = inst[i];
    s->motion = 0;
    for (int f = 1; f <= 2; ++f) {
        const float *M = (f == 1) ? M1 : M2;
        const float *m = (f == 1) ? mat1 : mat2;
        for (int k = 0; k < n; ++k) {
            for (int i = 0; i < 12; ++i) s->M[f][k][i] = M[12 * k + i];
            s->dyn_mat[f][k] = read_material(m + 12 * k);
        }
        if (s->has_edit) { free(s->dyn_world[f]); bvh_free(&s->dyn_bvh[f]); }
        s->dyn_world[f] = (tri *)malloc(sizeof(tri) * (size_t)(s->n_dyn > 0 ? s->n_dyn : 1));
        for (int i = 0; i < s->n_dyn; ++i) {
            const double *Mk = s->M[f][inst[i]];
            s->dyn_world[f][i].v0 = apply_M(Mk, s->dyn_obj[i].v0);
            s->dyn_world[f][i].v1 = apply_M(Mk, s->dyn_obj[i].v1);
            s->dyn_world[f][i].v2 = apply_M(Mk, s->dyn_obj[i].v2);
        }
        bvh_build(&s->dyn_bvh[f], s->dyn_world[f], s->n_dyn, s->n_static);
    }
    for (int i = 0; i < 12 * n; ++i)
        if (M1[i] != M2[i]) s->motion = 1;
    s->has_edit = 1;
    return 0;
}

/* an edit of the whole dynamic mesh as one object */
int oracle_set_edit(void *h, const float *M1, const float *M2, const float *mat1,
                    const float *mat2) {
    oscene *s = (oscene *)h;
    int *inst = (int *)calloc((size_t)(s->n_dyn > 0 ? s->n_dyn : 1), sizeof(int));
    int r = oracle_set_edit_multi(h, 1, inst, M1, M2, mat1, mat2);
    free(inst);
    return r;
}

void oracle_set_brute_force(void *h, int on) { ((oscene *)h)->brute_force = on; }

/* path mapping mode: 2 (default) camera replay for paths whose first edge
 * is dynamic, else the object transform; 1 the object transform for every
 * path; 0 no mapping (a base path of frame g adds s_g f_g(x) / (N P_g(x))
 * and each frame's paths come from its own sampling) */
void oracle_set_mapping(void *h, int mode) { ((oscene *)h)->map_mode = mode; }

void oracle_destroy(void *h) {
    oscene *s = (oscene *)h;
    if (!s) return;
    bvh_free(&s->stat_bvh);
    if (s->has_edit)
        for (int f = 1; f <= 2; ++f) { free(s->dyn_world[f]); bvh_free(&s->dyn_bvh[f]); }
    free(s->stat); free(s->stat_mat); free(s->dyn_obj); free(s->mats);
    free(s->dyn_cdf); free(s->emit_ids); free(s->emit_cdf); free(s->dyn_inst);
    free(s->guide);
    free(s);
}

/* technique mask bits: 0 (1), 1 (2), 2 (3), 3 path tracing, 4 (4), 5 (5), 6 (6) */
static techmask mask_from(int m) {
    techmask t = {(m >> 0) & 1, (m >> 1) & 1, (m >> 2) & 1, (m >> 3) & 1,
                  (m >> 4) & 1, (m >> 5) & 1, (m >> 6) & 1};
    return t;
}

/* the denominator's terms for the frame-g path x_0 = camera, x_i = the point
 * (bary[2(i-1)], bary[2(i-1)+1]) on prim[i-1] for i = 1..k-1, x_{k-1} on an
 * emitter (Sec. 4.3; ghost terms Sec. 4.2): up to cap (technique, density)
 * pairs are written; returns the number of terms, -1 on a bad argument */
int oracle_mis_terms(void *h, int g, int k, const int *prim, const double *bary, int tech_mask,
                     int *tech, double *dens, int cap) {
    const oscene *s = (const oscene *)h;
    if (!s || k < 2 || k > 15 || (g != 1 && g != 2)) return -1;
    vtx x[16];
    x[0] = camera_vertex(s);
    for (int i = 1; i < k; ++i) {
        if (prim[i - 1] < 0 || prim[i - 1] >= s->n_static + s->n_dyn) return -1;
        if (prim[i - 1] >= s->n_static && !s->has_edit) return -1;
        x[i] = make_vertex(s, g, prim[i - 1], bary[2 * (i - 1)], bary[2 * (i - 1) + 1]);
    }
    termacc acc = {0.0, 0, cap, dens, tech};
    mis_terms(s, g, x, k, mask_from(tech_mask), &acc);
    return acc.n;
}

/* run roots [r0, r1) of one technique in one frame */
static void run_roots(sink *k, int tech, int g, uint32_t r0, uint32_t r1, uint64_t seed) {
    for (uint32_t r = r0; r < r1; ++r) {
        switch (tech) {
        case TECH_T1: root_T1(k, g, r, seed); break;
        case TECH_T2: root_T2(k, g, r, seed); break;
        case TECH_T3: root_T3(k, g, r, seed); k->vscale = 0.0; break;
        case TECH_T4: root_T4(k, g, r, seed); break;
        case TECH_T5: root_T5(k, g, r, seed); break;
        case TECH_T6: root_T6(k, g, r, seed); break;
        case TECH_T7: root_PT(k, g, r, seed, TECH_T7); break;
        default: root_PT(k, g, r, seed, TECH_PT); break;
        }
    }
}

/* residual image I2 - I1 accumulated into img (H*W*3, row 0 at the top),
 * over roots [r0, r1) of every enabled technique in both frames;
 * counters (8 entries, may be NULL) receive rejection statistics */
int oracle_render_residual(void *h, uint32_t spp, uint64_t seed, uint32_t r0, uint32_t r1,
                           int tech_mask, double *img, int64_t *counters) {
    oscene *s = (oscene *)h;
    sink k;
    memset(&k, 0, sizeof k);
    k.s = s; k.img = img; k.N = (double)spp * s->W * s->H;
    k.tm = mask_from(tech_mask); k.residual = 1;
    const int techs[7] = {TECH_T1, TECH_T2, TECH_T3, TECH_T7, TECH_T4, TECH_T5, TECH_T6};
    for (int g = 1; g <= 2; ++g)
        for (int t = 0; t < 7; ++t)
            if ((tech_mask >> t) & 1) run_roots(&k, techs[t], g, r0, r1, seed);
    if (counters) memcpy(counters, k.counters, sizeof k.counters);
    return 0;
}

/* primal image of frame g by path tracing with next-event estimation,
 * restricted to the paths of `domain` (in_domain; 0 keeps every path) */
int oracle_render_primal_domain(void *h, int g, uint32_t spp, uint64_t seed, uint32_t r0,
                                uint32_t r1, int domain, double *img) {
    oscene *s = (oscene *)h;
    sink k;
    memset(&k, 0, sizeof k);
    k.s = s; k.img = img; k.N = (double)spp * s->W * s->H;
    k.residual = 0;
    k.domain = domain;
    run_roots(&k, TECH_PT, g, r0, r1, seed);
    return 0;
}

/* primal image of frame g by path tracing with next-event estimation */
int oracle_render_primal(void *h, int g, uint32_t spp, uint64_t seed, uint32_t r0, uint32_t r1,
                         double *img) {
    return oracle_render_primal_domain(h, g, spp, seed, r0, r1, 0, img);
}

/* per-sample records of technique `tech` in frame g for roots [r0, r1) */
int64_t oracle_dump(void *h, int tech, int g, uint32_t spp, uint64_t seed, uint32_t r0,
                    uint32_t r1, int tech_mask, orecord *rec, int64_t max_rec) {
    oscene *s = (oscene *)h;
    sink k;
    int64_t n = 0;
    memset(&k, 0, sizeof k);
    k.s = s; k.rec = rec; k.max_rec = max_rec; k.n_rec = &n;
    k.N = (double)spp * s->W * s->H;
    k.tm = mask_from(tech_mask); k.residual = 1;
    run_roots(&k, tech, g, r0, r1, seed);
    return n;
}

int oracle_record_size(void) { return (int)sizeof(orecord); }

/* closest hits for n rays in frame g: t (inf on miss), prim (-1), b1, b2 */
void oracle_closest_hit(void *h, int g, int n, const double *orig, const double *dir, double *t,
                        int *prim, double *b1, double *b2) {
    oscene *s = (oscene *)h;
    for (int i = 0; i < n; ++i) {
        hitrec hr;
        vec3 o = v3(orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]);
        vec3 d = v3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
        if (scene_trace(s, g, o, d, 0.0, INFINITY, -1, -1, 0, 0, &hr)) {
            t[i] = hr.t; prim[i] = hr.prim; b1[i] = hr.b1; b2[i] = hr.b2;
        } else {
            t[i] = INFINITY; prim[i] = -1; b1[i] = b2[i] = 0.0;
        }
    }
}

/* --- BSDF probes for the quadrature tests ------------------------------- */

void oracle_bsdf(const float *mrow, const double *n, const double *wi, const double *wo,
                 double *rho3, double *pdf) {
    material m = read_material(mrow);
    vec3 N = v3(n[0], n[1], n[2]), I = v3(wi[0], wi[1], wi[2]), O = v3(wo[0], wo[1], wo[2]);
    vec3 r = bsdf_eval(&m, N, I, O);
    rho3[0] = r.x; rho3[1] = r.y; rho3[2] = r.z;
    *pdf = bsdf_pdf(&m, N, I, O);
}

int oracle_bsdf_sample(const float *mrow, const double *n, const double *wc, double u1, double u2,
                       double *wo, double *u_back) {
    material m = read_material(mrow);
    vec3 N = v3(n[0], n[1], n[2]), C = v3(wc[0], wc[1], wc[2]), O;
    if (!bsdf_sample(&m, N, C, u1, u2, &O)) return 0;
    wo[0] = O.x; wo[1] = O.y; wo[2] = O.z;
    bsdf_inverse(&m, N, C, O, &u_back[0], &u_back[1]);
    return 1;
}

void oracle_tangent_frame(const double *n, double *t, double *b) {
    vec3 T, B;
    tangent_frame(v3(n[0], n[1], n[2]), &T, &B);
    t[0] = T.x; t[1] = T.y; t[2] = T.z;
    b[0] = B.x; b[1] = B.y; b[2] = B.z;
}

/* --- mapping self-checks (bijectivity and finite-difference Jacobians) ---- */

typedef struct {
    sink *k;
    int64_t n_pairs, n_bad_inverse, n_jac_checked;
    double max_pos_err, max_jac_err, max_fd_err;
} mapcheck;

static mapcheck *g_mc;

/* index of the conditioning vertex used when the mapping replays vertex b
 * (-1: cosine step), and the vertex a it is sampled from */
static void replay_geometry(const vtx *x, int n, int b, int *a, int *c) {
    int i = -1;
    for (int j = 1; j <= n - 2; ++j)
        if (x[j].dyn) i = j;
    if (b > i) {
        *a = b - 1;
        *c = (b == i + 1) ? ((i == 1) ? 0 : -1) : b - 2;
    } else {
        *a = b + 1;
        *c = (b == i - 1) ? ((i == n - 2) ? n - 1 : i + 1) : b + 2;
    }
}

/* map a base path, map the image back and compare; for every replayed vertex
 * compare the analytic per-vertex Jacobian with finite differences of the
 * mapping under perturbation of the base vertex within its triangle */
static void check_pair(const oscene *s, int g, const vtx *x, int n) {
    int g2 = 3 - g;
    vtx y[16], xb[16];
    mapinfo mi, mb;
    map_path(s, g, g2, x, n, y, &mi);
    if (mi.status != MAP_ACCEPT) return;
    if (!mapped_visible(s, g2, x, y, n, &mi)) return;
    int pb;
    if (is_zero3(path_throughput(s, y, n, &pb))) return;
    g_mc->n_pairs++;
    map_path(s, g2, g, y, n, xb, &mb);
    if (mb.status != MAP_ACCEPT) { g_mc->n_bad_inverse++; return; }
    double e = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = length(sub(xb[j].p, x[j].p));
        if (xb[j].prim != x[j].prim) d = INFINITY;
        if (d > e) e = d;
    }
    if (e > g_mc->max_pos_err) g_mc->max_pos_err = e;
    double je = fabs(mi.J * mb.J - 1.0);
    if (je > g_mc->max_jac_err) g_mc->max_jac_err = je;
    for (int b = 1; b <= n - 2; ++b) {
        if (!mi.replayed[b]) continue;
        /* central differences of the image point in the two barycentric
         * directions of the base vertex */
        const double h = 1e-6;
        const double db[4][2] = {{h, 0.0}, {-h, 0.0}, {0.0, h}, {0.0, -h}};
        vec3 px4[4], py4[4];
        int ok = 1;
        for (int m = 0; m < 4 && ok; ++m) {
            vtx xp[16], yp[16];
            mapinfo mp;
            memcpy(xp, x, sizeof(vtx) * (size_t)n);
            xp[b] = make_vertex(s, g, x[b].prim, x[b].b1 + db[m][0], x[b].b2 + db[m][1]);
            map_path(s, g, g2, xp, n, yp, &mp);
            if (mp.status != MAP_ACCEPT || !mp.replayed[b] || yp[b].prim != y[b].prim) ok = 0;
            px4[m] = xp[b].p;
            py4[m] = yp[b].p;
        }
        if (!ok) continue;
        double ax = length(cross(sub(px4[0], px4[1]), sub(px4[2], px4[3])));
        double ay = length(cross(sub(py4[0], py4[1]), sub(py4[2], py4[3])));
        int a, c;
        replay_geometry(x, n, b, &a, &c);
        const int cam_rule = s->map_mode == 2 && first_edge_dynamic(s, g, x, n);
        if (cam_rule) { a = b - 1; c = b - 2; }
        double pxd, pyd;
        if (cam_rule && b == 1) {
            pxd = pdf_camera_area(s, &x[1]);
            pyd = pdf_camera_area(s, &y[1]);
        } else if (c < 0) {
            pxd = area_from_dir(cosine_pdf(x[a].n, normalize(sub(x[b].p, x[a].p))), x[a].p, &x[b]);
            pyd = area_from_dir(cosine_pdf(y[a].n, normalize(sub(y[b].p, y[a].p))), y[a].p, &y[b]);
        } else {
            pxd = step_pdf(x, c, a, b);
            pyd = step_pdf(y, c, a, b);
        }
        double rel = fabs((ay / ax) / (pxd / pyd) - 1.0);
        g_mc->n_jac_checked++;
        if (rel > g_mc->max_fd_err) g_mc->max_fd_err = rel;
    }
}

static void mc_evaluate(sink *k, int g, const vtx *x, int n) {
    int pa;
    if (is_zero3(path_throughput(k->s, x, n, &pa))) return;
    check_pair(k->s, g, x, n);
}

/* run the sampler of `tech` and, for every accepted pair, map back and
 * compare; out[0..5] = pairs, bad inverses, max position error, max |J J' - 1|,
 * finite-difference checks, max relative FD error */
int oracle_check_mapping(void *h, int tech, int g, uint32_t spp, uint64_t seed, uint32_t r0,
                         uint32_t r1, double *out) {
    oscene *s = (oscene *)h;
    sink k;
    mapcheck mc;
    memset(&k, 0, sizeof k);
    memset(&mc, 0, sizeof mc);
    k.s = s; k.N = (double)spp * s->W * s->H; k.tm = mask_from(15); k.residual = 1;
    mc.k = &k;
    g_mc = &mc;
    g_check_mode = 1;
    run_roots(&k, tech, g, r0, r1, seed);
    g_check_mode = 0;
    out[0] = (double)mc.n_pairs; out[1] = (double)mc.n_bad_inverse;
    out[2] = mc.max_pos_err; out[3] = mc.max_jac_err;
    out[4] = (double)mc.n_jac_checked; out[5] = mc.max_fd_err;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* learned proposal: entry points                                            */
/* ------------------------------------------------------------------------- */

/* attach an integer network to technique (3) of this scene (W = NULL
 * detaches): W[20480] layer-major [out][in], shift[4], out_exp, box =
 * (center xyz, inverse half extent xyz) of the object-space inputs */
int oracle_set_guide(void *h, const int32_t *W, const int32_t *shift, int out_exp,
                     const float *box) {
    oscene *s = (oscene *)h;
    free(s->guide);
    s->guide = NULL;
    if (!W) return 0;
    oguide *gd = (oguide *)calloc(1, sizeof(oguide));
    memcpy(gd->W, W, sizeof gd->W);
    for (int l = 0; l < 4; ++l) gd->shift[l] = shift[l];
    gd->out_exp = out_exp;
    for (int c = 0; c < 3; ++c) { gd->center[c] = box[c]; gd->inv_half[c] = box[3 + c]; }
    s->guide = gd;
    return 0;
}

void oracle_guide_encode(const float *box, const double *p, const double *n, int32_t *m) {
    double c[3] = {box[0], box[1], box[2]}, ih[3] = {box[3], box[4], box[5]};
    guide_encode(c, ih, v3(p[0], p[1], p[2]), v3(n[0], n[1], n[2]), m);
}

/* rows of integer inputs m[rows][80] -> out[rows][48] */
void oracle_guide_forward(const int32_t *W, const int32_t *shift, int out_exp, const int32_t *m,
                          int rows, double *out) {
    oguide *gd = (oguide *)calloc(1, sizeof(oguide));
    memcpy(gd->W, W, sizeof gd->W);
    for (int l = 0; l < 4; ++l) gd->shift[l] = shift[l];
    gd->out_exp = out_exp;
    for (int r = 0; r < rows; ++r) guide_forward(gd, m + (size_t)r * G_IN, out + (size_t)r * G_OUT);
    free(gd);
}

double oracle_vmf_pdf(const double *mu, double kappa, const double *w) {
    return vmf_pdf(v3(mu[0], mu[1], mu[2]), kappa, v3(w[0], w[1], w[2]));
}

void oracle_vmf_sample(const double *mu, double kappa, double u1, double u2, double *w) {
    vec3 r = vmf_sample(v3(mu[0], mu[1], mu[2]), kappa, u1, u2);
    w[0] = r.x; w[1] = r.y; w[2] = r.z;
}

/* mixture of network outputs o[48]: pi[8], mu[8][3], kappa[8] */
void oracle_guide_mixture(const double *o, double *pi, double *mu, double *kappa) {
    vec3 m[G_LOBES];
    guide_mixture(o, m, kappa, pi);
    for (int j = 0; j < G_LOBES; ++j) { mu[3 * j] = m[j].x; mu[3 * j + 1] = m[j].y; mu[3 * j + 2] = m[j].z; }
}

/* float network: out[rows][48] for inputs x[rows][80] */
void oracle_mlp_forward(const double *W, const double *x, int rows, double *out) {
    double a0[G_IN], a1[G_HID], a2[G_HID], a3[G_HID], a4[G_HID], a5[G_OUT];
    double *acts[G_LAYERS + 1] = {a0, a1, a2, a3, a4, a5};
    for (int r = 0; r < rows; ++r) {
        mlp_forward_float(W, x + (size_t)r * G_IN, acts);
        memcpy(out + (size_t)r * G_OUT, a5, sizeof a5);
    }
}

/* mean loss (1/rows) sum_r -wt_r log q(w_r) of the float network and its
 * gradient grad[20480] with respect to W (back-propagation through the
 * mixture, the output layer and the ReLU layers) */
double oracle_mlp_loss_grad(const double *W, const double *x, const double *omega,
                            const double *wt, int rows, double *grad) {
    double a0[G_IN], a1[G_HID], a2[G_HID], a3[G_HID], a4[G_HID], a5[G_OUT];
    double *acts[G_LAYERS + 1] = {a0, a1, a2, a3, a4, a5};
    double loss = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 20480);
    for (int r = 0; r < rows; ++r) {
        mlp_forward_float(W, x + (size_t)r * G_IN, acts);
        double dcur[G_HID] = {0}, dprev[G_IN];
        const double *om = omega + 3 * (size_t)r;
        loss += mixture_nll(a5, v3(om[0], om[1], om[2]), wt[r], 1.0 / rows, grad ? dcur : NULL) / rows;
        if (!grad) continue;
        for (int l = G_LAYERS - 1; l >= 0; --l) {
            const int K = G_DIM_IN[l], N = G_DIM_OUT[l];
            /* dcur: gradient of the layer's pre-activation output z_l */
            for (int o = 0; o < N; ++o)
                for (int i = 0; i < K; ++i) grad[G_OFF[l] + o * K + i] += dcur[o] * acts[l][i];
            if (l == 0) break;
            for (int i = 0; i < K; ++i) {
                double d = 0.0;
                for (int o = 0; o < N; ++o) d += W[G_OFF[l] + o * K + i] * dcur[o];
                dprev[i] = acts[l][i] > 0.0 ? d : 0.0;     /* ReLU of the layer below */
            }
            for (int i = 0; i < K; ++i) dcur[i] = dprev[i];
        }
    }
    return loss;
}
