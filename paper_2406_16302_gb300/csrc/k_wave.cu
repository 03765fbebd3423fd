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
#include <algorithm>

#include "wave_body.cuh"

namespace rp {

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



namespace {
struct EncodeArgs {
    float box[6];
    const double *p;
    const float *nrm;
    uint32_t n;
    int8_t *out;
};
}  // namespace





template <int T>
__global__ void __launch_bounds__(256) k_gen(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    Ctx c(A, nullptr);
    BodyState st{};
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        gen_body<T>(A, c, st, r, 0);

}

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

// the learned proposal's input features of given points (rp_guide_encode)
__global__ void __launch_bounds__(128) k_guide_encode(const __grid_constant__ EncodeArgs E) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < E.n; i += gridDim.x * blockDim.x)
        store_features(E.out + (size_t)i * kGIn, E.box, d3(E.p[3 * i], E.p[3 * i + 1], E.p[3 * i + 2]),
                       f3(E.nrm[3 * i], E.nrm[3 * i + 1], E.nrm[3 * i + 2]));
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
            wl = vmf_sample_d(A.S, guide_lobe_dir_d(A.G.gout + (size_t)r * kGOut, j),
                              (double)mix.kappa[j], u.x, u.y);
            w = dlinear(M, wl);
        }
        const double cw = ddot(nw, w);
        const float pc = cw > 0.0 ? (float)(cw / kPiD) : 0.f;
        const float3 wlf = tof(wl);
        const float pv = mix_pdf_f(mix, wlf);
        A.G.gratio[r] = pc / (0.5f * pc + 0.5f * pv);
        const uint32_t slot = guide_slot(A.G, g, root);
        if (slot != ~0u) {
            const uint32_t C = A.G.smp.cap;
            A.G.smp.w[slot] = wlf.x; A.G.smp.w[C + slot] = wlf.y;
            A.G.smp.w[2 * C + slot] = wlf.z;
        }
        const float3 wf = tof(w);
        if (dot3(xD.n, wf) > 0.f) push_closest(A, 0, 0, xD.p, wf, xD.prim, make_tag(r, SIDE_LIGHT, 1));
    }
}

// techniques (1) and (2): start the walk of roots whose root connection is visible
template <int T>
__global__ void __launch_bounds__(256) k_start(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    Ctx c(A, nullptr);
    BodyState st{};
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        start_body<T>(A, c, st, r, 0);

}

// consume the hits of iteration it-1's closest rays; emit iteration it's rays
template <int T>
__global__ void __launch_bounds__(256) k_extend(const __grid_constant__ LaunchArgs A, int it) {
    const uint32_t n = min(A.W.counts[cnt_closest(it - 1)], A.W.qc);
    Ctx c(A, nullptr);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        extend_body<T>(A, c, st, i, it);

}

// closest hits of a queue
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_closest(const __grid_constant__ LaunchArgs A, int it) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n = min(A.W.counts[cnt_closest(it)], A.W.qc);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        trace_closest_body(A, c, st, i, it);

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
    const uint32_t n = min(A.W.counts[cnt_shadow(it)], A.W.qa);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        trace_shadow_body(A, c, st, i, it);

    if (A.stats) {
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_NODES_S, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS_S, c.cnt.tris);
    }
}

// motion: every non-static base path of a root becomes a mapping task
template <int T>
__global__ void __launch_bounds__(128) k_enum(const __grid_constant__ LaunchArgs A) {
    const uint32_t n = A.root_end - A.root_begin;
    Ctx c(A, nullptr);
    Vtx x[1];
    BodyState st{};
    st.x = x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        enum_body<T>(A, c, st, r, 0);

    if (A.stats) add_stat(A.stats, ST_ROOTS, st.roots);
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
    Ctx c(A, nullptr);
    BodyState st{};
    st.s_light = s_light;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        eval_fast_body<T>(A, c, st, r, 0);

    if (A.stats) {
        add_stat(A.stats, ST_ROOTS, st.roots);
        add_stat(A.stats, ST_PATHS, st.pc.paths);
        add_stat(A.stats, ST_ACCEPTED, st.pc.accepted);
    }
}

// stage C1: one thread per mapping task: the start of its mapping (camera
// replay or object transform, Sec. 5) and its steps up to the first replay
__global__ void __launch_bounds__(kBlock, RP_MAP_MINBLOCKS) k_map_start(const __grid_constant__ LaunchArgs A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n = min(A.W.counts[cnt_tasks()], A.W.qt);
    BodyState st{};
    for (uint32_t ti = blockIdx.x * blockDim.x + threadIdx.x; ti < n; ti += gridDim.x * blockDim.x)
        map_start_body(A, c, st, ti, 0);

    if (A.stats) {
        add_stat(A.stats, ST_PATHS, st.pc.paths);
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_ACCEPTED, st.pc.accepted);
        add_stat(A.stats, ST_REJECTED, st.pc.rejected);
    }
}

// stage C2a: the directions of the round's random-seed replays (double
// precision, one thread per queued replay)
__global__ void __launch_bounds__(kBlock, RP_MAP_MINBLOCKS) k_replay_dir(const __grid_constant__ LaunchArgs A, int round) {
    Ctx c(A, nullptr);
    const uint32_t n = min(A.W.counts[cnt_replay(round)], A.W.qr);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        replay_dir_body(A, c, st, i, round);
}

// stage C2b: closest hits of the mapping's replay rays of one round, in the
// other frame
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_map(const __grid_constant__ LaunchArgs A, int round) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n = min(A.W.counts[cnt_replay(round)], A.W.qr);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        trace_map_body(A, c, st, i, round);

    if (A.stats) {
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
    }
}

// stage C2c: resume the tasks of one round with their hits; the next
// replay rays go to round + 1
__global__ void __launch_bounds__(kBlock, RP_MAP_MINBLOCKS) k_map_step(const __grid_constant__ LaunchArgs A, int round) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n = min(A.W.counts[cnt_replay(round)], A.W.qr);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        map_step_body(A, c, st, i, round);

    if (A.stats) {
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
    }
}

// stage C3: every task with its mapped path: values, MIS, queued visibility
// of the mapped path (finish_task); the accepted tasks first, then the others
__global__ void __launch_bounds__(kBlock, RP_MAPFIN_MINBLOCKS) k_map_fin(const __grid_constant__ LaunchArgs A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n_acc = min(A.W.counts[cnt_fin_acc()], A.W.qt);
    const uint32_t n = min(n_acc + A.W.counts[cnt_fin_rej()], A.W.qt);
    Vtx x[kMaxVerts];
    BodyState st{};
    st.x = x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        map_fin_body(A, c, st, j, 0);

    if (A.stats) {
        add_stat(A.stats, ST_PATHS, st.pc.paths);
        add_stat(A.stats, ST_RAYS_SHADOW, c.cnt.rays_shadow);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_ACCEPTED, st.pc.accepted);
        add_stat(A.stats, ST_REJECTED, st.pc.rejected);
    }
}

// stage C2: the queued edges of mapped paths, in the other frame; a blocked
// edge makes its task's pair invalid
__global__ void __launch_bounds__(kBlock, RP_TRACE_MINBLOCKS) k_trace_vis(const __grid_constant__ LaunchArgs A) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t n = min(A.W.counts[cnt_vis()], A.W.qv);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        trace_vis_body(A, c, st, i, 0);

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
    const uint32_t n = min(A.W.counts[cnt_pend()], A.W.qt);
    BodyState st{};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        map_b_body(A, c, st, i, 0);

    if (A.stats) add_stat(A.stats, ST_ACCEPTED, st.accepted);
}

// the learned proposal's input features of given points (rp_guide_encode)
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
        const bool t_ = a.timer && a.timer->wants(name);                             \
        if (t_) timer_begin(a.timer, s, &e0_, &e1_);                                 \
        kernel<<<(grid), (block), 0, s>>>(__VA_ARGS__);                             \
        if (t_) timer_end(a.timer, name, s, e0_, e1_);                               \
    } while (0)

// stage C: map every task, trace the mapped paths' queued edges, emit
void map_stage(const LaunchArgs &a, cudaStream_t s, int gQ) {
    RP_LAUNCH("k_map_start", gQ, kBlock, k_map_start, a);
    // a mapping program has at most max_depth - 1 replay steps (the camera
    // ray and the walk vertices x_2 .. x_{k-2})
    const int rounds = a.S.max_depth - 1;
    for (int r = 0; r < rounds && r + 1 < kMaxIter; ++r) {
        RP_LAUNCH("k_replay_dir", gQ, kBlock, k_replay_dir, a, r);
        RP_LAUNCH("k_trace_map", gQ, kBlock, k_trace_map, a, r);
        RP_LAUNCH("k_map_step", gQ, kBlock, k_map_step, a, r);
    }
    RP_LAUNCH("k_map_fin", gQ, kBlock, k_map_fin, a);
    RP_LAUNCH("k_trace_vis", gQ, kBlock, k_trace_vis, a);
    RP_LAUNCH("k_map_b", gQ, 256, k_map_b, a);
}

// The grid of the queue kernels: one block per 256 roots of the wave,
// between 16 and 128 blocks per SM.  The kernels stride over device-side
// queue counts of up to about one ray per root; blocks beyond the resident
// ones start as others finish, which evens out the rays' unequal costs
// (2^24-root waves of the terrain: 3.6 % less time per render at 128 per SM
// than at 16), while small waves pay for their empty blocks (2^18-root
// waves: 16 per SM is best).
inline int queue_grid(uint32_t n) {
    const uint32_t sms = (uint32_t)device_sm_count();
    return (int)std::min(std::max(n / 256u, 16u * sms), 128u * sms);
}

template <int T>
cudaError_t run_wave(const LaunchArgs &a, cudaStream_t s) {
    const uint32_t n = a.root_end - a.root_begin;
    const int D = a.S.max_depth;
    const int gR = grid_for(n, 256, 1 << 20);
    const int gQ = a.grid_q > 0 ? a.grid_q : queue_grid(n);
    cudaError_t e = cudaMemsetAsync(a.W.counts, 0, sizeof(unsigned int) * kCountSlots, s);
    if (e != cudaSuccess) return e;
    RP_LAUNCH("k_gen", gR, 256, k_gen<T>, a);
    if (T == T_3 && a.G.use_net) {
        RP_LAUNCH("k_encode3", gR, 128, k_encode3, a);
        cudaEvent_t e0_ = nullptr, e1_ = nullptr;
        const bool t_ = a.timer && a.timer->wants("k_guide_infer");
        if (t_) timer_begin(a.timer, s, &e0_, &e1_);
        e = launch_guide_infer(a.G.net, a.G.gin, n, a.G.gout, a.G.err, s);
        if (t_) timer_end(a.timer, "k_guide_infer", s, e0_, e1_);
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
