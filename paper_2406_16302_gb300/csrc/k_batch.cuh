// Persistent batch kernel: many waves (jobs) of a batch of edits in one
// launch.
//
// A job is one wave of one item of the batch: a root range of one technique
// in one frame, with its own LaunchArgs (scene view of the item's moved
// object, edit, image, seed, resolution) and its own wavefront buffers.  A
// round is a set of jobs of the same technique, frame and edit kind, so they
// share the stage sequence of run_wave (k_wave.cu).  One launch runs a whole
// round: for every stage, the warps pull work items (job, chunk of the
// stage's roots, rays or tasks) from a device counter and run the stage's
// per-element work (wave_body.cuh); a grid barrier separates the stages.  The
// launch is cooperative, so every block is resident and the barrier cannot
// wait on a block that never runs; its waits are bounded all the same (a
// block that waits about two seconds records a timeout and the launch ends).
#pragma once

#include <algorithm>

#include "wave_body.cuh"

namespace rp {

namespace {

enum StageKind {
    SK_CLEAR = 0, SK_GEN, SK_START, SK_SHADOW, SK_CLOSEST, SK_EXTEND, SK_ENUM, SK_EVAL,
    SK_MAP_START, SK_TRACE_MAP, SK_MAP_STEP, SK_MAP_FIN, SK_TRACE_VIS, SK_MAP_B, SK_REPLAY_DIR
};

constexpr uint64_t kBarrierNs = 2000000000ull;      // a barrier wait gives up after 2 s

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// elements of stage (kind, it) of one job
__device__ __forceinline__ uint32_t stage_elems(const LaunchArgs &A, int kind, int it) {
    const WaveBuf &W = A.W;
    switch (kind) {
    case SK_CLEAR: return 1u;
    case SK_GEN:
    case SK_START:
    case SK_ENUM:
    case SK_EVAL: return A.root_end - A.root_begin;
    case SK_SHADOW: return min(__ldcg(W.counts + cnt_shadow(it)), W.qa);
    case SK_CLOSEST: return min(__ldcg(W.counts + cnt_closest(it)), W.qc);
    case SK_EXTEND: return min(__ldcg(W.counts + cnt_closest(it - 1)), W.qc);
    case SK_MAP_START: return min(__ldcg(W.counts + cnt_tasks()), W.qt);
    case SK_REPLAY_DIR:
    case SK_TRACE_MAP:
    case SK_MAP_STEP: return min(__ldcg(W.counts + cnt_replay(it)), W.qr);
    case SK_MAP_FIN:
        return min(__ldcg(W.counts + cnt_fin_acc()) + __ldcg(W.counts + cnt_fin_rej()), W.qt);
    case SK_TRACE_VIS: return min(__ldcg(W.counts + cnt_vis()), W.qv);
    case SK_MAP_B: return min(__ldcg(W.counts + cnt_pend()), W.qt);
    default: return 0u;
    }
}

template <int T>
__device__ __forceinline__ void stage_element(const LaunchArgs &A, Ctx &c, BodyState &st, int kind,
                                              int it, uint32_t i) {
    switch (kind) {
    case SK_CLEAR:
        for (int k = 0; k < kCountSlots; ++k) A.W.counts[k] = 0u;
        break;
    case SK_GEN: gen_body<T>(A, c, st, i, 0); break;
    case SK_START:
        if constexpr (T == T_1 || T == T_2) start_body<T>(A, c, st, i, 0);
        break;
    case SK_SHADOW: trace_shadow_body(A, c, st, i, it); break;
    case SK_CLOSEST: trace_closest_body(A, c, st, i, it); break;
    case SK_EXTEND: extend_body<T>(A, c, st, i, it); break;
    case SK_ENUM: enum_body<T>(A, c, st, i, 0); break;
    case SK_EVAL:
        if constexpr (T == T_1 || T == T_2 || T == T_3 || T == T_PT) eval_fast_body<T>(A, c, st, i, 0);
        break;
    case SK_MAP_START: map_start_body(A, c, st, i, 0); break;
    case SK_REPLAY_DIR: replay_dir_body(A, c, st, i, it); break;
    case SK_TRACE_MAP: trace_map_body(A, c, st, i, it); break;
    case SK_MAP_STEP: map_step_body(A, c, st, i, it); break;
    case SK_MAP_FIN: map_fin_body(A, c, st, i, 0); break;
    case SK_TRACE_VIS: trace_vis_body(A, c, st, i, 0); break;
    case SK_MAP_B: map_b_body(A, c, st, i, 0); break;
    default: break;
    }
}

// all blocks of the launch meet; false when a wait gave up (then *err is
// set and the caller returns)
__device__ bool grid_barrier(unsigned int *count, volatile unsigned int *gen, unsigned int blocks,
                             int *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        const unsigned int g0 = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == blocks - 1u) {
            *count = 0u;
            __threadfence();
            atomicAdd((unsigned int *)gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*gen == g0) {
                if (*(volatile int *)err || globaltimer_ns() - t0 > kBarrierNs) {
                    atomicExch(err, 1);
                    s_ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace

// blocks per SM the persistent kernel is compiled for (its register budget)
#ifndef RP_BATCH_MINBLOCKS
#define RP_BATCH_MINBLOCKS 8
#endif

template <int T>
__global__ void __launch_bounds__(kBlock, RP_BATCH_MINBLOCKS) k_batch(const __grid_constant__ BatchRound R) {
    __shared__ int s_stack[kStackDepth * kBlock];
    __shared__ float s_light[T == T_3 ? kT3LightSlots * 10 * kBlock : 1];
    __shared__ uint32_t s_n[kMaxBatchJobs];          // elements of each job in this stage
    __shared__ uint32_t s_first[kMaxBatchJobs + 1];  // first work item of each job
    const uint32_t chunk = R.chunk;
    Vtx x[kMaxVerts];
    for (int s = 0; s < R.n_stages; ++s) {
        const int kind = R.stages[s].x, it = R.stages[s].y;
        for (int j = threadIdx.x; j < R.n_jobs; j += blockDim.x) s_n[j] = stage_elems(R.jobs[j], kind, it);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0u;
            for (int j = 0; j < R.n_jobs; ++j) {
                s_first[j] = acc;
                acc += (s_n[j] + chunk - 1u) / chunk;
            }
            s_first[R.n_jobs] = acc;
        }
        __syncthreads();
        const uint32_t items = s_first[R.n_jobs];
        // each warp pulls its own work items: no block-wide wait inside a
        // stage, so a warp never idles behind another warp's longest ray
        const int lane = threadIdx.x & 31;
        for (;;) {
            uint32_t w = 0u;
            if (lane == 0) w = atomicAdd(R.work + s, 1u);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w >= items) break;
            int j = 0;
            while (s_first[j + 1] <= w) ++j;
            const LaunchArgs &A = R.jobs[j];
            Ctx c(A, s_stack + threadIdx.x);
            BodyState st{};
            st.x = x;
            st.s_light = s_light;
            const uint32_t e0 = (w - s_first[j]) * chunk, e1 = min(s_n[j], e0 + chunk);
            if (kind == SK_CLEAR) {
                if (lane == 0) stage_element<T>(A, c, st, kind, it, 0u);
            } else {
                for (uint32_t i = e0 + lane; i < e1; i += 32u) stage_element<T>(A, c, st, kind, it, i);
            }
            __syncwarp();
        }
        if (!grid_barrier(R.bar, R.bar + 1, gridDim.x, R.err)) return;
    }
}

// a cooperative launch of k_batch<T> for one round
template <int T>
cudaError_t launch_round(const BatchRound &R, int blocks_per_sm, cudaStream_t s) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<T>, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int per_sm = blocks_per_sm > 0 ? std::min(occ, blocks_per_sm) : occ;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(per_sm * device_sm_count()));
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch<T>, R);
}

}  // namespace rp
