// The persistent batch kernel's stage lists and the dispatch of one round to
// the kernel instance of its technique (each instance is compiled in its own
// translation unit, k_batch_t*.cu).
#include "k_batch.cuh"

namespace rp {

cudaError_t launch_round_t1(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_t2(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_t3(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_t4(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_t5(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_t6(const BatchRound &R, int blocks_per_sm, cudaStream_t s);
cudaError_t launch_round_pt(const BatchRound &R, int blocks_per_sm, cudaStream_t s);

// the stage sequence of one wave of technique `tech` (run_wave)
int batch_stages(int tech, int D, bool mapped, int2 *out) {
    int n = 0;
    auto add = [&](int k, int it) { out[n++] = make_int2(k, it); };
    add(SK_CLEAR, 0);
    add(SK_GEN, 0);
    if (tech == T_1 || tech == T_2) {
        add(SK_SHADOW, 0);
        add(SK_START, 0);
        add(SK_SHADOW, 1);
    }
    for (int it = 1; it <= D + 1 && it + 1 < kMaxIter; ++it) {
        add(SK_CLOSEST, it - 1);
        add(SK_EXTEND, it);
        add(SK_SHADOW, it + 1);
    }
    if (mapped) {
        add(SK_ENUM, 0);
        add(SK_MAP_START, 0);
        for (int r = 0; r < D - 1 && r + 1 < kMaxIter; ++r) {
            add(SK_REPLAY_DIR, r);
            add(SK_TRACE_MAP, r);
            add(SK_MAP_STEP, r);
        }
        add(SK_MAP_FIN, 0);
        add(SK_TRACE_VIS, 0);
        add(SK_MAP_B, 0);
    } else {
        add(SK_EVAL, 0);
    }
    return n;
}

cudaError_t launch_batch_round(int tech, const BatchRound &R, int blocks_per_sm, cudaStream_t s) {
    switch (tech) {
    case 1: return launch_round_t1(R, blocks_per_sm, s);
    case 2: return launch_round_t2(R, blocks_per_sm, s);
    case 3: return launch_round_t3(R, blocks_per_sm, s);
    case 4: return launch_round_t4(R, blocks_per_sm, s);
    case 5: return launch_round_t5(R, blocks_per_sm, s);
    case 6: return launch_round_t6(R, blocks_per_sm, s);
    case 7:
    case 0: return launch_round_pt(R, blocks_per_sm, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rp
