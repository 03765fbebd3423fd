// The persistent batch kernel for technique T_6 (k_batch.cuh).
#include "k_batch.cuh"

namespace rp {

cudaError_t launch_round_t6(const BatchRound &R, int blocks_per_sm, cudaStream_t s) {
    return launch_round<T_6>(R, blocks_per_sm, s);
}

}  // namespace rp
