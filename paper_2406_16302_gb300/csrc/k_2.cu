// Path kernel of technique 2 (see rp_device.cuh): one thread per root.
#include "rp_device.cuh"

namespace rp {

__global__ void __launch_bounds__(kBlock) k_roots_2(const __grid_constant__ LaunchArgs A) {
    run_roots<T_2>(A);
}

cudaError_t launch_roots_2(const LaunchArgs &a, cudaStream_t s) {
    const uint32_t n = a.root_end - a.root_begin;
    if (n == 0) return cudaSuccess;
    const uint32_t grid = (n + kBlock - 1) / kBlock;
    k_roots_2<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rp
