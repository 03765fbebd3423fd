// Dispatch of the path kernels and the small utility kernels: ray queries for
// intersection tests, Philox known answers, FP64 -> FP32 image resolve.
#include "rp_device.cuh"

namespace rp {

cudaError_t launch_roots_1(const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_roots_2(const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_roots_3(const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_roots_7(const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_roots_pt(const LaunchArgs &a, cudaStream_t s);

cudaError_t launch_residual(int tech, const LaunchArgs &a, cudaStream_t s) {
    switch (tech) {
    case 1: return launch_roots_1(a, s);
    case 2: return launch_roots_2(a, s);
    case 3: return launch_roots_3(a, s);
    case 7: return launch_roots_7(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_primal(const LaunchArgs &a, cudaStream_t s) { return launch_roots_pt(a, s); }

__global__ void __launch_bounds__(kBlock) k_trace(const __grid_constant__ LaunchArgs A, uint32_t n,
                                                  const float *o, const float *d, float *t,
                                                  int32_t *prim, float *b1, float *b2) {
    __shared__ int s_stack[kStackDepth * kBlock];
    Ctx c(A, s_stack + threadIdx.x);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {      // no early return: the counters below are summed over whole warps
        Hit h;
        const float3 oo = f3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        const float3 dd = f3(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        ++c.cnt.rays_closest;
        if (scene_trace(c, A.frame, oo, dd, 0.0f, __int_as_float(0x7f800000), -1, -1, false, false, h)) {
            t[i] = h.t;
            prim[i] = h.prim;
            b1[i] = h.b1;
            b2[i] = h.b2;
        } else {
            t[i] = __int_as_float(0x7f800000);
            prim[i] = -1;
            b1[i] = 0.f;
            b2[i] = 0.f;
        }
    }
    if (A.stats) {
        add_stat(A.stats, ST_RAYS_CLOSEST, c.cnt.rays_closest);
        add_stat(A.stats, ST_NODES, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS, c.cnt.tris);
        add_stat(A.stats, ST_NODES_C, c.cnt.nodes);
        add_stat(A.stats, ST_TRIS_C, c.cnt.tris);
    }
}

cudaError_t launch_trace(const DevScene &S, const DevEdit &E, int frame, uint32_t n, const float *o,
                         const float *d, float *t, int32_t *prim, float *b1, float *b2,
                         unsigned long long *stats, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    LaunchArgs a{};
    a.S = S;
    a.E = E;
    a.frame = frame;
    a.stats = stats;
    k_trace<<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(a, n, o, d, t, prim, b1, b2);
    return cudaGetLastError();
}

__global__ void k_philox(uint32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    uint4 r = philox4x32_10(c, k);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

cudaError_t launch_philox(uint32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, s>>>(n, ctr, key, out);
    return cudaGetLastError();
}

__global__ void k_add_f64_to_f32(const double *src, float *dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] += (float)src[i];
}

int device_sm_count() {
    // per device, looked up once (attribute queries are not stream work, so
    // this is safe inside a stream capture)
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    if (dev < 64) cache[dev] = n;
    return n;
}

cudaError_t launch_add_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    const int cap = device_sm_count() * 8;       // 8 resident blocks of 256 per SM
    if (grid > cap) grid = cap;
    k_add_f64_to_f32<<<grid, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace rp
