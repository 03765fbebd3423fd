// Learned proposal of technique (3): device views of the network and the
// launchers of its tensor-core kernels (internal, not part of the ABI).
//
// The network maps 80 input features of an object-space point and normal to
// 48 outputs: 8 von Mises-Fisher lobes of (direction 3, log kappa, logit),
// outputs 40..47 unused.  Layers (out x in): 64x80, 64x64, 64x64, 64x64,
// 48x64, ReLU after the first four, no biases besides a constant input.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rp {

constexpr int kGIn = 80, kGHid = 64, kGOut = 48, kGLobes = 8, kGLayers = 5;
constexpr int kGWeights = 20480;
__host__ __device__ constexpr int guide_off(int l) {
    return l == 0 ? 0 : l == 1 ? 5120 : l == 2 ? 9216 : l == 3 ? 13312 : l == 4 ? 17408 : 20480;
}
__host__ __device__ constexpr int guide_in(int l) { return l == 0 ? kGIn : kGHid; }
__host__ __device__ constexpr int guide_out(int l) { return l == 4 ? kGOut : kGHid; }

// integer network used while rendering: weights in [-127, 127] stored as
// bf16 (exact), hidden requantisation h = clamp(rint(z 2^-shift), 0, 255),
// outputs z 2^-out_exp
struct GuideNet {
    const __nv_bfloat16 *Wq;
    float hid_scale[4];         // 2^-shift[l]
    float out_scale;            // 2^-out_exp
    float box[6];               // center xyz, inverse half extent xyz (object space)
};

// training samples gathered from guided renders of technique (3), one per
// root below the capacity (SoA)
struct GuideSamples {
    float *p, *n, *w;           // [3][cap]: object-space point, normal, light-side direction
    float *wt;                  // [cap]: |contribution| of the root
    uint32_t cap;
};

struct GuideTrain {
    const __nv_bfloat16 *W;     // [20480] bf16 weights, layer-major [out][in]
    const __nv_bfloat16 *X;     // [n][80] input features
    const float *omega;         // [n][3] directions (object space, unit)
    const float *wt;            // [n] sample weights
    uint32_t n;
    float inv_n;                // scale of the mean loss (used when wsum is null)
    const float *wsum;          // if set, the loss is scaled by 1 / *wsum instead
    float *grad;                // [20480] accumulated with atomics
    float *loss;                // [1] accumulated
    unsigned int *amax;         // [4] max hidden activation (float bits, non-negative)
    int *err;                   // set on a tensor-core wait timeout
};

cudaError_t launch_guide_infer(const GuideNet &net, const int8_t *m_in, uint32_t n, float *out,
                               int *err, cudaStream_t s);
cudaError_t launch_guide_train(const GuideTrain &t, cudaStream_t s);
// one tile of the inference kernel with its MMA completion withheld and the
// barrier wait bounded by limit_ns (the timeout path's self-test)
cudaError_t launch_guide_wait_selftest(const GuideNet &net, const int8_t *m_in, float *out, int *err,
                                       uint64_t limit_ns, cudaStream_t s);
// training batch from the samples: features, directions, weights, and the
// sum of the weights into *wsum
cudaError_t launch_guide_features(const GuideSamples &smp, const float *box, uint32_t n,
                                  __nv_bfloat16 *X, float *omega, float *wt, float *wsum,
                                  cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float *src, __nv_bfloat16 *dst, size_t n, cudaStream_t s);
// input features of n points (double) and normals (float): out[n][80]
cudaError_t launch_guide_encode(const float *box, const double *p, const float *nrm, uint32_t n,
                                int8_t *out, cudaStream_t s);
cudaError_t launch_guide_adam(float *W, float *m, float *v, const float *grad,
                              __nv_bfloat16 *Wbf, int n, float lr, float b1, float b2, float eps,
                              float c1, float c2, cudaStream_t s);

}  // namespace rp
