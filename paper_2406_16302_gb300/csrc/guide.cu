// Tensor-core kernels of the learned proposal (technique (3)'s light-side
// direction): integer-exact inference, fused forward + backward training
// with FP32 accumulation in tensor memory, feature encoding and Adam.
//
// Both network kernels keep one 128-row tile of activations per CTA in
// shared memory and run each layer as one chain of tcgen05.mma (M = 128
// rows, N = layer width, K = 16 per instruction) into tensor memory; four
// warps then read their 32 lanes back with tcgen05.ld for the epilogue
// (ReLU / requantisation, the mixture loss, the ReLU masks of the backward
// pass).  The training kernel also keeps every layer's activations and the
// current layer's output gradient transposed ([feature][row]) so that the
// weight gradients dW_l = dZ_l^T A_l are tensor-core products with K = 128
// rows, accumulated in tensor memory across all tiles of the CTA and
// flushed once with atomics.  Hidden activations enter the forward products
// as a high and a low BF16 part (an FP32 value to about 16 significant bits),
// because the mixture loss amplifies a BF16 rounding of the network outputs
// by up to kappa.
#include <cuda_bf16.h>

#include "guide.h"
#include "tc05.cuh"

namespace rp {

int device_sm_count();          // k_misc.cu

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;     // tensor-core waits give up after 2 s

// --- integer-exact inference ------------------------------------------------

constexpr uint32_t kI_W = 0;                    // weights of the five layers, 40960 bytes
constexpr uint32_t kI_A = 40960;                // activation tile [128][80], 20480 bytes
constexpr uint32_t kI_MBAR = 61440;
constexpr uint32_t kI_TSLOT = 61448;
constexpr uint32_t kI_SMEM = 61456;

__host__ __device__ constexpr uint32_t w_tile_off(int l) {
    // bf16 [out][in] tiles back to back: 64*80*2, 64*64*2 x3, 48*64*2
    return l == 0 ? 0u : l == 1 ? 10240u : l == 2 ? 18432u : l == 3 ? 26624u : 34816u;
}

__device__ void load_weights(unsigned char *sm, uint32_t base, const __nv_bfloat16 *W) {
    for (int l = 0; l < kGLayers; ++l) {
        const int K = guide_in(l), N = guide_out(l);
        const __nv_bfloat16 *src = W + guide_off(l);
        unsigned char *dst = sm + base + w_tile_off(l);
        for (int idx = threadIdx.x; idx < N * K; idx += blockDim.x) {
            const int o = idx / K, i = idx - o * K;
            *reinterpret_cast<__nv_bfloat16 *>(dst + tc::kmaj_off(o, i, K)) = src[idx];
        }
    }
}

// 8 consecutive values of one row into a K-major tile (one 16-byte store)
__device__ __forceinline__ void store8(unsigned char *tile, int row, int k, int K, const float *v) {
    __nv_bfloat162 p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    *reinterpret_cast<uint4 *>(tile + tc::kmaj_off(row, k, K)) = *reinterpret_cast<uint4 *>(p);
}

// withhold: the self-test of the timeout path (rp_guide_wait_selftest)
// issues no MMA and no commit, so nothing arrives at the barrier and the
// bounded wait runs out after limit_ns
__global__ void __launch_bounds__(128) k_guide_infer(const GuideNet net, const int8_t *__restrict__ m_in,
                                                     uint32_t n, float *__restrict__ out, int *err,
                                                     uint64_t limit_ns, int withhold) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kI_MBAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kI_TSLOT);
    load_weights(sm, kI_W, net.Wq);
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, 64);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    unsigned char *A = sm + kI_A;
    const uint32_t a_addr = tc::smem_u32(A);
    uint32_t phase = 0;
    int ok = 1;
    const uint32_t tiles = (n + 127u) / 128u;
    for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const uint32_t row = t * 128u + (uint32_t)tid;
        // layer-0 inputs: integer features as bf16 (exact)
        for (int k = 0; k < kGIn; k += 8) {
            float v[8];
            if (row < n) {
                const uint2 q = *reinterpret_cast<const uint2 *>(m_in + (size_t)row * kGIn + k);
                const int8_t *b = reinterpret_cast<const int8_t *>(&q);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = (float)b[j];
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.f;
            }
            store8(A, tid, k, kGIn, v);
        }
        tc::fence_async_smem();
        __syncthreads();
        for (int l = 0; l < kGLayers; ++l) {
            const int K = guide_in(l), N = guide_out(l);
            if (tid == 0 && !withhold) {
                tc::fence_after_sync();
                const uint32_t b_addr = tc::smem_u32(sm + kI_W + w_tile_off(l));
                for (int ks = 0; ks < K / 16; ++ks)
                    tc::mma_bf16(tmem, tc::desc_tile(a_addr, K, ks), tc::desc_tile(b_addr, K, ks),
                                 tc::idesc_bf16(128, N), ks > 0 ? 1u : 0u);
                tc::commit(mbar);
            }
            __syncwarp();
            const int got = tc::mbar_wait(mbar, phase, limit_ns) ? 1 : 0;
            phase ^= 1u;
            tc::fence_after_sync();
            ok = __syncthreads_and(got);
            if (!ok) break;
            if (l < kGLayers - 1) {
                const float sc = net.hid_scale[l];
                for (int c = 0; c < kGHid; c += 16) {
                    float z[16];
                    tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, c), z);
#pragma unroll
                    for (int j = 0; j < 16; ++j) z[j] = fminf(fmaxf(rintf(z[j] * sc), 0.f), 255.f);
                    store8(A, tid, c, kGHid, z);
                    store8(A, tid, c + 8, kGHid, z + 8);
                }
            } else {
                for (int c = 0; c < kGOut; c += 16) {
                    float z[16];
                    tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, c), z);
                    if (row < n) {
                        float4 *dst = reinterpret_cast<float4 *>(out + (size_t)row * kGOut + c);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            dst[j] = make_float4(z[4 * j] * net.out_scale, z[4 * j + 1] * net.out_scale,
                                                 z[4 * j + 2] * net.out_scale,
                                                 z[4 * j + 3] * net.out_scale);
                    }
                }
            }
            tc::fence_before_sync();
            tc::fence_async_smem();
            __syncthreads();
        }
    }
    if (!ok) {
        // let a late MMA finish before the tensor memory is released (none
        // was issued when withheld)
        if (!withhold) tc::mbar_wait(mbar, phase ^ 1u, limit_ns);
        if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// --- training: fused forward and backward ----------------------------------

// shared memory (bytes).  The forward input tiles (high and low BF16 parts
// of the activations) share their space with the backward tiles: a tile's
// forward pass ends before its backward pass starts.
constexpr uint32_t kT_W = 0;               // W_l [out][in] K-major, 40960
constexpr uint32_t kT_WT = 40960;          // W_l^T [in][out] for l = 1..4, 30720
constexpr uint32_t kT_AT = 71680;          // A_l^T [in][128] for l = 0..4, 20480 + 4 x 16384
constexpr uint32_t kT_BWD = 157696;        // 49152 bytes shared by:
constexpr uint32_t kT_XH = kT_BWD;         //   forward: A tile [128][<=80], high part
constexpr uint32_t kT_XL = kT_BWD + 20480; //   forward: A tile, low part
constexpr uint32_t kT_DZT = kT_BWD;        //   backward: dZ_l^T [128 (out, padded)][128]
constexpr uint32_t kT_DZ = kT_BWD + 32768; //   backward: dZ_l [128][<=64]
constexpr uint32_t kT_MBAR = 206848;
constexpr uint32_t kT_TSLOT = 206856;
constexpr uint32_t kT_SMEM = 206864;

__host__ __device__ constexpr uint32_t wt_tile_off(int l) {   // l = 1..4
    return l == 1 ? 0u : l == 2 ? 8192u : l == 3 ? 16384u : 24576u;
}
__host__ __device__ constexpr uint32_t at_tile_off(int l) {   // l = 0..4
    return l == 0 ? 0u : 20480u + (uint32_t)(l - 1) * 16384u;
}
// tensor-memory columns: scratch [0, 64), dW_l at dw_col(l)
__host__ __device__ constexpr int dw_col(int l) {
    return l == 0 ? 64 : l == 1 ? 160 : l == 2 ? 224 : l == 3 ? 288 : 352;
}

__device__ __forceinline__ void st_t(unsigned char *tile, int feat, int row, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(tile + tc::kmaj_off(feat, row, 128)) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ float ld_t(const unsigned char *tile, int feat, int row) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(tile + tc::kmaj_off(feat, row, 128)));
}

// gradient of -wt log sum_j pi_j vMF_j(w) with respect to the 48 outputs
// (log-space mixture; outputs 5j..5j+4 = direction, log kappa, logit)
__device__ float mixture_grad(const float *o, float3 w, float wt, float scale, float *d) {
    const float kTwoPi = 6.283185307179586f;
    float lmax = o[4];
#pragma unroll
    for (int j = 1; j < kGLobes; ++j) lmax = fmaxf(lmax, o[5 * j + 4]);
    float ls = 0.f;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) ls += __expf(o[5 * j + 4] - lmax);
    const float lse = lmax + logf(ls);
    float lv[kGLobes], kap[kGLobes], cs[kGLobes], len[kGLobes];
    float3 mu[kGLobes];
    float mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) {
        const float k = expf(fminf(6.2f, fmaxf(-4.0f, o[5 * j + 3])));
        float3 m = make_float3(o[5 * j], o[5 * j + 1], o[5 * j + 2]);
        const float l = sqrtf(m.x * m.x + m.y * m.y + m.z * m.z);
        float3 u = l > 1e-12f ? make_float3(m.x / l, m.y / l, m.z / l) : make_float3(0.f, 0.f, 1.f);
        const float c = u.x * w.x + u.y * w.y + u.z * w.z;
        kap[j] = k; cs[j] = c; len[j] = l; mu[j] = u;
        lv[j] = (o[5 * j + 4] - lse) + logf(k) - logf(kTwoPi) - logf(-expm1f(-2.f * k)) + k * (c - 1.f);
        mx = fmaxf(mx, lv[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) s += expf(lv[j] - mx);
    const float logq = mx + logf(s);
#pragma unroll
    for (int j = 0; j < kGLobes; ++j) {
        const float resp = expf(lv[j] - logq);
        const float pij = expf(o[5 * j + 4] - lse);
        const float k = kap[j], c = cs[j];
        d[5 * j + 4] = scale * -wt * (resp - pij);
        const float kr = o[5 * j + 3];
        if (kr > -4.0f && kr < 6.2f) {
            const float dlogv = 1.f / k - 2.f * expf(-2.f * k) / -expm1f(-2.f * k) + (c - 1.f);
            d[5 * j + 3] = scale * -wt * resp * k * dlogv;
        } else {
            d[5 * j + 3] = 0.f;
        }
        if (len[j] > 1e-12f) {
            const float f = scale * -wt * resp * k / len[j];
            d[5 * j + 0] = f * (w.x - c * mu[j].x);
            d[5 * j + 1] = f * (w.y - c * mu[j].y);
            d[5 * j + 2] = f * (w.z - c * mu[j].z);
        } else {
            d[5 * j + 0] = d[5 * j + 1] = d[5 * j + 2] = 0.f;
        }
    }
#pragma unroll
    for (int j = 5 * kGLobes; j < kGOut; ++j) d[j] = 0.f;
    return -wt * logq;
}

__device__ __forceinline__ void issue_wait(uint64_t *mbar, uint32_t &phase, int &ok) {
    if (threadIdx.x == 0) tc::commit(mbar);
    __syncwarp();
    const int got = tc::mbar_wait(mbar, phase, kWaitNs) ? 1 : 0;
    phase ^= 1u;
    tc::fence_after_sync();
    ok = __syncthreads_and(got);
}

__global__ void __launch_bounds__(128, 1) k_guide_train(const GuideTrain T) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kT_MBAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kT_TSLOT);
    // weights and their transposes
    load_weights(sm, kT_W, T.W);
    for (int l = 1; l < kGLayers; ++l) {
        const int K = guide_in(l), N = guide_out(l);      // W_l is N x K; W_l^T is K x N
        const __nv_bfloat16 *src = T.W + guide_off(l);
        unsigned char *dst = sm + kT_WT + wt_tile_off(l);
        for (int idx = tid; idx < N * K; idx += blockDim.x) {
            const int o = idx / K, i = idx - o * K;
            *reinterpret_cast<__nv_bfloat16 *>(dst + tc::kmaj_off(i, o, N)) = src[idx];
        }
    }
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    unsigned char *XH = sm + kT_XH, *XL = sm + kT_XL, *DZ = sm + kT_DZ, *DZT = sm + kT_DZT;
    const uint32_t xh_addr = tc::smem_u32(XH), xl_addr = tc::smem_u32(XL);
    const uint32_t dz_addr = tc::smem_u32(DZ), dzt_addr = tc::smem_u32(DZT);
    uint32_t phase = 0;
    int ok = 1, ntile = 0;
    float loss_acc = 0.f;
    const float scale = T.wsum ? 1.f / fmaxf(*T.wsum, 1e-30f) : T.inv_n;
    float amax[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t tiles = (T.n + 127u) / 128u;
    for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++ntile) {
        const uint32_t row = t * 128u + (uint32_t)tid;
        const bool live = row < T.n;
        // inputs: row-major for the forward product, transposed for dW_0
        for (int k = 0; k < kGIn; k += 8) {
            float v[8];
            if (live) {
                const uint4 q = *reinterpret_cast<const uint4 *>(T.X + (size_t)row * kGIn + k);
                const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = __bfloat162float(b[j]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.f;
            }
            store8(XH, tid, k, kGIn, v);      // the features are BF16 values: no low part
#pragma unroll
            for (int j = 0; j < 8; ++j) st_t(sm + kT_AT + at_tile_off(0), k + j, tid, v[j]);
        }
        tc::fence_async_smem();
        __syncthreads();
        // forward
        float o[kGOut];
        for (int l = 0; l < kGLayers && ok; ++l) {
            const int K = guide_in(l), N = guide_out(l);
            if (tid == 0) {
                // hidden activations are the sum of a high and a low BF16 part
                // (two products into one FP32 accumulator)
                tc::fence_after_sync();
                const uint32_t b_addr = tc::smem_u32(sm + kT_W + w_tile_off(l));
                for (int ks = 0; ks < K / 16; ++ks) {
                    tc::mma_bf16(tmem, tc::desc_tile(xh_addr, K, ks), tc::desc_tile(b_addr, K, ks),
                                 tc::idesc_bf16(128, N), ks > 0 ? 1u : 0u);
                    if (l > 0)
                        tc::mma_bf16(tmem, tc::desc_tile(xl_addr, K, ks), tc::desc_tile(b_addr, K, ks),
                                     tc::idesc_bf16(128, N), 1u);
                }
            }
            issue_wait(mbar, phase, ok);
            if (!ok) break;
            if (l < kGLayers - 1) {
                unsigned char *AT = sm + kT_AT + at_tile_off(l + 1);
                for (int c = 0; c < kGHid; c += 16) {
                    float z[16], lo[16];
                    tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, c), z);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        z[j] = live ? fmaxf(z[j], 0.f) : 0.f;
                        amax[l] = fmaxf(amax[l], z[j]);
                        st_t(AT, c + j, tid, z[j]);
                        lo[j] = z[j] - __bfloat162float(__float2bfloat16_rn(z[j]));
                    }
                    store8(XH, tid, c, kGHid, z);
                    store8(XH, tid, c + 8, kGHid, z + 8);
                    store8(XL, tid, c, kGHid, lo);
                    store8(XL, tid, c + 8, kGHid, lo + 8);
                }
            } else {
                for (int c = 0; c < kGOut; c += 16) tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, c), o + c);
            }
            tc::fence_before_sync();
            tc::fence_async_smem();
            __syncthreads();
        }
        if (!ok) break;
        // loss and its gradient with respect to the outputs
        float d[kGHid];
        const float wrow = live ? T.wt[row] : 0.f;
        if (wrow > 0.f) {
            const float3 w = make_float3(T.omega[3 * (size_t)row], T.omega[3 * (size_t)row + 1],
                                         T.omega[3 * (size_t)row + 2]);
            loss_acc += mixture_grad(o, w, wrow, scale, d) * scale;
        } else {
#pragma unroll
            for (int j = 0; j < kGOut; ++j) d[j] = 0.f;
        }
        // backward: dW_l += dZ_l^T A_l; dA_l = dZ_l W_l; dZ_{l-1} = dA_l * (A_l > 0)
        for (int l = kGLayers - 1; l >= 0 && ok; --l) {
            const int K = guide_in(l), N = guide_out(l);
            for (int j = 0; j < N; j += 8) store8(DZ, tid, j, N, d + j);
            for (int j = 0; j < N; ++j) st_t(DZT, j, tid, d[j]);
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t at_addr = tc::smem_u32(sm + kT_AT + at_tile_off(l));
                for (int ks = 0; ks < 8; ++ks)
                    tc::mma_bf16(tmem + (uint32_t)dw_col(l), tc::desc_tile(dzt_addr, 128, ks),
                                 tc::desc_tile(at_addr, 128, ks), tc::idesc_bf16(128, K),
                                 (ntile > 0 || ks > 0) ? 1u : 0u);
                if (l > 0) {
                    const uint32_t wt_addr = tc::smem_u32(sm + kT_WT + wt_tile_off(l));
                    for (int ks = 0; ks < N / 16; ++ks)
                        tc::mma_bf16(tmem, tc::desc_tile(dz_addr, N, ks), tc::desc_tile(wt_addr, N, ks),
                                     tc::idesc_bf16(128, K), ks > 0 ? 1u : 0u);
                }
            }
            issue_wait(mbar, phase, ok);
            if (!ok) break;
            if (l > 0) {
                const unsigned char *AT = sm + kT_AT + at_tile_off(l);
                for (int c = 0; c < kGHid; c += 16) {
                    float z[16];
                    tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, c), z);
#pragma unroll
                    for (int j = 0; j < 16; ++j) d[c + j] = ld_t(AT, c + j, tid) > 0.f ? z[j] : 0.f;
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
    }
    // flush the weight gradients accumulated in tensor memory
    if (ok && ntile > 0) {
        for (int l = 0; l < kGLayers; ++l) {
            const int K = guide_in(l), N = guide_out(l);
            for (int c = 0; c < K; c += 16) {
                float z[16];
                tc::tmem_ld16(tc::tmem_lane_col(tmem, warp, dw_col(l) + c), z);
                if (tid < N) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(T.grad + guide_off(l) + tid * K + c + j, z[j]);
                }
            }
        }
    }
    // loss and activation maxima
    for (int off = 16; off > 0; off >>= 1) {
        loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
#pragma unroll
        for (int l = 0; l < 4; ++l) amax[l] = fmaxf(amax[l], __shfl_xor_sync(0xffffffffu, amax[l], off));
    }
    if ((tid & 31) == 0) {
        atomicAdd(T.loss, loss_acc);
#pragma unroll
        for (int l = 0; l < 4; ++l) atomicMax(T.amax + l, __float_as_uint(amax[l]));
    }
    if (!ok) {
        tc::mbar_wait(mbar, phase ^ 1u, kWaitNs);
        if (tid == 0) atomicExch(T.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// --- features, conversions, Adam --------------------------------------------

// input features of the float network (same definition as the integer
// network's, unquantised): sin and cos of 2^f pi c for f = 0..5 of the
// normalised position and of the normal, the raw values, the constant 127/128
__global__ void k_guide_features(const GuideSamples smp, const float *box, uint32_t n,
                                 __nv_bfloat16 *X, float *omega, float *wt, float *wsum) {
    float acc = 0.f;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        float u[3], nn[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = fminf(1.f, fmaxf(-1.f, (smp.p[c * smp.cap + r] - box[c]) * box[3 + c]));
            nn[c] = smp.n[c * smp.cap + r];
        }
        __nv_bfloat16 *x = X + (size_t)r * kGIn;
        int i = 0;
        for (int v = 0; v < 2; ++v)
            for (int c = 0; c < 3; ++c)
                for (int f = 0; f < 6; ++f) {
                    const float a = ldexpf(v == 0 ? u[c] : nn[c], f);
                    x[i++] = __float2bfloat16_rn(sinpif(a));
                    x[i++] = __float2bfloat16_rn(cospif(a));
                }
        for (int c = 0; c < 3; ++c) x[i++] = __float2bfloat16_rn(u[c]);
        for (int c = 0; c < 3; ++c) x[i++] = __float2bfloat16_rn(nn[c]);
        x[78] = __float2bfloat16_rn(127.f / 128.f);
        x[79] = __float2bfloat16_rn(0.f);
        for (int c = 0; c < 3; ++c) omega[3 * (size_t)r + c] = smp.w[c * smp.cap + r];
        const float w = smp.wt[r];
        const bool ok = isfinite(w) && w > 0.f;
        wt[r] = ok ? w : 0.f;
        acc += ok ? w : 0.f;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc > 0.f) atomicAdd(wsum, acc);
}

__global__ void k_f32_to_bf16(const float *src, __nv_bfloat16 *dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_guide_adam(float *W, float *m, float *v, const float *grad, __nv_bfloat16 *Wbf,
                             int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float w = W[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        W[i] = w;
        Wbf[i] = __float2bfloat16_rn(w);
    }
}

}  // namespace

cudaError_t launch_guide_infer(const GuideNet &net, const int8_t *m_in, uint32_t n, float *out,
                               int *err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_guide_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kI_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint32_t tiles = (n + 127u) / 128u;
    const uint32_t grid = tiles < (uint32_t)(3 * device_sm_count()) ? tiles : (uint32_t)(3 * device_sm_count());
    k_guide_infer<<<grid, 128, kI_SMEM, s>>>(net, m_in, n, out, err, kWaitNs, 0);
    return cudaGetLastError();
}

cudaError_t launch_guide_wait_selftest(const GuideNet &net, const int8_t *m_in, float *out, int *err,
                                       uint64_t limit_ns, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_guide_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kI_SMEM);
    if (e != cudaSuccess) return e;
    k_guide_infer<<<1, 128, kI_SMEM, s>>>(net, m_in, 128u, out, err, limit_ns, 1);
    return cudaGetLastError();
}

cudaError_t launch_guide_train(const GuideTrain &t, cudaStream_t s) {
    if (t.n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_guide_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kT_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint32_t tiles = (t.n + 127u) / 128u;
    const uint32_t grid = tiles < (uint32_t)device_sm_count() ? tiles : (uint32_t)device_sm_count();
    k_guide_train<<<grid, 128, kT_SMEM, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_guide_features(const GuideSamples &smp, const float *box, uint32_t n,
                                  __nv_bfloat16 *X, float *omega, float *wt, float *wsum,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wsum, 0, sizeof(float), s);
    if (e != cudaSuccess || n == 0) return e;
    const uint32_t g = (n + 255u) / 256u;
    k_guide_features<<<g < 4096u ? g : 4096u, 256, 0, s>>>(smp, box, n, X, omega, wt, wsum);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float *src, __nv_bfloat16 *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t g = (n + 255) / 256;
    k_f32_to_bf16<<<(unsigned)(g < 4096 ? g : 4096), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_guide_adam(float *W, float *m, float *v, const float *grad,
                              __nv_bfloat16 *Wbf, int n, float lr, float b1, float b2, float eps,
                              float c1, float c2, cudaStream_t s) {
    k_guide_adam<<<(n + 255) / 256, 256, 0, s>>>(W, m, v, grad, Wbf, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace rp
