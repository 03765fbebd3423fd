// rp_render_residual_f32_noalloc: the float32 residual render of
// rp_render_residual_f32 without any device allocation.
//
// rp_render_residual_f32 accumulates into an FP64 scratch image that the
// library allocates with cudaMalloc on first use.  Some callers cannot let a
// library allocate: hosts that own every byte of device memory through their
// own pool, run under a hard memory cap, or forbid allocation after start-up
// because cudaMalloc can synchronise the device and stall their other work.
// This entry point takes its scratch from a fixed array in the library's own
// device image instead, so the call allocates nothing.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rp.h"
#include "rp_internal.h"

namespace rp {
rp_status set_last_error(rp_status s, const char *msg);
rp_status scene_image_size(const rp_scene *scene, int *w, int *h);
rp_status render_residual_into(rp_scene *scene, const rp_edit_handle *edit, uint32_t spp,
                               uint64_t seed, uint32_t tech_mask, double *d_img,
                               cudaStream_t stream);
}  // namespace rp

namespace {

constexpr size_t kMaxPixels = (size_t)RP_NOALLOC_MAX_PIXELS;

// The scratch FP64 image: part of the library's device image.  A device holds
// it (24 MiB) from the first call on it (lazy module loading, CUDA's default;
// from library load with CUDA_MODULE_LOADING=EAGER) until the process exits.
__device__ __align__(256) double g_scratch[kMaxPixels * 3];

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_mutex;

// Host code may not use g_scratch directly (on the host it names a stand-in,
// not device memory): fetch its device address once per device, with that
// device current.
rp_status scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return rp::set_last_error(RP_ERR_CUDA, "cudaGetDevice failed (no usable CUDA device)");
    if (dev < 0 || dev >= kMaxDevices)
        return rp::set_last_error(RP_ERR_UNSUPPORTED, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return rp::set_last_error(RP_ERR_CUDA, "cudaGetSymbolAddress of the scratch image failed");
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return RP_OK;
}

}  // namespace

extern "C" rp_status rp_render_residual_f32_noalloc(rp_scene *scene, const rp_edit_handle *edit,
                                                     uint32_t spp, uint64_t seed,
                                                     uint32_t tech_mask, float *d_out,
                                                     void *stream) {
    int w = 0, h = 0;
    if (rp_status s = rp::scene_image_size(scene, &w, &h)) return s;
    if (!d_out) return rp::set_last_error(RP_ERR_INVALID_ARG, "null image");
    const size_t pixels = (size_t)w * (size_t)h;
    if (pixels > kMaxPixels)
        return rp::set_last_error(RP_ERR_INVALID_ARG,
                                  "image too large for rp_render_residual_f32_noalloc: width * "
                                  "height must not exceed RP_NOALLOC_MAX_PIXELS (1048576)");
    double *scratch = nullptr;
    if (rp_status s = scratch_for_current_device(&scratch)) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear the part this call uses
    cudaError_t e = cudaMemsetAsync(scratch, 0, pixels * 3 * sizeof(double), st);
    if (e != cudaSuccess) return rp::set_last_error(RP_ERR_CUDA, cudaGetErrorString(e));
    if (rp_status s = rp::render_residual_into(scene, edit, spp, seed, tech_mask, scratch, st))
        return s;
    e = rp::launch_add_f64_to_f32(scratch, d_out, pixels * 3, st);
    if (e != cudaSuccess) return rp::set_last_error(RP_ERR_CUDA, cudaGetErrorString(e));
    return RP_OK;
}
