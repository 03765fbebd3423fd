"""Benchmark: residual samples/s of the residual path integral estimator on GB300.

Workload (default, `terrain_motion_1024`): the scale configuration -- a
seeded fBm terrain of about 1M triangles with 200 instanced Lambert/GGX
primitives, a 50k-triangle object rotated by 10 degrees and translated by 5 %
of the scene extent between the frames; 1024x1024, 256 spp, max depth 8;
techniques (1), (2), (3) and path tracing with rejection, both frames, every
base path mapped into the other frame (object transform, camera replay,
reconnection, random replay) and weighted by the two-way balance heuristic.
`--workload box_blob_material_256` runs the material edit (256x256, 64 spp).

One step = one residual render of the whole image (every root of every
technique in both frames), i.e. one rp_render_residual call.  A residual sample = one root
of one technique in one frame, with every base path it generates, their
mapped paths, MIS denominators and splats; a step processes
spp * W * H * 4 * 2 of them.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.  `--workload device_peaks`
measures the L2 read bandwidth and FP32 FMA rate that the traversal
roofline uses beside the HBM copy bandwidth.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 operation counts of the traversal kernels' inner loops (FMA = 2):
# a node visit tests two child boxes (per box 6 FMA, 12 min/max, 1 mul,
# 1 compare), a triangle test is the watertight test (9 subtractions, 6 FMA
# for the shear, 6 mul + 3 sub for the edge functions, 2 add for the
# determinant, 6 mul + 2 FMA for the distance, 1 reciprocal, 3 mul).
FLOP_PER_NODE = 2 * (6 * 2 + 12 + 2)
FLOP_PER_TRI = 9 + 6 * 2 + 9 + 2 + 6 + 2 * 2 + 1 + 3
# GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA per clock (nominal)
SMS, FP32_LANES = 152, 128
# The L2 read bandwidth and FP32 FMA rate are measured in every run by the
# probe below (device_peaks()); the HBM copy bandwidth comes from
# MEASURED_PEAKS.json.
# algorithmic bytes of the traversal kernels, no cache credit: a node visit
# reads one 64-byte two-child node, a triangle test one 48-byte triangle; a
# closest-hit ray reads its 32-byte queue entry and writes a 28-byte hit, a
# shadow ray reads a 40-byte entry
BYTES_PER_NODE, BYTES_PER_TRI = 64, 48
BYTES_PER_RAY = {"k_trace_closest": 32 + 28, "k_trace_shadow": 40}
# DRAM traffic of the dominant traversal kernel per workload, from ncu
# captures of every launch of that kernel in one render at reduced spp
# (profiles/k_trace_closest_*.md): dram read + write bytes per traced ray,
# valid while the kernel's sources hash to sources_sha
TRAFFIC_CAPTURE = {
    "box_blob_material_256": {"kernel": "k_trace_closest",
                              "dram_bytes_per_ray": (2126.010368e6 + 445.262080e6) / 57820270.0,
                              "sources_sha": "ca6e970db6ab6a9a"},
    # the 72 launches of one 16 spp render (2^24-root waves, as at 256 spp)
    "terrain_motion_1024": {"kernel": "k_trace_closest",
                            "dram_bytes_per_ray": (22144.531712e6 + 4244.507392e6) / 223016348.0,
                            "sources_sha": "7b5999697f545cd7"},
}
KERNEL_SOURCES = ["rp_device.cuh", "wave_body.cuh", "k_wave.cu", "rp_internal.h", "rp_wave.h"]


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2406_16302_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]



# A standalone probe of the device peaks that the traversal roofline needs
# besides the HBM copy bandwidth: the read bandwidth of an L2-resident buffer
# (48 MB read 20 times per launch with __ldcg, which caches in L2 and not in
# L1) and the FP32 FMA rate (eight independent FMA chains per thread).  It
# prints one JSON object; compiled on first use into the package's build
# folder.
_PEAKS_CU = r"""
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_)); std::exit(1); } } while (0)
__global__ void l2_read(const float4 *__restrict__ buf, size_t n4, int reps, float *out) {
    float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += step) {
            const float4 v = __ldcg(buf + i);
            a += v.x; b += v.y; c += v.z; d += v.w;
        }
    if (a + b + c + d == -1.2345f) out[0] = a;
}
__global__ void fma_rate(float *out, int iters, float m, float k) {
    float x[8];
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], m, k);
    float s = 0.f;
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.2345f) out[0] = s;
}
__global__ void atomics(double *img, unsigned n_img, unsigned long long n_add) {
    const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n_add;
         i += step)
        atomicAdd(img + (unsigned)((i * 2654435761ull) % n_img), 1e-9);
}
template <class F> static float best_ms(F f, int runs) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
    f(); CK(cudaDeviceSynchronize());
    float best = 1e30f;
    for (int r = 0; r < runs; ++r) {
        CK(cudaEventRecord(a)); f(); CK(cudaEventRecord(b)); CK(cudaEventSynchronize(b));
        float ms = 0.f; CK(cudaEventElapsedTime(&ms, a, b)); if (ms < best) best = ms;
    }
    return best;
}
int main() {
    int dev = 0, sms = 0, l2 = 0, clk = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    float *out = nullptr; CK(cudaMalloc(&out, sizeof(float)));
    const size_t bytes = 48ull << 20, n4 = bytes / sizeof(float4);
    const int reps = 20;
    float4 *buf = nullptr; CK(cudaMalloc(&buf, bytes)); CK(cudaMemset(buf, 0, bytes));
    const float l2_ms = best_ms([&] { l2_read<<<sms * 8, 256>>>(buf, n4, reps, out); }, 5);
    CK(cudaGetLastError());
    const int iters = 1 << 16, blocks = sms * 8, threads = 256;
    const float f_ms = best_ms([&] { fma_rate<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f); }, 5);
    CK(cudaGetLastError());
    const unsigned n_img = 256u * 256u * 3u;
    const unsigned long long n_add = 1ull << 26;
    double *img = nullptr; CK(cudaMalloc(&img, sizeof(double) * n_img));
    CK(cudaMemset(img, 0, sizeof(double) * n_img));
    const float a_ms = best_ms([&] { atomics<<<sms * 8, 256>>>(img, n_img, n_add); }, 3);
    CK(cudaGetLastError());
    std::printf("{\"sms\": %d, \"l2_bytes\": %d, \"clock_mhz_attr\": %.0f, "
                "\"l2_read_gbs\": %.1f, \"l2_read_buffer_mb\": %zu, \"fp32_fma_tflops\": %.2f, "
                "\"fp64_atomic_gops\": %.2f, \"fp64_atomic_image\": \"256x256x3 doubles\"}\n",
                sms, l2, clk / 1e3, (double)bytes * reps / (l2_ms * 1e-3) / 1e9, bytes >> 20,
                16.0 * iters * (double)blocks * threads / (f_ms * 1e-3) / 1e12,
                (double)n_add / (a_ms * 1e-3) / 1e9);
    CK(cudaFree(buf)); CK(cudaFree(img)); CK(cudaFree(out));
    return 0;
}
"""

_PEAKS = None


def build_peak_probe():
    """Compile the probe (once per source version); returns the executable."""
    import hashlib
    from paper_2406_16302_gb300.build import ARCH, OUT_DIR, nvcc
    tag = hashlib.sha256(_PEAKS_CU.encode()).hexdigest()[:12]
    exe = os.path.join(OUT_DIR, f"bench_peaks_{tag}")
    if not os.path.exists(exe):
        os.makedirs(OUT_DIR, exist_ok=True)
        src = exe + ".cu"
        with open(src, "w") as f:
            f.write(_PEAKS_CU)
        r = subprocess.run([nvcc(), "-O3", "-std=c++17", src, "-o", exe] + ARCH,
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compiling the peak probe failed:\n{r.stderr}")
    return exe


def device_peaks():
    """L2 read bandwidth and FP32 FMA rate of this GPU, measured once per
    process by the probe above (a few hundred milliseconds)."""
    global _PEAKS
    if _PEAKS is None:
        out = subprocess.run([build_peak_probe()], capture_output=True, text=True,
                             check=True).stdout
        _PEAKS = json.loads(out.strip().splitlines()[-1])
    return _PEAKS


def workload(name):
    from paper_2406_16302_gb300 import scenes
    if name == "box_blob_material_256":
        scene, edit = scenes.cfg2_box_blob()
        return scene, edit, 64
    if name == "box_sphere_motion_64":
        scene, edit = scenes.cfg1_box_sphere()
        return scene, edit, 16
    if name == "box_sphere_motion_256":
        scene, edit = scenes.cfg1_box_sphere(width=256, height=256, max_depth=6)
        return scene, edit, 64
    if name == "terrain_motion_1024":
        scene, edit = scenes.cfg3_terrain()
        return scene, edit, 256
    if name == "batch_32_edits":
        # one item as a single-object problem (the oracle arm)
        scene, frames = batch_workload()
        edit, w, h, spp = frames[0]
        view = scenes.object_view(scene, edit.object)
        import dataclasses
        view = dataclasses.replace(view, camera=dataclasses.replace(view.camera, width=w, height=h))
        return view, dataclasses.replace(edit, object=0), spp
    if name == "box_blob_side_light_256":
        scene, edit = scenes.box_blob_side_light(width=256, height=256, max_depth=8, blob_level=5)
        return scene, edit, 64
    raise SystemExit(f"unknown workload {name}")


BATCH_SPP_SCALE = 32      # the batch workload's 64-256 spp divided by this in timed runs


def batch_workload(spp_scale=BATCH_SPP_SCALE):
    """32 animation frames, each moving one of 32 objects (1k-200k triangles)
    of the box scene, at 256^2..1024^2; spp 64-256 divided by spp_scale."""
    from paper_2406_16302_gb300 import scenes
    scene, frames = scenes.cfg4_batch()
    return scene, [(e, w, h, max(1, int(round(spp / spp_scale)))) for e, w, h, spp in frames]


def run_batch(args):
    """Batched edits: 32 animation frames, each moving one object of 1k-200k
    triangles at 256^2, 512^2 or 1024^2, at the configuration's spp divided by
    batch_spp_scale.  The autotuned batch (a graph of per-wave launches, or
    rounds of the persistent kernel) runs as one CUDA graph launch per step;
    beside it the other batch mode, the same items rendered one by one, the
    equal-time residual MSE of both on a sample of items against a converged
    reference, and a stated subset of the items at the configuration's full
    spp."""
    import dataclasses
    import torch
    from paper_2406_16302_gb300 import build, rp
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    rp.lib()
    scene, frames = batch_workload(args.batch_spp_scale)
    sc = rp.Scene(scene)
    edits = [rp.Edit(sc, f[0]) for f in frames]
    outs = [torch.zeros((h, w, 3), dtype=torch.float64, device="cuda") for _, w, h, _ in frames]
    items = [(edits[i], w, h, spp, 1000 * (rank + 1) + i, 15, outs[i])
             for i, (_, w, h, spp) in enumerate(frames)]
    samples = sum(spp * w * h * 8 for _, w, h, spp in frames)
    t0 = time.perf_counter()
    cfg, tune_ms = rp.rp_batch_autotune(sc, items, spp_divisor=8)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_launches(b, steps, warmup, seed_base, clk=None):
        for w in range(warmup):
            rp.rp_batch_launch(b)
        torch.cuda.synchronize()
        ts = []
        for k in range(steps):
            flush.zero_()
            rp.rp_batch_set_seeds(b, [seed_base * (k + 1) + i for i in range(len(b.items))])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rp.rp_batch_launch(b)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        rp.rp_batch_status(b)
        return float(np.mean(ts))

    def timed_render(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    batch = rp.Batch(sc, items, config=cfg)
    _, nodes = rp.rp_batch_info(batch)
    with ClockSampler(local) as clk:
        ms = timed_launches(batch, args.steps, args.warmup, 100000)
    # the other batch mode at its defaults
    other_cfg = (1 << 20, 8, 0, 1) if not cfg[3] else (min(1 << 22, max(spp * w * h for _, w, h, spp in frames)), 1, 16, 0)
    other = rp.Batch(sc, items, config=other_cfg)
    other_ms = timed_launches(other, 2, 1, 200000)
    del other
    # the same items one by one (each image size is a scene of its own camera)
    by_size = {}
    for _, w, h, _ in frames:
        if (w, h) not in by_size:
            by_size[(w, h)] = rp.Scene(dataclasses.replace(
                scene, camera=dataclasses.replace(scene.camera, width=w, height=h)))
    seq_ms = 0.0
    kern = {}
    work = {"nodes_closest": 0, "tris_closest": 0, "rays_closest": 0}
    for i, (f, w, h, spp) in enumerate(frames):
        s2 = by_size[(w, h)]
        e2 = rp.Edit(s2, f)
        out = torch.zeros((h, w, 3), dtype=torch.float64, device="cuda")
        rp.rp_enable_stats(s2, True)
        rp.rp_render_residual(s2, e2, spp, 7, out)
        st = rp.rp_get_stats(s2)
        rp.rp_enable_stats(s2, False)
        for key in work:
            work[key] += st[key]
        rp.rp_get_kernel_times(s2)
        rp.rp_enable_timing(s2, True)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rp.rp_render_residual(s2, e2, spp, 8, out)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        for name, (n, t) in rp.rp_get_kernel_times(s2).items():
            a_ = kern.setdefault(name, [0, 0.0])
            a_[0] += n
            a_[1] += t
        rp.rp_enable_timing(s2, False)
    # equal-time residual MSE on a sample of items: the batch's image of one
    # launch, the same item rendered alone with the same seed, against a
    # reference of 16 renders at 4x the item's spp; MSE x time is constant for
    # an unbiased estimator, so the equal-time ratio is MSE_b t_b / (MSE_1 t_1)
    sample = list(range(0, len(frames), 8))
    for o in outs:
        o.zero_()
    seeds = [300000 + i for i in range(len(items))]
    rp.rp_batch_set_seeds(batch, seeds)
    rp.rp_batch_launch(batch)
    torch.cuda.synchronize()
    mse = []
    for i in sample:
        f, w, h, spp = frames[i]
        s2 = by_size[(w, h)]
        e2 = rp.Edit(s2, f)
        alone = rp.render_residual(s2, e2, spp, seeds[i])
        ref = sum(rp.render_residual(s2, e2, 4 * spp, 400000 + 97 * i + r) for r in range(16)) / 16
        mb = float(((outs[i] - ref) ** 2).mean().item())
        m1 = float(((alone - ref) ** 2).mean().item())
        scale = float(alone.abs().max().item()) or 1.0
        mse.append({"item": i, "size": [w, h], "spp": spp, "mse_batch": mb, "mse_alone": m1,
                    "max_diff_rel": float((outs[i] - alone).abs().max().item()) / scale})
    mse_b = float(np.mean([m["mse_batch"] for m in mse]))
    mse_1 = float(np.mean([m["mse_alone"] for m in mse]))
    # a subset of the items at the configuration's full spp
    _, full = batch_workload(1)
    order = sorted(range(len(full)), key=lambda i: full[i][3] * full[i][1] * full[i][2])
    subset, budget = [], 0
    for i in order:
        e, w, h, spp = full[i]
        if budget + spp * w * h * 8 > 2.0e9:
            break
        subset.append(i)
        budget += spp * w * h * 8
    f_outs = [torch.zeros((full[i][2], full[i][1], 3), dtype=torch.float64, device="cuda")
              for i in subset]
    f_items = [(edits[i], full[i][1], full[i][2], full[i][3], 500000 + i, 15, f_outs[k])
               for k, i in enumerate(subset)]
    fb = rp.Batch(sc, f_items, config=cfg)
    full_ms = timed_launches(fb, 1, 1, 600000)
    del fb
    # the same 32 edits as small items (128 x 128, 16 spp: one wave of 2^18
    # roots per technique and frame, too small to fill the GPU alone): both
    # batch modes at their defaults and the items one by one
    small_scene = dataclasses.replace(scene, camera=dataclasses.replace(scene.camera, width=128,
                                                                       height=128))
    ssc = rp.Scene(small_scene)
    s_edits = [rp.Edit(ssc, f[0]) for f in frames]
    s_outs = [torch.zeros((128, 128, 3), dtype=torch.float64, device="cuda") for _ in frames]
    s_items = [(s_edits[i], 128, 128, 16, 700000 + i, 15, s_outs[i]) for i in range(len(frames))]
    small = {}
    for name, c in (("graph", (1 << 18, 4, 16, 0)), ("persistent", (1 << 18, 32, 0, 1))):
        b2 = rp.Batch(ssc, s_items, config=c)
        small[name] = {"config": list(c), "ms": timed_launches(b2, 3, 1, 800000)}
        del b2
    t_one = 0.0
    for i in range(len(frames)):
        o = torch.zeros((128, 128, 3), dtype=torch.float64, device="cuda")
        t_one += timed_render(lambda: rp.rp_render_residual(ssc, s_edits[i], 16, 900000 + i, o,
                                                            stream=stream))
    small["one_by_one"] = {"ms": t_one}
    small["samples"] = 128 * 128 * 16 * 8 * len(frames)
    n_launch, ms_tot = kern["k_trace_closest"]
    bytes_total = (work["nodes_closest"] * BYTES_PER_NODE + work["tris_closest"] * BYTES_PER_TRI
                   + work["rays_closest"] * BYTES_PER_RAY["k_trace_closest"])
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_total / n_launch / (ms_tot / n_launch / 1e3) / 1e9
    value = samples / (ms / 1e3)
    mode = "persistent" if cfg[3] else "graph"
    launches = nodes // 2 if cfg[3] else int(sum(v[0] for v in kern.values()))
    line = {
        "metric": "residual samples/s", "value": value, "unit": "residual samples/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch_32_edits", "items": len(frames),
                   "object_triangles": [int(r[1]) for r in scene.object_ranges],
                   "resolutions": [w for _, w, _, _ in frames],
                   "spp": [spp for *_, spp in frames],
                   "spp_scale": f"the configuration's 64-256 spp divided by {args.batch_spp_scale}",
                   "samples_per_step": samples, "graph_nodes": nodes,
                   "autotuned": {"mode": mode, "wave_roots": cfg[0], "streams": cfg[1],
                                 "blocks_per_sm": cfg[2], "proxy_ms": tune_ms, "tuning_s": tune_s},
                   "l2": "flushed between timed steps (256 MB write)"},
        "batch_vs_one_by_one": {"one_by_one_ms": seq_ms, "batch_ms": ms, "speedup": seq_ms / ms},
        "batch_modes": {mode: {"config": list(cfg), "ms": ms},
                        ("graph" if cfg[3] else "persistent"): {"config": list(other_cfg),
                                                                "ms": other_ms}},
        "equal_time_mse": {"items": mse, "reference": "16 renders at 4x the item's spp",
                           "mse_batch": mse_b, "mse_one_by_one": mse_1,
                           "ratio_at_equal_time": (mse_b * ms) / (mse_1 * seq_ms)},
        "small_items": small,
        "full_spp_subset": {"items": subset, "spp": [full[i][3] for i in subset],
                            "resolutions": [full[i][1] for i in subset],
                            "samples": budget, "ms": full_ms,
                            "samples_per_s": budget / (full_ms / 1e3),
                            "selection": "the smallest items by roots, up to 2e9 samples"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "kernel": "k_trace_closest",
                     "basis": "the items rendered one by one with per-kernel events",
                     "peak_basis": "hbm_gbs of MEASURED_PEAKS.json (measured copy bandwidth)"},
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sweep(args):
    """Hard-case sweeps on the cfg1 box (trend only; the paper's own table is
    on its scenes): `sweep_displacement` translates the sphere by d along x,
    `sweep_objects` moves 1, 2, 4 or 8 small objects at once (each by 0.1 in
    a seeded horizontal direction).  Per case: equal-time residual MSE of the
    residual estimator with the camera mapping (default), the
    object-transform mapping and without mapping, with the four and with all
    seven techniques, and of correlated path tracing, against a converged
    reference (all seven techniques at 16 x 64 spp)."""
    import torch
    from paper_2406_16302_gb300 import build, rp, scenes
    build.build()
    rp.lib()
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def cases():
        if args.workload == "sweep_objects":
            full = scenes.box_objects(width=128, height=128, max_depth=6)
            for k in (1, 2, 4, 8):
                yield {"moving_objects": k}, full, scenes.move_objects(full, k, 0.1)
        else:
            for d in (0.02, 0.05, 0.1, 0.2, 0.4):
                scene, edit = scenes.cfg1_box_sphere(width=128, height=128, max_depth=6)
                edit.M2 = edit.M1.copy()
                edit.M2[0, 3] += d
                yield {"displacement": d}, scene, edit

    spp, K, R = 16, 4, 16
    rows = []
    for key, scene, edit in cases():
        sc = rp.Scene(scene)
        ed = rp.Edit(sc, edit)

        def residual(s_, seed, mask, mapping=2):
            rp.rp_scene_set_mapping(sc, mapping)
            out = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
            t = timed(lambda: rp.rp_render_residual(sc, ed, s_, seed, out, tech_mask=mask, stream=stream))
            rp.rp_scene_set_mapping(sc, 2)
            return out, t

        def primal(frame, s_, seed):
            out = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
            return out, timed(lambda: rp.rp_render_primal(sc, ed, frame, s_, seed, out, stream=stream))

        ref = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
        for i in range(R):
            ref += residual(4 * spp, 800000 + i, 127)[0]
        ref /= R
        residual(spp, 809999, 15)                  # untimed: buffers at this root count
        row = dict(key)
        budget = None
        for name, mask, mapping in (("camera_4", 15, 2), ("object_4", 15, 1), ("off_4", 15, 0),
                                    ("camera_7", 127, 2), ("object_7", 127, 1)):
            ms, ts = [], []
            for k in range(K):
                img, t = residual(spp, 810000 + 10 * k, mask, mapping)
                ms.append(float(((img - ref) ** 2).mean().item()))
                ts.append(t)
            t = float(np.mean(ts))
            budget = budget or t
            row[name] = {"mse": float(np.mean(ms)), "ms": t, "mse_at_budget": float(np.mean(ms)) * t / budget}
        primal(1, spp, 829999)                  # untimed: allocates the primal wave buffers
        ms, ts = [], []
        for k in range(K):
            i2, ta = primal(2, spp, 820000 + k)
            i1, tb = primal(1, spp, 820000 + k)
            ms.append(float(((i2 - i1 - ref) ** 2).mean().item()))
            ts.append(ta + tb)
        t = float(np.mean(ts))
        row["correlated_pt"] = {"spp": spp, "mse": float(np.mean(ms)), "ms": t,
                                "mse_at_budget": float(np.mean(ms)) * t / budget}
        rows.append(row)
    desc = ("box_objects 128x128, max depth 6, objects moved by 0.1"
            if args.workload == "sweep_objects" else "cfg1_box_sphere 128x128, max depth 6")
    print(json.dumps({"experiment": args.workload, "scene": desc, "spp": spp, "repeats": K,
                      "reference": f"all seven techniques, {R} x {4 * spp} spp", "rows": rows}),
          flush=True)


def equal_time_mse(rp, sc, ed, scene, spp, K=4, ref_renders=16, guide_iters=30, guide_lr=1e-2):
    """Equal-time residual MSE against a converged reference (the plain
    method at ref_renders x 4 x spp, averaged over independent seeds).  Each
    method runs K times at its own sample count; its MSE is brought to the
    plain method's time T by MSE(T) = MSE(t) t / T (Monte Carlo variance
    falls as 1 / time).  Methods: the plain residual estimator; the same with
    the learned proposal after guide_iters online training iterations (the
    training time reported beside it); re-rendering frame 2 by path tracing
    against a converged frame 1; correlated path tracing (both frames with
    the same numbers)."""
    import torch
    from paper_2406_16302_gb300 import scenes
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def residual(s, seed):
        out = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
        return out, timed(lambda: rp.rp_render_residual(sc, ed, s, seed, out, stream=stream))

    def primal(frame, s, seed):
        out = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
        return out, timed(lambda: rp.rp_render_primal(sc, ed, frame, s, seed, out, stream=stream))

    ref = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
    for i in range(ref_renders):
        ref += residual(4 * spp, 700000 + i)[0]
    ref /= ref_renders

    def mse(img):
        return float(((img - ref) ** 2).mean().item())

    out = {"reference": f"plain residual, {ref_renders} x {4 * spp} spp averaged",
           "spp": spp, "repeats": K}
    # plain method
    ms, ts = [], []
    for k in range(K):
        img, t = residual(spp, 710000 + k)
        ms.append(mse(img)); ts.append(t)
    T = float(np.mean(ts))
    out["budget_ms"] = T
    out["plain"] = {"mse": float(np.mean(ms)), "ms": T, "mse_at_budget": float(np.mean(ms))}
    # path tracing re-render of frame 2 against a converged frame 1
    _, t1 = primal(2, spp, 720000)
    s_pt = max(1, int(round(spp * T / t1)))
    I1 = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
    for i in range(ref_renders):
        I1 += primal(1, 4 * spp, 730000 + i)[0]
    I1 /= ref_renders
    ms, ts = [], []
    for k in range(K):
        img, t = primal(2, s_pt, 740000 + k)
        ms.append(mse(img - I1)); ts.append(t)
    out["pt_rerender"] = {"spp": s_pt, "mse": float(np.mean(ms)), "ms": float(np.mean(ts)),
                          "mse_at_budget": float(np.mean(ms)) * float(np.mean(ts)) / T}
    # correlated path tracing: both frames with the same numbers
    s_c = max(1, s_pt // 2)
    ms, ts = [], []
    for k in range(K):
        i2, ta = primal(2, s_c, 750000 + k)
        i1, tb = primal(1, s_c, 750000 + k)
        ms.append(mse(i2 - i1)); ts.append(ta + tb)
    out["correlated_pt"] = {"spp": s_c, "mse": float(np.mean(ms)), "ms": float(np.mean(ts)),
                            "mse_at_budget": float(np.mean(ms)) * float(np.mean(ts)) / T}
    # all seven techniques (the ghost techniques (4)-(6) added; without
    # motion there is no ghost and this is the plain method again)
    ms, ts = [], []
    for k in range(K):
        o7 = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
        t = timed(lambda: rp.rp_render_residual(sc, ed, spp, 780000 + k, o7,
                                               tech_mask=rp.RP_TECH_SEVEN, stream=stream))
        ms.append(mse(o7)); ts.append(t)
    out["seven_techniques"] = {"mse": float(np.mean(ms)), "ms": float(np.mean(ts)),
                               "mse_at_budget": float(np.mean(ms)) * float(np.mean(ts)) / T}
    # learned proposal, trained online on the method's own samples
    box = scenes.guide_box(scene.dyn_vertices)
    batch = 1 << 20
    guide = rp.Guide(box, batch=batch, seed=1)
    rp.rp_scene_set_guide(sc, guide)
    s_train = max(1, (batch // 2 + sc.width * sc.height - 1) // (sc.width * sc.height))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for i in range(guide_iters):
        residual(s_train, 760000 + i)
        losses.append(rp.rp_guide_train_step(guide, lr=guide_lr))
    train_s = time.perf_counter() - t0
    ms, ts = [], []
    for k in range(K):
        img, t = residual(spp, 770000 + k)
        ms.append(mse(img)); ts.append(t)
    rp.rp_scene_set_guide(sc, None)
    out["guided"] = {"mse": float(np.mean(ms)), "ms": float(np.mean(ts)),
                     "mse_at_budget": float(np.mean(ms)) * float(np.mean(ts)) / T,
                     "training": {"iterations": guide_iters, "spp_per_iteration": s_train,
                                  "batch": batch, "seconds": train_s,
                                  "loss_first_last": [losses[0], losses[-1]]}}
    out["ratios_at_budget"] = {k: out[k]["mse_at_budget"] / out["plain"]["mse_at_budget"]
                               for k in ("guided", "pt_rerender", "correlated_pt",
                                         "seven_techniques") if k in out}
    return out


MSE_SPP = 16             # spp of each render in the equal-time MSE comparison


def e2e_calls(steps):
    """Calls timed by the end-to-end leg: half the timed steps, 3 to 10."""
    return max(3, min(10, steps // 2))


def bvh_footprint(scene):
    """Bytes of scene data the traversal kernels read: BVH nodes and leaf
    triangles of the static scene and the dynamic mesh (from the library's
    own host BVH builder) and the 48-byte triangles by id that the closest
    hit's refinement reads."""
    from paper_2406_16302_gb300 import rp
    total = 0
    for v, t in ((scene.static_vertices, scene.static_triangles),
                 (scene.dyn_vertices, scene.dyn_triangles)):
        if len(t):
            b = rp.rp_bvh_build_host(v, np.asarray(t, np.uint32))
            total += b["nodes"].nbytes + b["tris"].nbytes + 48 * len(t)
    return int(total)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(scene, edit, spp, target_s=15.0):
    """The oracle as it stands, single-threaded, on roots [0, R) of every
    technique in both frames, R grown until the run takes about target_s."""
    import oracle
    o = oracle.Oracle(scene, edit)
    R = 256
    while True:
        t0 = time.perf_counter()
        o.render_residual(spp, 1, 0, R)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or R >= o.n_roots(spp):
            break
        R = min(o.n_roots(spp), int(R * max(2.0, target_s / 4 / max(dt, 1e-3))))
    reps = max(1, int(target_s / max(dt, 1e-3)))
    t0 = time.perf_counter()
    for i in range(reps):
        o.render_residual(spp, 2 + i, 0, R)
    dt = (time.perf_counter() - t0) / reps
    return {"value": R * 8 / dt, "unit": "residual samples/s", "cores": 1, "kind": "oracle",
            "sample": f"roots [0, {R}) of each of the 4 techniques in both frames "
                      f"({R * 8} residual samples) per run, {reps} runs, single-threaded FP64 C",
            "roots": R, "n_roots": o.n_roots(spp)}


def compare_records(gpu, ora, rel=1e-4):
    """Per-sample agreement of two record sets keyed by (root, technique,
    frame, sa, sb): both splats on the same pixels and each value within
    rel of the sample's magnitude.  Returns (matching, total, max relative
    error over samples present on both sides)."""
    def key(r):
        return (int(r["root"]), int(r["tech"]), int(r["frame"]), int(r["sa"]), int(r["sb"]))
    go = {key(r): r for r in gpu}
    oo = {key(r): r for r in ora}
    good, worst = 0, 0.0
    for k in set(go) | set(oo):
        g, o = go.get(k), oo.get(k)
        if g is None or o is None:
            continue
        scale = max(float(np.abs(o["va"]).max()), float(np.abs(o["vb"]).max()), 1e-300)
        err = max(float(np.abs(g["va"] - o["va"]).max()), float(np.abs(g["vb"] - o["vb"]).max()))
        same_pix = g["pix_a"] == o["pix_a"] and g["pix_b"] == o["pix_b"]
        if same_pix:
            worst = max(worst, err / scale)
        if same_pix and err <= rel * scale:
            good += 1
    return good, len(set(go) | set(oo)), worst


def oracle_error(rp, sc, ed, scene, edit, spp, seed, ranges=8, width=32):
    """Error of the timed workload's samples against the FP64 oracle: the
    same seed's records of root ranges spread over the whole root range, every
    technique and both frames, compared sample by sample (this is the
    cpu_baseline leg's second use of the oracle)."""
    import oracle
    o = oracle.Oracle(scene, edit)
    N = sc.n_roots(spp)
    starts = np.linspace(0, N - width, ranges).astype(np.int64)
    good = total = 0
    worst = 0.0
    for tech in (1, 2, 3, 7):
        for frame in (1, 2):
            g = np.concatenate([rp.dump_samples(sc, ed, tech, frame, spp, seed, int(a), int(a) + width)
                                for a in starts])
            r = np.concatenate([o.dump(tech, frame, spp, seed, int(a), int(a) + width)
                                for a in starts])
            ng, nt, w = compare_records(g, r)
            good += ng
            total += nt
            worst = max(worst, w)
    return {"rel_tol": 1e-4, "samples": total, "within_tol": good / max(total, 1),
            "max_rel_err": worst, "roots": f"{ranges} ranges of {width} roots spread over [0, {N}) "
                                            f"per technique and frame, seed {seed}"}


def _oracle_worker(name, spp, a, R, seed, barrier, results):
    """One process of the multi-core oracle timing: roots [a, a+R) of every
    technique in both frames, started together with the others."""
    import oracle
    scene, edit, _ = workload(name)
    o = oracle.Oracle(scene, edit)
    o.render_residual(spp, seed, a, a + min(R, 16))          # page in, build the BVH
    barrier.wait()
    t0 = time.perf_counter()
    o.render_residual(spp, seed, a, a + R)
    results.put(time.perf_counter() - t0)


def cpu_baseline_multicore(name, spp, R, n_roots, cores=None):
    """The single-threaded oracle run in one spawned process per host core on
    disjoint root ranges of R roots each; value = all roots / the wall time
    from a common start to the last process's end."""
    import multiprocessing as mp
    if cores is None:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = max(1, min(cores, n_roots // max(R, 1)))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores + 1)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker,
                         args=(name, spp, i * R, R, 7 + i, barrier, results), daemon=True)
             for i in range(cores)]
    for p in procs:
        p.start()
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    per = [results.get(timeout=600) for _ in procs]
    wall = time.perf_counter() - t0
    for p in procs:
        p.join()
    return {"value": cores * R * 8 / wall, "unit": "residual samples/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} processes, each roots [{R}i, {R}(i+1)) of every technique in both "
                      f"frames ({cores * R * 8} residual samples), wall {wall:.2f} s "
                      f"(per process {min(per):.2f}-{max(per):.2f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    scene, edit, spp = workload(args.workload)
    import oracle
    o = oracle.Oracle(scene, edit)
    # size one step at about 10 s of CPU work
    R = 512
    t0 = time.perf_counter()
    o.render_residual(spp, 1, 0, R)
    dt = time.perf_counter() - t0
    N = o.n_roots(spp)
    R = min(N, max(64, int(R * 10.0 / max(dt, 1e-3))))

    def start(j):
        # successive steps take successive root ranges, wrapping inside [0, N)
        return (j * R) % (N - R) if N > R else 0

    for w in range(args.warmup):
        o.render_residual(spp, 100 + w, start(w), start(w) + R)
    times = []
    for k in range(args.steps):
        a = start(args.warmup + k)
        t0 = time.perf_counter()
        o.render_residual(spp, 1, a, a + R)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = R * 8 / (ms / 1e3)
    line = {"impl": "reference", "metric": "residual samples/s", "value": value,
            "unit": "residual samples/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "width": scene.camera.width,
                       "height": scene.camera.height, "spp": spp, "max_depth": scene.max_depth},
            "cpu_baseline": {"value": value, "unit": "residual samples/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"{R} roots of each technique in both frames per step"},
            "e2e": {"value": value, "unit": "residual samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="terrain_motion_1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mse", action="store_true", help="skip the equal-time MSE comparison")
    ap.add_argument("--spp", type=int, default=None, help="override the workload's spp "
                    "(smaller cases for profiling; not a benchmark number)")
    ap.add_argument("--batch-spp-scale", type=int, default=BATCH_SPP_SCALE,
                    help="divide the batch workload's spp by this")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_32_edits":
        return run_batch(args)
    if args.workload in ("sweep_displacement", "sweep_objects"):
        return run_sweep(args)
    if args.workload == "device_peaks":
        print(json.dumps(device_peaks()), flush=True)
        return

    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2406_16302_gb300 import build, rp
    from paper_2406_16302_gb300.dist import max_over_ranks
    if rank == 0 or ws == 1:
        build.build()
    if dist:
        dist.barrier()
    rp.lib()
    scene, edit, spp = workload(args.workload)
    if args.spp:
        spp = args.spp
    sc = rp.Scene(scene)
    ed = rp.Edit(sc, edit)
    N = sc.n_roots(spp)
    samples_per_step = N * 4 * 2
    stream = torch.cuda.current_stream()
    out = torch.zeros(sc.shape, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2
    seed0 = 1000 * (rank + 1)

    # algorithmic work of one step (untimed counting pass)
    rp.rp_enable_stats(sc, True)
    rp.rp_render_residual(sc, ed, spp, seed0, out, stream=stream)
    work = rp.rp_get_stats(sc)
    rp.rp_enable_stats(sc, False)

    def step(seed):
        rp.rp_render_residual(sc, ed, spp, seed, out, stream=stream)

    # warm-up; the last warm-up step brackets every launch with events (the
    # per-kernel breakdown), the timed steps only the dominant traversal
    # kernel's launches (its roofline), so that the timed region carries few
    # extra events
    n_warm = max(1, args.warmup)                # the breakdown needs one warm-up step
    for w in range(n_warm):
        if w == n_warm - 1:
            torch.cuda.synchronize()
            rp.rp_get_kernel_times(sc)                     # discard
            rp.rp_enable_timing(sc, True)
        step(seed0 + 1 + w)
    torch.cuda.synchronize()
    breakdown = rp.rp_get_kernel_times(sc)
    rp.rp_enable_timing(sc, False)
    trav = {"k_trace_closest": (work["nodes_closest"], work["tris_closest"], work["rays_closest"]),
            "k_trace_shadow": (work["nodes_shadow"], work["tris_shadow"], work["rays_shadow"])}
    dom = max(trav, key=lambda k: breakdown.get(k, (0, 0.0))[1])
    rp.rp_enable_timing_of(sc, dom)
    step_ms = []
    kern = {}
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()                       # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(seed0 + 100 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for name, (n, ms) in rp.rp_get_kernel_times(sc).items():
                a_ = kern.setdefault(name, [0, 0.0])
                a_[0] += n
                a_[1] += ms
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    rp.rp_enable_timing(sc, False)
    my_ms = float(np.mean(step_ms))
    worst_ms = max_over_ranks(my_ms, device="cuda")
    value = samples_per_step * ws / (worst_ms / 1e3)
    launches_per_step = sum(n for n, _ in breakdown.values())

    # end to end through the host-buffer entry point: edit upload, render,
    # image copy back, every step
    e2e = None
    if not args.no_e2e:
        host = np.zeros(sc.shape, dtype=np.float64)
        rp.rp_render_residual_host(sc, edit, spp, seed0, host)
        times = []
        for k in range(e2e_calls(args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp.rp_render_residual_host(sc, edit, spp, seed0 + 200 + k, host)
            times.append(time.perf_counter() - t0)
        e_ms = 1e3 * float(np.mean(times))
        e_ms = max_over_ranks(e_ms, device="cuda")
        e2e = {"value": samples_per_step * ws / (e_ms / 1e3), "unit": "residual samples/s",
               "h2d_bytes_per_step": 4 * 48, "d2h_bytes_per_step": int(host.nbytes),
               "ms_per_step": e_ms}

    # roofline of the dominant traversal kernel: its algorithmic bytes (node
    # visits, triangle tests, queue entries) per launch over its CUDA-event
    # time, against the L2 read bandwidth when the BVH fits in L2 and the
    # HBM copy bandwidth otherwise; FP32 work against the FMA rate beside it
    total_ms = max(sum(v[1] for v in breakdown.values()), 1e-9)
    per_kernel = {k: {"launches_per_step": n, "ms_per_step": ms, "share": ms / total_ms}
                  for k, (n, ms) in sorted(breakdown.items(), key=lambda kv: -kv[1][1])}
    n_launch, ms_tot = kern[dom]
    launch_ms = ms_tot / n_launch
    nodes, tris, rays = trav[dom]
    launches_one_step = n_launch / args.steps
    bytes_launch = (nodes * BYTES_PER_NODE + tris * BYTES_PER_TRI
                    + rays * BYTES_PER_RAY[dom]) / launches_one_step
    flops_launch = (nodes * FLOP_PER_NODE + tris * FLOP_PER_TRI) / launches_one_step
    peaks = measured_peaks()
    probe = device_peaks()
    clock = clk.summary()
    peak_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = probe["sms"] * FP32_LANES * 2 * peak_mhz * 1e6 / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_launch / (launch_ms / 1e3) / 1e9
    footprint = bvh_footprint(scene)
    l2_resident = footprint <= probe["l2_bytes"]
    traffic = None
    cap = TRAFFIC_CAPTURE.get(args.workload)
    if cap and dom == cap["kernel"] and kernel_sources_sha() == cap["sources_sha"]:
        # DRAM bytes per traced ray of an ncu capture of the same kernel,
        # scaled to this launch by its rays
        traffic = cap["dram_bytes_per_ray"] * rays / launches_one_step
    achieved_tf = flops_launch / (launch_ms / 1e3) / 1e12
    hbm_basis = ("hbm_gbs of MEASURED_PEAKS.json (measured copy bandwidth)"
                 if "hbm_gbs" in peaks else "fallback 6800 GB/s (MEASURED_PEAKS.json absent)")
    l2_basis = "L2 read bandwidth measured in this run (48 MB resident buffer, __ldcg)"
    roofline = {"bound": "l2" if l2_resident else "hbm", "achieved": achieved,
                "peak": probe["l2_read_gbs"] if l2_resident else hbm, "unit": "GB/s",
                "frac": achieved / (probe["l2_read_gbs"] if l2_resident else hbm),
                "traffic": traffic, "kernel": dom, "launch_ms": launch_ms,
                "peak_basis": l2_basis if l2_resident else hbm_basis,
                "bvh_footprint_bytes": footprint, "l2_bytes": probe["l2_bytes"],
                "bytes_per_launch": bytes_launch,
                "work_per_launch": {"node_visits": nodes / launches_one_step,
                                    "triangle_tests": tris / launches_one_step,
                                    "rays": rays / launches_one_step,
                                    "bytes_per_node": BYTES_PER_NODE, "bytes_per_tri": BYTES_PER_TRI,
                                    "bytes_per_ray": BYTES_PER_RAY[dom]},
                "hbm": {"achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                        "peak_basis": hbm_basis},
                "l2": {"achieved": achieved, "peak": probe["l2_read_gbs"], "unit": "GB/s",
                       "frac": achieved / probe["l2_read_gbs"], "peak_basis": l2_basis},
                "fp32": {"achieved_tflops": achieved_tf, "peak_tflops": peak_tflops,
                         "frac": achieved_tf / peak_tflops,
                         "measured_peak_tflops": probe["fp32_fma_tflops"],
                         "frac_of_measured": achieved_tf / probe["fp32_fma_tflops"],
                         "basis": f"{probe['sms']} SMs x 128 lanes x 2 flop x {peak_mhz:.0f} MHz; "
                                  f"{FLOP_PER_NODE} flop per node, {FLOP_PER_TRI} per triangle"},
                "share_of_step": breakdown[dom][1] / total_ms,
                "timing": "the kernel's own launches bracketed by CUDA events on the render "
                          "stream in every timed step (no other launch is)"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    err = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(scene, edit, spp)
        cpu["multi_core"] = cpu_baseline_multicore(args.workload, spp, cpu["roots"],
                                                   cpu["n_roots"])
        err = oracle_error(rp, sc, ed, scene, edit, spp, seed0 + 100)
    et_mse = None
    if not args.no_mse and ws == 1:
        et_mse = equal_time_mse(rp, sc, ed, scene, min(spp, MSE_SPP))
    line = {
        "metric": "residual samples/s", "value": value, "unit": "residual samples/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": worst_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "width": scene.camera.width,
                   "height": scene.camera.height, "spp": spp, "max_depth": scene.max_depth,
                   "triangles": scene.n_static + scene.n_dyn, "edit": edit.name,
                   "techniques": "1,2,3,7", "roots_per_technique_frame": N,
                   "samples_per_step": samples_per_step, "accumulation": "fp64 atomics",
                   "l2": "flushed between timed steps (256 MB write)",
                   "per_kernel": per_kernel,
                   "per_kernel_basis": "one warm-up step with every launch bracketed by CUDA "
                                       "events (not the timed steps)",
                   "rays_per_step": work["rays_closest"] + work["rays_shadow"],
                   "paths_per_step": work["paths"],
                   # splatted base paths per pixel (the paper's spp convention, Sec. 6)
                   "spp_equivalent": work["paths"] / (scene.camera.width * scene.camera.height)},
        "root_samples_per_s": value,
        "roofline": roofline, "cpu_baseline": cpu, "oracle_error": err, "e2e": e2e,
        "equal_time_mse": et_mse,
        "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clock,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
