"""Benchmark: residual samples/s of the residual path integral estimator on GB300.

Workload (default): the material-edit box scene at 256x256, 64 spp, max depth
8 -- a Cornell-style box with a static sphere and a 20480-triangle seeded
blob that changes from Lambert (albedo 0.8) to GGX (alpha 0.3, F0 0.04);
techniques (1), (2), (3) and path tracing with rejection, both frames.

One step = one residual render of the whole image (every root of every
technique in both frames: 8 kernel launches).  A residual sample = one root
of one technique in one frame, with every base path it generates, their
mapped paths, MIS denominators and splats; a step processes
spp * W * H * 4 * 2 of them.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
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
# GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA per clock
SMS, FP32_LANES = 152, 128

TECHS = [(1, 1), (2, 2), (3, 4), (7, 8)]   # (technique, mask bit)


def workload(name):
    from paper_2406_16302_gb300 import scenes
    if name == "box_blob_material_256":
        scene, edit = scenes.cfg2_box_blob()
        return scene, edit, 64
    if name == "box_sphere_motion_64":
        scene, edit = scenes.cfg1_box_sphere()
        return scene, edit, 16
    if name == "terrain_motion_1024":
        scene, edit = scenes.cfg3_terrain()
        return scene, edit, 16
    raise SystemExit(f"unknown workload {name}")


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
                      f"({R * 8} residual samples) per run, {reps} runs, single-threaded FP64 C"}


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
    R = max(64, int(R * 10.0 / max(dt, 1e-3)))
    N = o.n_roots(spp)
    for w in range(args.warmup):
        o.render_residual(spp, 100 + w, (w * R) % (N - R), (w * R) % (N - R) + R)
    times = []
    for k in range(args.steps):
        a = ((args.warmup + k) * R) % (N - R)
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
    ap.add_argument("--workload", default="box_blob_material_256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--spp", type=int, default=None, help="override the workload's spp "
                    "(smaller cases for profiling; not a benchmark number)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

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

    # algorithmic work per technique launch pair (untimed counting pass)
    rp.rp_enable_stats(sc, True)
    work = {}
    for tech, mask in TECHS:
        rp.rp_render_residual(sc, ed, spp, seed0, out, tech_mask=mask)
        work[tech] = rp.rp_get_stats(sc)
    rp.rp_enable_stats(sc, False)

    def step(seed, events=None):
        for tech, mask in TECHS:
            if events is not None:
                events[tech][0].record(stream)
            rp.rp_render_residual(sc, ed, spp, seed, out, tech_mask=mask, stream=stream)
            if events is not None:
                events[tech][1].record(stream)

    for w in range(args.warmup):
        step(seed0 + 1 + w)
    torch.cuda.synchronize()
    per_tech = {t: 0.0 for t, _ in TECHS}
    step_ms = []
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()                       # evict L2 between timed steps
            ev = {t: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for t, _ in TECHS}
            step(seed0 + 100 + k, ev)
            torch.cuda.synchronize()
            ms = {t: ev[t][0].elapsed_time(ev[t][1]) for t, _ in TECHS}
            for t in ms:
                per_tech[t] += ms[t]
            step_ms.append(sum(ms.values()))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    my_ms = float(np.mean(step_ms))
    worst_ms = my_ms
    if dist:
        t = torch.tensor([my_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        worst_ms = float(t.item())
    value = samples_per_step * ws / (worst_ms / 1e3)

    # end to end through the host-buffer entry point: edit upload, render,
    # image copy back, every step
    e2e = None
    if not args.no_e2e:
        host = np.zeros(sc.shape, dtype=np.float64)
        rp.rp_render_residual_host(sc, edit, spp, seed0, host)
        times = []
        for k in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp.rp_render_residual_host(sc, edit, spp, seed0 + 200 + k, host)
            times.append(time.perf_counter() - t0)
        e_ms = 1e3 * float(np.mean(times))
        if dist:
            t = torch.tensor([e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": samples_per_step * ws / (e_ms / 1e3), "unit": "residual samples/s",
               "h2d_bytes_per_step": 4 * 48, "d2h_bytes_per_step": int(host.nbytes),
               "ms_per_step": e_ms}

    # roofline of the dominant kernel (the technique with the largest time)
    dom = max(per_tech, key=per_tech.get)
    dom_ms = per_tech[dom] / args.steps / 2          # one launch per frame
    w = work[dom]
    flops_launch = (w["nodes_visited"] * FLOP_PER_NODE + w["tris_tested"] * FLOP_PER_TRI) / 2
    peaks = measured_peaks()
    clock = clk.summary()
    peak_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = SMS * FP32_LANES * 2 * peak_mhz * 1e6 / 1e12
    achieved = flops_launch / (dom_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "kernel": f"k_roots_{dom}", "launch_ms": dom_ms,
                "peak_basis": f"152 SMs x 128 FP32 lanes x 2 flop x {peak_mhz:.0f} MHz "
                              "(sm_max_mhz of MEASURED_PEAKS.json)",
                "work_per_launch": {"node_visits": w["nodes_visited"] // 2,
                                    "triangle_tests": w["tris_tested"] // 2,
                                    "rays": (w["rays_closest"] + w["rays_shadow"]) // 2,
                                    "flop_per_node": FLOP_PER_NODE, "flop_per_tri": FLOP_PER_TRI},
                "share_of_step": per_tech[dom] / sum(per_tech.values())}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(scene, edit, spp)
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
                   "per_technique_ms": {str(t): per_tech[t] / args.steps for t in per_tech}},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 8 * args.steps, "clocks": clock,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
