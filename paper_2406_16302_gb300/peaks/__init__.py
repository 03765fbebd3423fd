"""Device peaks for the traversal roofline beside the measured HBM copy
bandwidth: L2-resident read bandwidth, FP32 FMA throughput and FP64
atomicAdd throughput (``peaks.cu``, a standalone program).

    python -m paper_2406_16302_gb300.peaks      # prints one JSON line
"""
from __future__ import annotations

import json
import os
import subprocess

from ..build import ARCH, OUT_DIR, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))
EXE = os.path.join(OUT_DIR, "peaks")


def build() -> str:
    src = os.path.join(HERE, "peaks.cu")
    if os.path.exists(EXE) and os.path.getmtime(EXE) >= os.path.getmtime(src):
        return EXE
    os.makedirs(OUT_DIR, exist_ok=True)
    cmd = [nvcc(), "-O3", "-std=c++17", "--extended-lambda", src, "-o", EXE] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling peaks.cu failed:\n{r.stdout}\n{r.stderr}")
    return EXE


def measure() -> dict:
    out = subprocess.run([build()], capture_output=True, text=True, check=True).stdout
    return json.loads(out.strip().splitlines()[-1])
