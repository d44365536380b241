"""Build and run the arithmetic-peak / latency microbenchmark (peaks.cu).

    python -m paper_1902_10078_gb300.microbench.peaks

prints one JSON object: FP32 and FP64 FMA throughput, DMMA (FP64 mma.sync)
and TF32 mma.sync throughput, and the cycles of dependent FP32/FP64 FMA,
sqrt, rsqrt, division and reciprocal chains.  The binary goes to _build/.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(HERE, "peaks.cu")
BIN = os.path.join(ROOT, "_build", "peaks")


def build() -> str:
    from paper_1902_10078_gb300.build import ARCH, nvcc
    if os.path.exists(BIN) and os.path.getmtime(BIN) >= os.path.getmtime(SRC):
        return BIN
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    subprocess.run([nvcc()] + ARCH + ["-O3", "-std=c++17", "-o", BIN, SRC], check=True)
    return BIN


def run() -> dict:
    out = subprocess.run([build()], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    print(json.dumps(run()))
