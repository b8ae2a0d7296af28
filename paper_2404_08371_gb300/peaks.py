"""Measure the roofline denominators of this GPU: FP64 / FP32 FMA-chain throughput and a streaming copy.

    python -m paper_2404_08371_gb300.peaks

Compiles peaks.cu with nvcc for sm_103a into _build/ and prints its JSON line.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def measure() -> str:
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "peaks")
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "peaks.cu")], check=True)
    return subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip()


if __name__ == "__main__":
    print(measure())
