"""Build and run the arithmetic-pipe probe (csrc/fp_peaks.cu) on the current GPU.

    python -m paper_1909_00101_gb300.fp_peaks

Prints one JSON object: DFMA, DMMA (FP64 mma.sync), FFMA and mma.sync (TF32,
BF16, FP16, S8 inputs) throughput, and FP64 DFMA/sqrt/division time with 1, 4, 8, 16, 32 active
lanes per warp (equal times = cost per warp instruction, not per lane).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    out = os.path.join(HERE, "_build", "fp_peaks")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    src = os.path.join(HERE, "csrc", "fp_peaks.cu")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", out, src])
    sys.exit(subprocess.call([out]))


if __name__ == "__main__":
    main()
