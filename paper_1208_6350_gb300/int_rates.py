"""Measures the integer SIMD issue rates the fill design rests on.

Compiles csrc_bench/int_rates.cu for sm_103a and runs it on the current GPU:
lane operations per clock per SM for s32 / s16x2 max, DPX add-max forms,
video SIMD u8x4 forms, PRMT and LOP3.

    python -m paper_1208_6350_gb300.int_rates
"""
import os
import subprocess
import sys

from . import _build

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc_bench", "int_rates.cu")
EXE = os.path.join(_build.OUT, "int_rates")


def main():
    os.makedirs(_build.OUT, exist_ok=True)
    subprocess.run([_build.nvcc()] + _build.ARCH + ["-O3", SRC, "-o", EXE], check=True)
    return subprocess.run([EXE]).returncode


if __name__ == "__main__":
    sys.exit(main())
