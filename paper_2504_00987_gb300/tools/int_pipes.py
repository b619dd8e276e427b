"""Builds and runs the integer-pipe probe (int_pipes.cu) on the current GPU:

    python -m paper_2504_00987_gb300.tools.int_pipes
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    from paper_2504_00987_gb300 import _build

    out_dir = os.path.join(os.path.dirname(HERE), "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "int_pipes")
    subprocess.check_call([_build.nvcc_path(), *_build.ARCH, "-O3", "-o", exe, os.path.join(HERE, "int_pipes.cu")])
    return subprocess.call([exe])


if __name__ == "__main__":
    sys.exit(main())
