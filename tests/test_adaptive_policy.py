"""The rule by which an adaptive mixed-precision step chooses its FP32
V-cycles (mg_next_inner, shared by the solve graph's control kernel and the
host-driven loop), compiled for the host from the library's own header and
checked on cases whose answer follows from the per-cycle contraction."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

CASES = [
    # rel_before, rel_after, ran, tol, inner_max, expected
    (1.0, 1e-3, 3, 1e-10, 8, 8),        # 0.1 per cycle: seven more cycles reach 1e-10, one spare after 3
    (1.0, 2e-3, 3, 1e-10, 12, 10),      # 0.126 per cycle: 8.1 cycles -> 9, one spare
    (1.0, 1e-3, 4, 1e-10, 12, 10),      # 0.178 per cycle over 4 cycles: 9.33 cycles -> 10, no spare
    (1e-4, 1e-7, 3, 1e-10, 8, 4),       # 0.1 per cycle: 3 cycles, one spare
    (1.0, 1e-3, 3, 1e-10, 5, 5),        # the cap
    (1.0, 0.125, 3, 1e-10, 8, 8),       # slow contraction: the cap
    (1e-3, 1e-3, 3, 1e-10, 8, 8),       # no contraction: the cap
    (1e-3, 2e-3, 3, 1e-10, 8, 8),       # growth: the cap
    (1.0, 1e-3, 3, 0.0, 8, 8),          # no tolerance to aim at: the cap
    (1e-3, 1e-11, 3, 1e-10, 8, 1),      # already below the tolerance
    (1.0, 1e-3, 0, 1e-10, 8, 8),        # no cycles ran
    (1e-2, 1e-9, 4, 1e-10, 8, 1),       # 1e-7 per 4 cycles: one more cycle suffices
]


def test_next_inner_policy(tmp_path):
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "policy.cpp"
    lines = ['#include "mg_internal.h"', "#include <cstdio>", "int main()", "{"]
    for rb, ra, ran, tol, cap, _ in CASES:
        lines.append(f'    std::printf("%d\\n", mg_next_inner({rb!r}, {ra!r}, {ran}, {tol!r}, {cap}));')
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "policy"
    subprocess.run([gxx, "-std=c++17", "-I", os.path.join(ROOT, "paper_2001_02327_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=30).stdout.split()
    got = [int(v) for v in out]
    assert got == [c[-1] for c in CASES], list(zip(CASES, got))
