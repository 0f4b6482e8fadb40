"""Host check of the boundary-phase mask the hop kernels use to skip the
multiplication by a phase of exactly 1 (phase_mask in the library's internal
header): bit mu is clear exactly when direction mu's phase is (1, 0), for
periodic, antiperiodic, twisted and nearly-1 phases.  No GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_2039_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include "wd_internal.cuh"
int main() {
    using namespace wd;
    struct Case { double ph[8]; unsigned want; };
    const double e = std::nextafter(1.0, 2.0);
    const Case cases[] = {
        {{1, 0, 1, 0, 1, 0, 1, 0}, 0x0u},                                   // periodic
        {{1, 0, 1, 0, 1, 0, -1, 0}, 0x8u},                                  // antiperiodic in t
        {{std::cos(0.3), std::sin(0.3), 1, 0, std::cos(-0.9), std::sin(-0.9), -1, 1e-16}, 0xDu},
        {{e, 0, 1, 1e-300, 1, -0.0, 0, 1}, 0xBu},                          // 1 + ulp, tiny imag, -0, i
        {{-1, 0, -1, 0, -1, 0, -1, 0}, 0xFu},
    };
    int bad = 0;
    for (const Case &c : cases) {
        const unsigned m = phase_mask(c.ph);
        if (m != c.want) { std::printf("mask %x want %x\n", m, c.want); ++bad; }
    }
    std::printf("%d\n", bad);
    return bad != 0;
}
"""


def test_phase_mask_marks_every_phase_that_is_not_exactly_one(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "mask.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "mask"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().splitlines()[-1] == "0", r.stdout
