"""Host check of the multiply-and-shift division the kernels use for site
coordinates (Geom::div_hx, div_y, div_z) and batch items (BtProb::div_nrhs).

The test compiles a host-only program against the library's internal header
and compares udiv(n, make_divisor(d)) with n / d for every divisor up to the
largest lattice extent (2^14), at every multiple-boundary n = k d - 1, k d
for k spread over the range, and at the largest index 2^31 - 1.  No GPU is
used.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_2039_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "wd_internal.cuh"
int main() {
    using namespace wd;
    long bad = 0, checked = 0;
    const unsigned NMAX = 0x7fffffffu;
    for (unsigned d = 1; d <= (1u << 14); ++d) {
        const Divisor v = make_divisor(d);
        if (v.s < 31 || v.s > 63) { ++bad; continue; }
        const unsigned kmax = NMAX / d;
        for (unsigned t = 0; t <= 64; ++t) {
            const unsigned k = (unsigned)((unsigned long long)kmax * t / 64);
            for (int e = -1; e <= 1; ++e) {
                const long long n = (long long)k * d + e;
                if (n < 0 || n > NMAX) continue;
                ++checked;
                if (udiv((unsigned)n, v) != (unsigned)n / d) ++bad;
            }
        }
        ++checked;
        if (udiv(NMAX, v) != NMAX / d) ++bad;
        for (unsigned n = 0; n < 3 * d && n < 4096; ++n) {
            ++checked;
            if (udiv(n, v) != n / d) ++bad;
        }
    }
    std::printf("%ld %ld\n", checked, bad);
    return bad != 0;
}
"""


def test_multiply_shift_division_matches_integer_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "div.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "div"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    checked, bad = (int(v) for v in r.stdout.split())
    assert checked > 10_000_000
    assert bad == 0 and r.returncode == 0
