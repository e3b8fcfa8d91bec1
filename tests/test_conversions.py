"""The FP32 <-> FP64 conversions the kernels run on the integer pipe
(common.cuh: f32_to_f64, f64_to_f32, written on the IEEE-754 bit fields)
compiled for the host from the same header (by nvcc, as host code) and held against the host's own
conversions (IEEE-754 round to nearest, ties to even) on random bit patterns
of every class: normals across the whole exponent range, values near the
binary32 limits, ties, subnormals, zeros and infinities (NaN only as NaN)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include "common.cuh"
#include <stdio.h>
using namespace hdmd;
static uint64_t s = 88172645463325252ull;
static uint64_t rnd() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
int main() {
    long bad = 0, n = 0;
    for (long i = 0; i < 4000000; ++i) {
        uint64_t b = rnd();
        const int mode = (int)(i % 5);
        if (mode == 1) b = (b & 0x800fffffffffffffull) | ((uint64_t)(800 + rnd() % 360) << 52);
        if (mode == 2) b = (b & ~0x1fffffffull & 0x800fffffffffffffull) | 0x10000000ull | ((uint64_t)(860 + rnd() % 60) << 52);
        if (mode == 3) b = (b & 0x800fffffffffffffull) | ((uint64_t)(1003 + rnd() % 20) << 52);
        if (mode == 4) b = (b & 0x800fffffffffffffull) | ((uint64_t)(rnd() % 2 ? 0 : 0x7ff) << 52);
        const double x = f64_bits(b);
        const float a = f64_to_f32(x), h = (float)x;
        if (!(x != x) && bits_f32(a) != bits_f32(h)) ++bad;
        if ((x != x) && !(a != a)) ++bad;
        const float f = f32_bits((uint32_t)rnd());
        const double y = f32_to_f64(f), z = (double)f;
        if (!(f != f) && bits_f64(y) != bits_f64(z)) ++bad;
        if ((f != f) && !(y != y)) ++bad;
        ++n;
    }
    printf("%ld %ld\n", n, bad);
    return 0;
}
'''


def test_bit_field_conversions_equal_the_host_conversions(tmp_path):
    from paper_2112_12271_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc is missing")
    src = tmp_path / "t.cu"
    src.write_text(SRC)
    exe = tmp_path / "t"
    # host code of the kernels' header (main runs on the CPU)
    subprocess.check_call([nvcc] + build.ARCH + ["-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2112_12271_gb300", "csrc"),
                           "-o", str(exe), str(src)])
    n, bad = (int(t) for t in subprocess.check_output([str(exe)], text=True).split())
    assert n == 4000000 and bad == 0
