"""The integer rounding of an FP64 product to FP32 used by the residual's load-only kernel
(`csrc/f64_round.cuh`), compiled for the host: it must give (float)(a * b) of FP64 arithmetic -- the
exact product rounded to 53 bits, then to 24, both to nearest even -- bit for bit, or decline (the
kernel then uses FP64 arithmetic).  Random operands: arbitrary bit patterns, moderate exponents, and
short mantissas whose products land on rounding ties at either step."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1805_06688_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include <math.h>
#include "f64_round.cuh"
static uint64_t s = 88172645463325252ull;
static uint64_t rnd() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
static double make(int mode) {
    uint64_t u = rnd();
    if (mode > 0) {
        const int e = (int)(rnd() % 80) - 40 + 1023;          // moderate exponents
        u = (u & 0x800FFFFFFFFFFFFFull) | ((uint64_t)e << 52);
        if (mode == 2) u &= ~0x1FFFFFFFull;                   // products near a 53-bit tie
        if (mode == 3) u &= ~0xFFFFFFFFFFull;                 // products near a 24-bit tie
    }
    double d;
    memcpy(&d, &u, 8);
    return d;
}
int main() {
    long bad = 0, done = 0, declined = 0;
    for (int mode = 0; mode < 4; ++mode)
        for (long i = 0; i < 1000000; ++i) {
            double a = make(mode), b = make(mode);
            if (i % 997 == 0) a = 0.0;
            if (i % 991 == 0) b = -0.0;
            volatile double p = a * b;
            const float ref = (float)p;
            float got;
            if (!sfde_round::mul_f64_to_f32(a, b, got)) { ++declined; continue; }
            ++done;
            uint32_t g, r;
            memcpy(&g, &got, 4);
            memcpy(&r, &ref, 4);
            if (g != r) ++bad;
        }
    printf("%ld %ld %ld\n", done, bad, declined);
    return 0;
}
"""


def test_fp64_product_rounded_to_fp32_in_integers(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:  # pragma: no cover
        pytest.skip("no host C++ compiler")
    src = tmp_path / "round_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "round_check"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    done, bad, declined = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.split())
    assert bad == 0
    assert done > 3_000_000          # only non-finite, subnormal or out-of-range cases decline
    assert declined < 1_000_000
