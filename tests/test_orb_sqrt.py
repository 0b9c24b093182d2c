"""The FP32 moment magnitude of the orientation (next row f3) is computed on
the device without double precision (ft_sqrt.h: an FP32 square root settled
by exact integer comparisons).  The header's host form is compiled here with
g++ and compared, bit for bit, with the reading's definition
float(sqrt((double)n)): every n up to 2^22, the perfect squares up to 2^41
and their neighbours, integers next to the squares of float midpoints, and
random n below 2^41."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_10757_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <random>
#include "ft_sqrt.h"
static uint64_t bad = 0, checked = 0;
static void check(uint64_t n) {
    if (n == 0 || n >= (1ull << 41)) return;
    const float want = (float)std::sqrt((double)n), got = ft::float_sqrt_rn(n);
    ++checked;
    if (ft::ft_float_bits(want) != ft::ft_float_bits(got)) {
        if (bad < 5) std::printf("n=%llu want %.9g got %.9g\n", (unsigned long long)n, want, got);
        ++bad;
    }
}
int main() {
    for (uint64_t n = 1; n <= (1ull << 22); ++n) check(n);
    for (uint64_t k = 1; k * k < (1ull << 41); ++k) { check(k * k - 1); check(k * k); check(k * k + 1); }
    std::mt19937_64 rng(7);
    for (int i = 0; i < 4000000; ++i) {
        // a float midpoint in [1, 2^20.5): odd multiple of half a unit in the last place
        const int e = (int)(rng() % 21);
        const uint64_t j = (rng() & 0x7fffffull) | 0x800000ull;           // 24-bit significand
        const long double m = (long double)(2 * j + 1) * std::ldexp(1.0L, e - 24);
        const long double sq = m * m;
        const uint64_t f = (uint64_t)std::floor(sq);
        check(f); check(f + 1);
        check(rng() % (1ull << 41));
    }
    std::printf("checked %llu bad %llu\n", (unsigned long long)checked, (unsigned long long)bad);
    return bad != 0;
}
"""


def test_float_sqrt_matches_the_double_definition(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    src = tmp_path / "sqrt_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "sqrt_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout
