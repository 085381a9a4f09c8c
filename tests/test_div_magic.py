"""Host check of div_magic (csrc/lbm_internal.h): the multiply-and-shift constants with which the
multi-domain density pass turns a cell index into (x, y, z).  Granlund and Montgomery (PLDI 1994,
Thm. 4.2) make floor(n / d) = (n * m) >> s exact for every n < 2^31; this test compiles the header
with the host compiler and compares against integer division for divisors 1 .. 2000, powers of two
and their neighbours, and large extents, on boundary numerators (multiples of d and their
neighbours, 2^31 - 1) and pseudo-random ones."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "lbm_internal.h"
#include <cstdio>
#include <vector>

static bool check(uint32_t d, uint32_t n, uint32_t m, int s) {
    const uint32_t q = (uint32_t)(((unsigned long long)m * n) >> s);
    if (q != n / d) {
        std::printf("mismatch d=%u n=%u got %u want %u (m=%u s=%d)\n", d, n, q, n / d, m, s);
        return false;
    }
    return true;
}

int main() {
    std::vector<uint32_t> ds;
    for (uint32_t d = 1; d <= 2000; ++d) ds.push_back(d);
    for (int k = 11; k <= 30; ++k) {
        ds.push_back((1u << k) - 1);
        ds.push_back(1u << k);
        ds.push_back((1u << k) + 1);
    }
    for (uint32_t d : {1290u * 1290u, 65535u, 65536u * 3u, 2147483647u, 1073741825u}) ds.push_back(d);
    unsigned long long checks = 0, x = 88172645463325252ull;
    for (uint32_t d : ds) {
        uint32_t m;
        int s;
        lbm::div_magic(d, m, s);
        if (s < 31 || s > 62) { std::printf("shift %d out of range for d=%u\n", s, d); return 1; }
        const uint32_t top = 2147483647u;
        std::vector<uint32_t> ns = {0u, 1u, d - 1, d, d + 1, top, top - 1, top - d};
        for (uint32_t k = top / d; k + 3 > top / d && k > 0; --k) {
            const unsigned long long a = (unsigned long long)k * d;
            if (a <= top) ns.push_back((uint32_t)a);
            if (a - 1 <= top) ns.push_back((uint32_t)(a - 1));
            if (a + 1 <= top) ns.push_back((uint32_t)(a + 1));
        }
        for (int r = 0; r < 2000; ++r) {   // xorshift64
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            ns.push_back((uint32_t)(x % (top + 1ull)));
        }
        for (uint32_t n : ns) {
            if (n > top) continue;
            if (!check(d, n, m, s)) return 1;
            ++checks;
        }
    }
    std::printf("ok %llu\n", checks);
    return 0;
}
"""


def test_div_magic_is_exact_below_2_31(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    from paper_2306_16274_gb300 import build
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    if not os.path.isfile(os.path.join(cuda_inc, "cuda.h")):
        pytest.skip("CUDA headers not found")
    src = tmp_path / "div_magic.cpp"
    exe = tmp_path / "div_magic"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2306_16274_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout
    assert int(out.stdout.split()[1]) > 4_000_000
