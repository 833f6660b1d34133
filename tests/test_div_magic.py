"""The divide-free quotient the bulk tile uses for quad -> row -> (y, z)
(magic_div / div_magic in lbsph_internal.cuh), checked on the host against
integer division: exhaustively for small divisors, and at every kind of
boundary (multiples of d, their neighbours, the top of the range) plus random
numerators for every divisor a box can give (nx/4 and ny up to 8192)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2403_05443_gb300", "csrc")

PROG = r"""
#include "lbsph_internal.cuh"
#include <cstdio>
using namespace lbsph;
static unsigned long long st = 88172645463325252ull;
static unsigned rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (unsigned)(st >> 33); }
static int bad = 0;
static void check(int n, unsigned d, unsigned m, int s) {
    if (div_magic(n, m, s) != (int)((unsigned)n / d)) {
        if (bad < 5) printf("d=%u n=%d got %d\n", d, n, div_magic(n, m, s));
        ++bad;
    }
}
int main() {
    for (unsigned d = 1; d <= 64; ++d) {
        unsigned m; int s; magic_div(d, m, s);
        for (int n = 0; n < (1 << 22); ++n) check(n, d, m, s);
    }
    for (unsigned d = 1; d <= 8192; ++d) {
        unsigned m; int s; magic_div(d, m, s);
        const long long top = 2147483647ll;
        for (long long k = 0; k <= 2000; ++k) {
            const long long a = k * d, b = top / d * d - k * d;
            for (long long n : {a - 1, a, a + 1, b - 1, b, b + 1})
                if (n >= 0 && n <= top) check((int)n, d, m, s);
        }
        for (int r = 0; r < 2000; ++r) check((int)(rnd() & 0x7fffffffu), d, m, s);
        check(2147483647, d, m, s);
    }
    printf("%s %d\n", bad ? "FAIL" : "OK", bad);
    return bad != 0;
}
"""


def test_magic_division_matches_integer_division():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "div.cu")
        exe = os.path.join(d, "div")
        with open(src, "w") as f:
            f.write(PROG)
        r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", SRC, src, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        print(r.stdout)
        assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout
