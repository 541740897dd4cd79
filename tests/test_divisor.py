"""Host check of the lattice kernels' division by an invariant divisor
(make_divisor / divide in csrc/lbp_internal.cuh: one 32x32->64-bit multiply
and a shift, exact for dividends below 2^31 by Granlund and Montgomery's
bound): the header itself, compiled for the host by nvcc, against the
integer quotient for every divisor up to 70000 (the rows and row segments of
any box the library accepts) and for divisors up to 2^31 - 1, at the
dividends where a rounding error would first show."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1909_13412_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "lbp_internal.cuh"
using lbp::Divisor;
using lbp::divide;
using lbp::make_divisor;

static unsigned long long state = 0x9e3779b97f4a7c15ull;
static unsigned next31() {  // splitmix64, top 31 bits
    unsigned long long z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (unsigned)((z ^ (z >> 31)) >> 33);
}

static int check(unsigned d, unsigned n, const Divisor &dv) {
    if (divide(n, dv) != n / d) {
        std::printf("FAIL d=%u n=%u got %u want %u\n", d, n, divide(n, dv), n / d);
        return 1;
    }
    return 0;
}

static int check_divisor(unsigned d) {
    const Divisor dv = make_divisor(d);
    const unsigned top = 0x7fffffffu;
    int bad = 0;
    // around multiples of d near 0, near the top of the range, and at random
    const unsigned lastq = top / d;
    for (unsigned q : {0u, 1u, 2u, 3u, lastq - 1, lastq})
        for (long long o = -2; o <= 2; ++o) {
            const long long n = (long long)q * d + o;
            if (n >= 0 && n <= top) bad |= check(d, (unsigned)n, dv);
        }
    for (int k = 0; k < 64; ++k) bad |= check(d, next31(), dv);
    bad |= check(d, top, dv);
    return bad;
}

int main() {
    int bad = 0;
    for (unsigned d = 1; d <= 70000 && !bad; ++d) bad |= check_divisor(d);
    for (int k = 0; k < 200000 && !bad; ++k) bad |= check_divisor(1u + next31() % 0x7fffffffu);
    for (unsigned l = 0; l < 31 && !bad; ++l)
        for (unsigned d : {(1u << l) - 1, 1u << l, (1u << l) + 1})
            if (d >= 1 && d <= 0x7fffffffu) bad |= check_divisor(d);
    if (!bad) std::printf("ok\n");
    return bad;
}
"""


def test_division_by_an_invariant_divisor_is_exact(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to compile the header")
    src = tmp_path / "divisor_check.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "divisor_check"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-2000:]
