"""The size limits of the mixed form's exact tensor-core products (host
header paper_2011_02436_gb300/csrc/mixed_limits.h, compiled here as host
C++), against a derivation from the digit scheme in Python integers.

The mixed Gram (Eqs. 9-13) and the mixed hidden layer (Eq. 1) add, per
K chunk of 1024, the exact diagonal sums of digit products into one int64
per output element, diagonal t = p + q weighted 2^(7 (TMAX - t)).  Digits
are integers of magnitude at most 64.  The worst case, every digit of both
operands at 64 with one sign, gives each chunk its largest contribution;
the limits are the chunk counts whose sum of worst cases stays below 2^63."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_02436_gb300", "csrc")
CHUNK = 1024


def worst_chunk(P, tmax, bits=7):
    total = 0
    for t in range(2, tmax + 1):
        pairs = sum(1 for p in range(1, P + 1) if 1 <= t - p <= P)
        total += pairs * (2 ** (bits - 1)) ** 2 * CHUNK * 2 ** (bits * (tmax - t))
    return total


def max_chunks(P, tmax):
    return (2 ** 63 - 1) // worst_chunk(P, tmax)


def test_limits_follow_from_the_digit_scheme():
    assert max_chunks(5, 6) == 8064          # Gram: five digits, diagonals 2..6
    assert max_chunks(6, 7) == 63            # hidden layer: six digits, diagonals 2..7
    # one more chunk of worst-case digits would wrap the int64 sum
    assert worst_chunk(5, 6) * 8065 > 2 ** 63 - 1
    assert worst_chunk(6, 7) * 64 > 2 ** 63 - 1


PROG = r"""
#include <cstdio>
#include "elm.h"
#include "mixed_limits.h"
int main() {
    std::printf("%lld %lld\n", (long long)elm::MIXED_MAX_ROWS, (long long)elm::MIXED_MAX_INPUTS);
    const long long N[] = {1, 500000, 8257536, 8257537, 8257600, 8257601, 20000000};
    const long long n[] = {1, 784, 64512, 64513, 64544, 100000};
    for (long long a : N)
        for (long long b : n) std::printf("%lld %lld %d\n", a, b, elm::mixed_fits(a, b) ? 1 : 0);
    return 0;
}
"""


@pytest.fixture(scope="module")
def limits_program(tmp_path_factory):
    d = tmp_path_factory.mktemp("limits")
    src, exe = d / "limits.cpp", d / "limits"
    src.write_text(PROG)
    subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src)], check=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")


def test_header_limits_and_predicate(limits_program):
    rows, inputs = map(int, limits_program[0].split())
    assert rows == max_chunks(5, 6) * CHUNK and inputs == max_chunks(6, 7) * CHUNK
    for line in limits_program[1:]:
        if not line:
            continue
        N, n, fits = map(int, line.split())
        Np, nK = -(-N // 64) * 64, -(-n // 32) * 32      # the products' padded K
        assert fits == int(Np <= rows and nK <= inputs), line


def test_binding_exposes_the_same_limits(limits_program):
    import paper_2011_02436_gb300 as elm
    rows, inputs = map(int, limits_program[0].split())
    assert (elm.MIXED_MAX_ROWS, elm.MIXED_MAX_INPUTS) == (rows, inputs)
