"""The size limits of the exact tensor-core products (host header
paper_2011_02436_gb300/csrc/mixed_limits.h, compiled here as host C++),
against a derivation from the digit schemes in Python integers.

The mixed Gram (Eqs. 9-13), the mixed hidden layer (Eq. 1) and the two
bands of the FP64-accurate products add, per K chunk, the exact diagonal
sums of digit products into one int64 per output element, diagonal t = p + q
weighted 2^(7 (TMAX - t)).  Digits are integers of magnitude at most 64.
Bounding every digit of both operands by 64 bounds each chunk's
contribution; the limits are the chunk counts whose sum of these bounds
stays below 2^63.  A request beyond its form's limits
runs in the next form: mixed, then FP64-accurate tensor cores, then FP64."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_02436_gb300", "csrc")
CHUNK = 1024


def worst_chunk(P, tmax, tmin=2, chunk=CHUNK, bits=7):
    total = 0
    for t in range(tmin, tmax + 1):
        pairs = sum(1 for p in range(1, P + 1) if 1 <= t - p <= P)
        total += pairs * (2 ** (bits - 1)) ** 2 * chunk * 2 ** (bits * (tmax - t))
    return total


def max_chunks(P, tmax, tmin=2, chunk=CHUNK):
    return (2 ** 63 - 1) // worst_chunk(P, tmax, tmin, chunk)


def exact_limit():
    # FP64-accurate products: diagonals 2..5 of four planes in chunks of
    # 1024, diagonals 6..9 of eight planes in chunks of 512
    return min(max_chunks(4, 5, 2, 1024) * 1024, max_chunks(8, 9, 6, 512) * 512)


def test_limits_follow_from_the_digit_scheme():
    assert max_chunks(5, 6) == 8064          # Gram: five digits, diagonals 2..6
    assert max_chunks(6, 7) == 63            # hidden layer: six digits, diagonals 2..7
    # one more chunk would exceed the bound
    assert worst_chunk(5, 6) * 8065 > 2 ** 63 - 1
    assert worst_chunk(6, 7) * 64 > 2 ** 63 - 1
    assert max_chunks(8, 9, 6, 512) == 415499 and exact_limit() == 415499 * 512
    assert worst_chunk(8, 9, 6, 512) * 415500 > 2 ** 63 - 1


PROG = r"""
#include <cstdio>
#include "elm.h"
#include "mixed_limits.h"
int main() {
    std::printf("%lld %lld %lld\n", (long long)elm::MIXED_MAX_ROWS,
                (long long)elm::MIXED_MAX_INPUTS, (long long)elm::EXACT_MAX_K);
    const long long N[] = {1, 500000, 8257536, 8257537, 8257600, 8257601, 20000000,
                           212735488, 212735489, 300000000};
    const long long n[] = {1, 784, 64512, 64513, 64544, 100000, 212735488, 212735489};
    for (long long a : N)
        for (long long b : n)
            for (int p = 0; p < 3; p++)
                std::printf("%lld %lld %d %d %d\n", a, b, p, elm::route_precision(p, a, b),
                            elm::mixed_fits(a, b) ? 1 : 0);
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


def test_header_limits_and_routing(limits_program):
    rows, inputs, exact = map(int, limits_program[0].split())
    assert rows == max_chunks(5, 6) * CHUNK and inputs == max_chunks(6, 7) * CHUNK
    assert exact == exact_limit()
    seen = set()
    for line in limits_program[1:]:
        if not line:
            continue
        N, n, asked, runs, fits = map(int, line.split())
        Np, nK = -(-N // 64) * 64, -(-n // 32) * 32      # the products' padded K
        mixed_ok = Np <= rows and nK <= inputs
        exact_ok = Np <= exact and nK <= exact
        assert fits == int(mixed_ok), line
        want = asked
        if want == 1 and not mixed_ok:
            want = 2
        if want == 2 and not exact_ok:
            want = 0
        assert runs == want, line
        seen.add((asked, runs))
    assert seen == {(0, 0), (1, 1), (1, 2), (1, 0), (2, 2), (2, 0)}


def test_binding_and_header_expose_the_same_limits(limits_program):
    import paper_2011_02436_gb300 as elm
    rows, inputs, exact = map(int, limits_program[0].split())
    assert (elm.MIXED_MAX_ROWS, elm.MIXED_MAX_INPUTS, elm.EXACT_MAX_K) == (rows, inputs, exact)
    hdr = open(os.path.join(ROOT, "include", "elm.h")).read()
    for name, v in (("ELM_MIXED_MAX_ROWS", rows), ("ELM_MIXED_MAX_INPUTS", inputs),
                    ("ELM_EXACT_MAX_K", exact)):
        assert int(re.search(r"#define %s (\d+)" % name, hdr).group(1)) == v
