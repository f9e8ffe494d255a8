"""The order in which the tensor kernel walks the Gram's lower triangle of
128 x 64 tiles (paper_2011_02436_gb300/csrc/oz_tiles.cuh, shared by host and
device code): every tile exactly once and inside the triangle for every
size up to 320 row blocks (the augmented Gram [H T] of the largest hidden
layer with thousands of targets), and a wave of 152 consecutive tiles
touches few operand row blocks (except in a last super-row of only one or
two row blocks, which the walk covers row after row).  Compiled as host C++."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_02436_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <set>
#include <vector>
#include "oz_tiles.cuh"
int main() {
    for (int64_t nJ = 1; nJ <= 320; nJ++) {          // L + m up to 40960 (128-row blocks)
        const int64_t n = nJ * (nJ + 1);
        std::vector<char> seen(n, 0);
        for (int64_t t = 0; t < n; t++) {
            int64_t J, cb;
            elm::gram_tile(t, nJ, J, cb);
            if (J < 0 || J >= nJ || cb < 0 || cb >= 2 * (J + 1)) { printf("outside %ld %ld\n", nJ, t); return 1; }
            const int64_t id = J * (J + 1) + cb;
            if (seen[id]) { printf("twice %ld %ld\n", nJ, t); return 1; }
            seen[id] = 1;
        }
    }
    int64_t worst = 0;
    for (int64_t nJ : {16, 63, 64}) {              // a last super-row of few rows excepted
        const int64_t n = nJ * (nJ + 1);
        for (int64_t w = 0; w * 152 < n; w++) {
            std::set<int64_t> blocks;                  // 128-row blocks of either operand
            for (int64_t t = w * 152; t < (w + 1) * 152 && t < n; t++) {
                int64_t J, cb;
                elm::gram_tile(t, nJ, J, cb);
                blocks.insert(J);
                blocks.insert(cb / 2);
            }
            if ((int64_t)blocks.size() > worst) worst = blocks.size();
        }
    }
    printf("%ld\n", worst);
    return 0;
}
"""


def test_every_tile_once_and_waves_stay_compact():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        with open(src, "w") as f:
            f.write(PROG)
        subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CSRC, src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout
        # row after row, a wave of a 63-row-block Gram touches 77 blocks
        assert int(out.stdout.strip()) <= 32
