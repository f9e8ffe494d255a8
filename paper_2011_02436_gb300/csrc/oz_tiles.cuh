// Order of the output tiles of a symmetric product (the Gram): the lower
// triangle of 128-row x 64-column tiles, row block J holding column blocks
// 0 .. 2J+1.  A persistent grid runs tiles t, t + G, ... per CTA, so the
// tiles of one wave are G consecutive indices; the order below keeps a wave
// inside a few super-blocks of GT_SJ row blocks x GT_SC column blocks (1024 x
// 1024 elements), so the wave's operand rows are few and shared through L2.
// (Row after row, a late wave of a large Gram covers one row block but about
// a hundred and fifty column blocks, none of them shared.)
// Super-row R, then its super-blocks C = 0 .. R (the diagonal one last),
// row-major inside each.  Host and device code share this mapping.
#pragma once
#include <math.h>
#include <stdint.h>

#ifndef __CUDACC__
#define OZ_HD
#else
#define OZ_HD __host__ __device__
#endif

namespace elm {

constexpr int64_t GT_SJ = 8, GT_SC = 16;   // 2 GT_SJ == GT_SC: square super-blocks

// tiles before super-row R when all super-rows before it are full
OZ_HD inline int64_t gram_tiles_before(int64_t R) {
    return (GT_SJ * GT_SC / 2) * R * (R - 1) + GT_SJ * (GT_SJ + 1) * R;
}

// Tile t (0 <= t < nJ (nJ + 1)) -> row block J and column block cb.
OZ_HD inline void gram_tile(int64_t t, int64_t nJ, int64_t &J, int64_t &cb) {
    // gram_tiles_before(R) = 64 R^2 + 8 R: a float estimate, then exact fixes
    int64_t R = (int64_t)((sqrt(64.0 + 256.0 * (double)t) - 8.0) / 128.0);
    if (R < 0) R = 0;
    while (R > 0 && gram_tiles_before(R) > t) R--;
    while (gram_tiles_before(R + 1) <= t) R++;
    const int64_t h = nJ - GT_SJ * R < GT_SJ ? nJ - GT_SJ * R : GT_SJ;   // rows of super-row R
    const int64_t u = t - gram_tiles_before(R);
    const int64_t off = R * GT_SC * h;   // tiles of its off-diagonal super-blocks
    if (u < off) {
        const int64_t C = u / (GT_SC * h), r = u - C * GT_SC * h;
        J = GT_SJ * R + r / GT_SC;
        cb = GT_SC * C + r % GT_SC;
    } else {
        // the diagonal super-block: its row j holds 2 (j + 1) tiles
        const int64_t v = u - off;
        int64_t j = (int64_t)((sqrt(4.0 * (double)v + 1.0) - 1.0) * 0.5);
        if (j < 0) j = 0;
        while (j > 0 && j * (j + 1) > v) j--;
        while ((j + 1) * (j + 2) <= v) j++;
        J = GT_SJ * R + j;
        cb = GT_SC * R + (v - j * (j + 1));
    }
}

}  // namespace elm
