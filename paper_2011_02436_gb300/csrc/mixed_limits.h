// Largest problems whose mixed-form tensor-core products stay exact (host
// code; no CUDA dependencies).
//
// The mixed Gram (Eqs. 9-13: five 7-bit digits per operand, kept diagonals
// t = 2..6, chunks of 1024 samples) and the mixed hidden layer's
// pre-activation (Eq. 1: six digits, t = 2..7, chunks of 1024 inputs) add
// each chunk's exact diagonal sums into one int64 running sum per output
// element, diagonal t weighted 2^(7 (TMAX - t)).  A digit is an integer of
// magnitude at most 64 and diagonal t pairs min(t - 1, 2 P + 1 - t) digits,
// so one chunk adds at most
//     C = sum_t pairs(t) 2^12 1024 2^(7 (TMAX - t))
// in magnitude: about 2^50.02 for the Gram and 2^57.02 for the hidden
// layer.  The running sums therefore stay below 2^63 for up to 8064 chunks
// of samples (8 257 536 samples) and 63 chunks of inputs (64 512 inputs),
// whatever the data.  A larger problem trains in the FP64 form with
// tensor-core products instead, whose digit bands weigh at most 2^21 per
// unit.
#pragma once
#include <stdint.h>

namespace elm {

constexpr int64_t MIXED_CHUNK = 1024;                   // K elements per exact chunk
constexpr int64_t MIXED_MAX_ROWS = 8064 * MIXED_CHUNK;  // samples N, padded to 64
constexpr int64_t MIXED_MAX_INPUTS = 63 * MIXED_CHUNK;  // inputs n, padded to 32
#ifdef ELM_MIXED_MAX_ROWS
static_assert(ELM_MIXED_MAX_ROWS == MIXED_MAX_ROWS && ELM_MIXED_MAX_INPUTS == MIXED_MAX_INPUTS,
              "the public limits match");
#endif

// Largest magnitude one chunk adds to a running sum: P digits of `bits` bits
// per operand, diagonals 2..tmax, `chunk` products per diagonal pair.  Exact
// in double for the sizes used (below 2^58, integer).
constexpr double mixed_chunk_bound(int P, int tmax, int bits, int64_t chunk) {
    double c = 0.0;
    for (int t = 2; t <= tmax; t++) {
        const int pairs = t - 1 < 2 * P + 1 - t ? t - 1 : 2 * P + 1 - t;
        double w = 1.0;
        for (int i = 0; i < bits * (tmax - t); i++) w *= 2.0;
        const double dmax = (double)(1 << (bits - 1));
        c += (double)pairs * dmax * dmax * (double)chunk * w;
    }
    return c;
}

constexpr double TWO_POW_63 = 9223372036854775808.0;
static_assert(mixed_chunk_bound(5, 6, 7, MIXED_CHUNK) * (double)(MIXED_MAX_ROWS / MIXED_CHUNK) <
                  TWO_POW_63,
              "mixed Gram running sums exceed int64");
static_assert(mixed_chunk_bound(6, 7, 7, MIXED_CHUNK) * (double)(MIXED_MAX_INPUTS / MIXED_CHUNK) <
                  TWO_POW_63,
              "mixed hidden-layer running sums exceed int64");

// True when N samples and n inputs fit the mixed form's exact products.
inline bool mixed_fits(int64_t N, int64_t n) {
    return (N + 63) / 64 * 64 <= MIXED_MAX_ROWS && (n + 31) / 32 * 32 <= MIXED_MAX_INPUTS;
}

}  // namespace elm
