// Largest problems whose tensor-core products stay exact (host code; no
// CUDA dependencies: the public header only).
//
// The tensor kernels add each K chunk's exact diagonal sums of digit
// products into one int64 running sum per output element, diagonal t = p + q
// weighted 2^(7 (TMAX - t)).  A digit is an integer of magnitude at most 64
// and diagonal t pairs min(t - 1, 2 P + 1 - t) of the P digits per operand,
// so one chunk adds at most
//     C = sum_{t = TMIN}^{TMAX} pairs(t) 2^12 chunk 2^(7 (TMAX - t))
// in magnitude, whatever the data:
//   * mixed Gram (Eqs. 9-13; P = 5, t = 2..6, chunks of 1024): about 2^50.02,
//     so 8064 chunks of samples (8 257 536 samples);
//   * mixed hidden layer (Eq. 1; P = 6, t = 2..7, chunks of 1024): about
//     2^57.02, so 63 chunks of inputs (64 512 inputs);
//   * FP64-accurate products (P = 8): the band t = 2..5 (four planes, chunks
//     of 1024) about 2^43.02, the band t = 6..9 (chunks of 512) about 2^44.34,
//     so 415 499 chunks of 512 (212 735 488 samples or inputs).
// A mixed request beyond its limits runs the FP64-accurate tensor-core form,
// and one beyond that form's limit the FP64 form.
#pragma once
#include <stdint.h>

#include "elm.h"

namespace elm {

constexpr int64_t MIXED_CHUNK = 1024;                   // K elements per exact chunk
constexpr int64_t MIXED_MAX_ROWS = 8064 * MIXED_CHUNK;  // samples N, padded to 64
constexpr int64_t MIXED_MAX_INPUTS = 63 * MIXED_CHUNK;  // inputs n, padded to 32
constexpr int64_t EXACT_MAX_K = 415499 * 512;           // FP64-accurate products: N and n
static_assert(ELM_MIXED_MAX_ROWS == MIXED_MAX_ROWS && ELM_MIXED_MAX_INPUTS == MIXED_MAX_INPUTS &&
                  ELM_EXACT_MAX_K == EXACT_MAX_K,
              "the public limits match");

// Largest magnitude one chunk adds to a running sum: P digits of `bits` bits
// per operand, diagonals tmin..tmax, `chunk` products per digit pair.  The
// result is an integer with at most 36 significant bits times a power of
// two, exact in double, and so are its products with the chunk counts.
constexpr double chunk_bound(int P, int tmin, int tmax, int bits, int64_t chunk) {
    double c = 0.0;
    for (int t = tmin; t <= tmax; t++) {
        const int pairs = t - 1 < 2 * P + 1 - t ? t - 1 : 2 * P + 1 - t;
        double w = 1.0;
        for (int i = 0; i < bits * (tmax - t); i++) w *= 2.0;
        const double dmax = (double)(1 << (bits - 1));
        c += (double)pairs * dmax * dmax * (double)chunk * w;
    }
    return c;
}
constexpr double TWO_POW_63 = 9223372036854775808.0;
constexpr bool sums_fit(double per_chunk, int64_t K, int64_t chunk) {
    return per_chunk * (double)((K + chunk - 1) / chunk) < TWO_POW_63;
}
static_assert(sums_fit(chunk_bound(5, 2, 6, 7, 1024), MIXED_MAX_ROWS, 1024), "mixed Gram");
static_assert(sums_fit(chunk_bound(6, 2, 7, 7, 1024), MIXED_MAX_INPUTS, 1024), "mixed hidden");
static_assert(sums_fit(chunk_bound(4, 2, 5, 7, 1024), EXACT_MAX_K, 1024), "exact band 2..5");
static_assert(sums_fit(chunk_bound(8, 6, 9, 7, 512), EXACT_MAX_K, 512), "exact band 6..9");

// True when N samples and n inputs fit the mixed form's exact products.
inline bool mixed_fits(int64_t N, int64_t n) {
    return (N + 63) / 64 * 64 <= MIXED_MAX_ROWS && (n + 31) / 32 * 32 <= MIXED_MAX_INPUTS;
}
// The same for the FP64-accurate tensor-core products.
inline bool exact_fits(int64_t N, int64_t n) {
    return (N + 63) / 64 * 64 <= EXACT_MAX_K && (n + 31) / 32 * 32 <= EXACT_MAX_K;
}
// The form (ELM_PREC_*) a request for `precision` runs in for N samples and
// n inputs.
inline int route_precision(int precision, int64_t N, int64_t n) {
    if (precision == ELM_PREC_MIXED && !mixed_fits(N, n)) precision = ELM_PREC_FP64_TC;
    if (precision == ELM_PREC_FP64_TC && !exact_fits(N, n)) precision = ELM_PREC_FP64;
    return precision;
}

}  // namespace elm
