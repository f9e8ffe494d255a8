// Trailing update of the pivoted factorisation on the tensor cores (Eq. 6;
// Algorithm 1, steps 3-4).  After a panel of up to 32 pivots every
// remaining entry of the active matrix becomes
//     A'[x, y] = A[rem x, rem y] - sum_t P[t, rem x] P[t, rem y],
// with rem the compaction map of the unpivoted columns.  Two schemes: the
// mixed form holds A and the panel rows P as double-float pairs (h + l, two
// floats in eight bytes), the FP64 form with tensor-core products as FP64.
//
// Digits.  The 32 panel entries of each remaining column x are scaled by a
// power of two s_x and split into signed 8-bit digits, integers |a_j| <= 128
// (exact in bf16), digit j of weight 2^(-7-8j): six digits of a
// double-float entry (|r| <= 2^-48 s_x), or seven of an FP64 entry taken
// from rint(v / s_x 2^55) by integer operations (|r| <= 2^-56 s_x).
// Products.  For a digit pair (i, j) one tcgen05 MMA (kind::f16, bf16
// operands, FP32 accumulator in tensor memory) sums the 32 products
// |a_i b_j| <= 2^14 of a pair: at most 2^19 per pair, and at most seven
// pairs share the weight 2^(-14-8d) of diagonal d = i + j, so every
// accumulator stays an integer below 2^22 and the FP32 accumulation is
// exact in any order.  Kept: pairs with i + j <= NDIG (26 of 36 pairs in
// seven diagonals; 34 of 49 in eight); the others weigh below 2^-48
// (2^-56) of s_x s_y.  The drain folds the exact diagonal sums and
// subtracts them, scaled by s_x s_y, from A's entry: in double-float
// (TwoSum on the FP32 pipes, about 2^-46 relative to s_x s_y, like the
// double-float update, in about 45 FP32 instructions per entry instead of 32
// products of 10), or exactly into two 47-bit integers and then two FP64
// FMAs (FP64 accuracy, two FP64 instructions per entry instead of 32).
// Symmetry.  The integer sums are symmetric in (x, y) and the scales are per
// column, so bitwise-equal columns stay bitwise equal (ties in the pivot
// search resolve as before) and A' is exactly symmetric; each lower tile
// also writes its mirror.
//
// Layout of the digit planes: G[c][p][32] bf16, p < Lcap (compacted column
// index, Lcap a multiple of 128), K = 32 panel rows (zero past the panel's
// pivots).  Plane c = NDIG - j holds digit j (c = 1..NDIG); plane 0 is all
// zeros and stands for an extra digit of the B operand, so that for every A
// digit i the pairs (i, NDIG-i..0) form one MMA over B planes i..NDIG whose
// diagonal d lands at tensor-memory column (NDIG - d) 32, with every MMA
// starting at column 0.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "df_arith.cuh"
#include "elm_internal.cuh"
#include "tc_ptx.cuh"

namespace elm {

namespace {

using df::F2;
using df::d2df;
using df::df_acc_prod;
using df::df_renorm;
using df::f2d;
using namespace tcx;

static_assert(TRAIL_TC_K == 32, "one 64-byte K row of bf16 digits per plane");
constexpr int TR = 128;                    // tile rows (TMEM lanes)
constexpr int TC = 32;                     // tile columns
constexpr uint32_t A_PLANE = TR * 64;      // bytes of one A plane (128 rows x 32 bf16)
constexpr uint32_t B_PLANE = TC * 64;      // bytes of one B plane
constexpr uint32_t TMEM_COLS = 256;        // NDIAG x 32 (224 or 256) used
// The two digit schemes: double-float entries (the mixed form) in six
// digits, FP64 entries (the FP64 form with tensor-core products) in seven;
// the kept diagonals are d = 0 .. NDIG and plane 0 of B is the zero plane.
template <bool F64>
struct Scheme {
    static constexpr int NDIG = F64 ? 7 : 6;
    static constexpr int NDIAG = NDIG + 1;
    static constexpr int NPLANE = NDIG + 1;
    static constexpr uint32_t A_BYTES = NDIG * A_PLANE;
    static constexpr uint32_t B_BYTES = NPLANE * B_PLANE;
};
using SDF = Scheme<false>;
using S64 = Scheme<true>;
// the mixed form's scheme (the K solve uses it)
constexpr int NDIG = SDF::NDIG;
constexpr int NDIAG = SDF::NDIAG;
constexpr int NPLANE = SDF::NPLANE;
constexpr uint32_t A_BYTES = SDF::A_BYTES;
constexpr uint32_t B_BYTES = SDF::B_BYTES;
constexpr int MAX_PLANES = S64::NPLANE;    // planes of the shared digit buffer
constexpr int TTHREADS = 256;              // two warps per TMEM lane quarter
// Dynamic shared memory: the operands (62 KB) and, once the MMAs are done,
// the transposed output tile.  Asking for 100 KB keeps at most two CTAs on
// an SM, whose tensor memory holds two allocations of 256 columns.
constexpr size_t TRAIL_SMEM = 100 * 1024;
constexpr uint64_t TRAIL_WAIT_NS = 2000000000ull;
// kind::f16, bf16 x bf16 -> f32, K-major operands, M = 128 (N set per MMA)
constexpr uint32_t IDESC_M128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TR >> 4) << 24);
static_assert(S64::NDIAG * TC <= (int)TMEM_COLS, "diagonals exceed the allocation");
static_assert(S64::NPLANE * TC <= 256, "widest MMA above N = 256");
static_assert(S64::A_BYTES + S64::B_BYTES + 1024 <= TRAIL_SMEM, "operands exceed shared memory");
static_assert((size_t)TR * (TC + 1) * 8 + 1024 <= TRAIL_SMEM, "output tile exceeds shared memory");
// the K solve's staged tile of B sits after the operands
constexpr size_t KS_STAGE_OFF = 64 * 1024;
static_assert(A_BYTES + B_BYTES <= KS_STAGE_OFF, "operands overlap the staged tile");
static_assert(KS_STAGE_OFF + (size_t)TR * (TC + 1) * 8 + 1024 <= TRAIL_SMEM,
              "staged tile exceeds shared memory");

__device__ __forceinline__ float rint_small(float x) {   // |x| < 2^22: nearest integer
    return __fadd_rn(__fadd_rn(x, 12582912.f), -12582912.f);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Digits of one K row of 32 values, one per lane of a warp (zero where the
// row is shorter): the smallest power of two s >= the largest |h| (1 for a
// zero row; a denormal maximum rounds up to 2^-126), then six signed 8-bit
// digits of v / s, digit j of weight 2^(-7-8j), into planes 6 - j of g
// (plane stride pstride elements; plane 0 zero).  *sc = s (lane 0).
__device__ __forceinline__ void warp_digits(F2 v, __nv_bfloat16 *g, int64_t pstride, float *sc) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(v.h)));
    uint32_t sb = (m + 0x7fffffu) & 0xff800000u;
    if (sb == 0u) sb = 0x3f800000u;
    const float inv = __uint_as_float((254u << 23) - sb);   // 1 / s, exact
    // x = v / s, |x| <= 1 + 2^-24
    float rh = v.h * inv * 128.f, rl = v.l * inv * 128.f;
    g[0] = __float2bfloat16_rn(0.f);   // the zero plane
#pragma unroll
    for (int j = 0; j < NDIG; j++) {
        const float a = rint_small(rh);   // |rh| <= 128 + 2^-9, so |a| <= 128
        float e;
        two_sum(rh - a, rl, rh, e);        // rh - a is exact, |.| <= 1/2
        rl = e;
        rh *= 256.f;
        rl *= 256.f;
        g[(int64_t)(NDIG - j) * pstride] = __float2bfloat16_rn(a);   // exact: |a| <= 128
    }
    if ((threadIdx.x & 31) == 0) *sc = __uint_as_float(sb);
}

// The same for FP64 values in seven digits: s = 2^(E+1) for the largest
// exponent E of the row (at least 2^-126, 1 for a zero row), |v| / s < 1;
// X = rint(v / s 2^55) (|X| < 2^55, the part below 2^-56 s dropped) split
// into balanced base-256 digits from the least significant one with
// integer operations (digit 0 the rest, |digit| <= 128).
__device__ __forceinline__ void warp_digits64(double v, __nv_bfloat16 *g, int64_t pstride,
                                              float *sc) {
    const uint32_t hw = (uint32_t)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
    const uint32_t m = __reduce_max_sync(0xffffffffu, hw);
    int e = (int)(m >> 20) - 1023 + 1;   // exponent of s
    if (m == 0u) e = 0;
    e = e < -126 ? -126 : (e > 127 ? 127 : e);   // a float scale
    const double inv = __longlong_as_double((long long)(1023 - e) << 52);   // 2^-e
    long long X = __double2ll_rn(v * inv * 0x1p55);
    float d[S64::NDIG];
#pragma unroll
    for (int j = S64::NDIG - 1; j >= 1; j--) {
        const long long r = ((X + 128) & 255) - 128;
        d[j] = (float)(int)r;
        X = (X - r) >> 8;
    }
    d[0] = (float)(int)X;
    g[0] = __float2bfloat16_rn(0.f);   // the zero plane
#pragma unroll
    for (int j = 0; j < S64::NDIG; j++)
        g[(int64_t)(S64::NDIG - j) * pstride] = __float2bfloat16_rn(d[j]);   // exact
    if ((threadIdx.x & 31) == 0) *sc = __uint_as_float((uint32_t)(e + 127) << 23);
}

// One warp per compacted column p < rows: scale and digits of its panel
// entries P[t, rem p], t < steps (zero beyond, and for p >= Ln).
template <bool F64>
__global__ void __launch_bounds__(256)
trail_digits_kernel(const double *__restrict__ P, int64_t ldp, const int32_t *__restrict__ rem,
                    const FactorState *__restrict__ st, __nv_bfloat16 *__restrict__ G,
                    float *__restrict__ gs, int64_t Lcap, int64_t rows) {
    const FactorState s = *st;
    if (s.done) return;
    const int64_t Ln = s.Lr;
    const int steps = (int)s.steps;
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= rows) return;
    const bool in = p < Ln && lane < steps;
    const int64_t i = in ? (int64_t)lane * ldp + rem[p] : 0;
    if constexpr (F64) {
        warp_digits64(in ? P[i] : 0.0, G + p * 32 + lane, Lcap * 32, gs + p);
    } else {
        warp_digits(in ? reinterpret_cast<const F2 *>(P)[i] : F2{0.f, 0.f}, G + p * 32 + lane,
                    Lcap * 32, gs + p);
    }
}

// Shared memory and tensor memory of one 128 x 32 output tile, and the
// steps every tile kernel takes: set-up (barriers, tensor memory), the TMA
// copies of both operands' digit planes with the MMAs (two per A digit,
// thread 0), the wait for them (all threads), the fold of the diagonal sums,
// and the tear-down.
struct TileSmem {
    uint64_t full_bar, mma_bar;
    uint32_t tmem;
    int abort;
};
__device__ __forceinline__ void tile_setup(TileSmem &t) {
    if (threadIdx.x == 0) {
        mbar_init(&t.full_bar, 1);
        mbar_init(&t.mma_bar, 1);
        t.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&t.tmem)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
// thread 0: A digits 5..0 of rows a_row.. (planes 1..6 of tmA), B digits
// "6", 5..0 of rows b_row.. (planes 0..6 of tmB)
template <class S = SDF>
__device__ __forceinline__ void tile_load(TileSmem &t, const CUtensorMap *tmA, const CUtensorMap *tmB,
                                          uint8_t *sA, uint8_t *sB, int a_row, int b_row) {
    mbar_expect_tx(&t.full_bar, S::A_BYTES + S::B_BYTES);
    tma_3d(tmA, &t.full_bar, sA, 0, a_row, 1);
    tma_3d(tmB, &t.full_bar, sB, 0, b_row, 0);
}
// thread 0, after tile_load: A digit i (smem plane 5 - i) against B planes
// i..6 (digits 6 - i .. 0), diagonal d = i + (6 - c) at column (6 - d) 32;
// i = 0 reaches every column and comes first.
template <class S = SDF>
__device__ __forceinline__ void tile_mma(TileSmem &t, uint8_t *sA, uint8_t *sB) {
    volatile int *abort = &t.abort;
    if (mbar_wait(&t.full_bar, 0, abort, TRAIL_WAIT_NS)) {
        tc_fence_after();
        const uint64_t da0 = desc_sw64(su32(sA)), db0 = desc_sw64(su32(sB));
#pragma unroll
        for (int i = 0; i < S::NDIG; i++) {
            const uint64_t da = da0 + (uint64_t)(((S::NDIG - 1 - i) * A_PLANE) >> 4);
            const uint64_t db = db0 + (uint64_t)((i * B_PLANE) >> 4);
            const uint32_t idesc = IDESC_M128 | ((uint32_t)(((S::NPLANE - i) * TC) >> 3) << 17);
#pragma unroll
            for (int kk = 0; kk < 2; kk++)   // K = 32: two steps of 16
                mma_bf16(t.tmem, da + 2 * kk, db + 2 * kk, idesc, (i == 0 && kk == 0) ? 0u : 1u);
        }
    }
    mma_commit(&t.mma_bar);   // arrives once every MMA issued above has completed
}
__device__ __forceinline__ bool tile_wait(TileSmem &t) {
    volatile int *abort = &t.abort;
    const bool ok = mbar_wait(&t.mma_bar, 0, abort, TRAIL_WAIT_NS) && !*abort;
    tc_fence_after();
    return ok;
}
// the 8 x NDIAG accumulators of columns col.. of this thread's TMEM lane
template <int ND>
__device__ __forceinline__ void tile_ld8(const TileSmem &t, int quarter, int col,
                                         uint32_t (&dg)[ND][8]) {
    const uint32_t tl = t.tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
    for (int d = 0; d < ND; d++) tmem_ld8(tl + (uint32_t)((ND - 1 - d) * TC + col), dg[d]);
    tmem_wait_ld();
#pragma unroll
    for (int d = 0; d < ND; d++) reg_fence8(dg[d]);
}
// a - c sum_d D_d 2^(-14-8d) in double-float: the two leading pairs exactly
// by TwoSum, the three smallest terms (below 2^-24) in FP32; c = s_x s_y
__device__ __forceinline__ F2 fold_sub(const uint32_t (&dg)[NDIAG][8], int k8, float c, F2 a) {
    float h1, l1, h2, l2, h, e;
    two_sum(__uint_as_float(dg[0][k8]) * 0x1p-14f, __uint_as_float(dg[1][k8]) * 0x1p-22f, h1, l1);
    two_sum(__uint_as_float(dg[2][k8]) * 0x1p-30f, __uint_as_float(dg[3][k8]) * 0x1p-38f, h2, l2);
    const float tail = __uint_as_float(dg[4][k8]) * 0x1p-46f +
                       (__uint_as_float(dg[5][k8]) * 0x1p-54f + __uint_as_float(dg[6][k8]) * 0x1p-62f);
    two_sum(h1, h2, h, e);
    const float l = (((l1 + l2) + e) + tail) * c;
    h *= c;
    float sh, se;
    two_sum(a.h, -h, sh, se);
    se += a.l - l;
    const float rh = sh + se;
    return F2{rh, se - (rh - sh)};
}
// exact value of an integer |v| < 2^53 as a double, by integer operations
__device__ __forceinline__ double i2d_exact(long long v) {
    if (v == 0) return 0.0;
    const unsigned long long sg = v < 0 ? 1ull << 63 : 0ull;
    const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    const int lz = __clzll((long long)a);
    const unsigned long long mant = lz == 63 ? 0ull : (a << (lz + 1)) >> 12;   // below the leading one
    return __longlong_as_double((long long)(sg | ((unsigned long long)(1023 + 63 - lz) << 52) | mant));
}
// a - c sum_d D_d 2^(-14-8d), d = 0..7, in FP64: the diagonals as integers
// (exact, |D_d| < 2^22), folded exactly into two 47-bit integers, then one
// FMA for their sum and one for the subtraction (c = s_x s_y exact): two
// FP64 instructions per entry
__device__ __forceinline__ double fold_sub64(const uint32_t (&dg)[S64::NDIAG][8], int k8, float c,
                                             double a) {
    long long hi = 0, lo = 0;
#pragma unroll
    for (int d = 0; d < 4; d++) {
        const int v = __float_as_int(__uint_as_float(dg[d][k8]) + 12582912.f) - 0x4B400000;
        hi = hi * 256 + v;
    }
#pragma unroll
    for (int d = 4; d < 8; d++) {
        const int v = __float_as_int(__uint_as_float(dg[d][k8]) + 12582912.f) - 0x4B400000;
        lo = lo * 256 + v;
    }
    // hi + lo 2^-32 rounded once; the 2^-38 joins the scale c (a power of two,
    // exact in both formats) through its exponent bits
    const double t = fma(i2d_exact(lo), 0x1p-32, i2d_exact(hi));
    const double cd = f2d(c);
    const double c38 = cd == 0.0 ? 0.0 : __longlong_as_double(__double_as_longlong(cd) - (38ll << 52));
    return fma(-t, c38, a);
}
__device__ __forceinline__ void tile_teardown(TileSmem &t, FactorState *st, int *flag) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem),
                     "r"(TMEM_COLS));
    }
    if (threadIdx.x == 0 && t.abort) {
        // let the copies land before the CTA's shared memory is released
        const uint64_t t0 = gtime();
        while (!mbar_try(&t.full_bar, 0) && gtime() - t0 < TRAIL_WAIT_NS) {
        }
        if (st) atomicOr(&st->flags, 2);
        if (flag) atomicOr(flag, 1);
    }
}

// Lower tiles of 128 rows x 32 columns: row block rb holds column blocks
// 0 .. 4 rb + 3.  Warp 0 allocates tensor memory; thread 0 issues the two
// TMA copies (all A planes of the tile's rows, all B planes of its columns)
// and the MMAs; all eight warps prefetch their entries of A, then drain
// (warp w: TMEM lanes 32 (w mod 4) .., columns 16 (w / 4) ..).  F64: the
// active matrix holds FP64 values and the seven-digit scheme applies;
// else double-float pairs and six digits.
template <bool F64>
__global__ void __launch_bounds__(TTHREADS, 2)
trailing_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const double *__restrict__ A, double *__restrict__ An, int64_t lda,
                   const int32_t *__restrict__ rem, const float *__restrict__ gs,
                   FactorState *st) {
    using S = Scheme<F64>;
    using V = typename std::conditional<F64, double, F2>::type;
    const V *Av = reinterpret_cast<const V *>(A);
    V *Anv = reinterpret_cast<V *>(An);
    const FactorState s = *st;
    if (s.done) return;
    const int64_t Ln = s.Lr;
    const int64_t b = blockIdx.x;
    int64_t rb = (int64_t)((sqrtf(2.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while (rb > 0 && 2 * rb * (rb + 1) > b) rb--;
    while (2 * (rb + 1) * (rb + 2) <= b) rb++;
    const int64_t cb = b - 2 * rb * (rb + 1);
    const int64_t r0 = rb * TR, c0 = cb * TC;
    if (r0 >= Ln || c0 >= Ln) return;   // uniform over the CTA

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm, *sB = sm + S::A_BYTES;
    V *stage = reinterpret_cast<V *>(sm);   // [TR][TC + 1], after the MMAs
    __shared__ __align__(8) TileSmem ts;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    tile_setup(ts);
    if (threadIdx.x == 0) tile_load<S>(ts, &tmA, &tmB, sA, sB, (int)r0, (int)c0);

    // this thread's row x and its 16 columns y = yb + k; the valid ones
    // (y < Ln, y <= x) are the prefix k < kv.  Their entries of A are read
    // transposed (A is symmetric), so that a warp's loads are contiguous.
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t x = r0 + quarter * 32 + lane;
    const int64_t yb = c0 + half * 16;
    int64_t kv = Ln - yb < x - yb + 1 ? Ln - yb : x - yb + 1;
    kv = x < Ln ? (kv < 16 ? kv : 16) : 0;
    const int64_t rx = x < Ln ? rem[x] : 0;
    const float sx = x < Ln ? gs[x] : 0.f;
    V av[16];
    float cy[16];   // s_x s_y, a product of two powers of two
#pragma unroll
    for (int k = 0; k < 16; k++) {
        av[k] = V{};
        cy[k] = 0.f;
        if (k < kv) {
            av[k] = Av[(int64_t)rem[yb + k] * lda + rx];
            cy[k] = sx * gs[yb + k];
        }
    }

    if (threadIdx.x == 0) tile_mma<S>(ts, sA, sB);
    const bool ok = tile_wait(ts);
    if (ok) {
        V *up = Anv + yb * lda + x;                                   // upper entries
        V *sp = stage + (quarter * 32 + lane) * (TC + 1) + half * 16;   // lower, staged
#pragma unroll
        for (int ps = 0; ps < 2; ps++) {
            uint32_t dg[S::NDIAG][8];
            tile_ld8<S::NDIAG>(ts, quarter, half * 16 + ps * 8, dg);
#pragma unroll
            for (int k8 = 0; k8 < 8; k8++) {
                const int k = ps * 8 + k8;
                if (k >= kv) break;
                V r;
                if constexpr (F64) r = fold_sub64(dg, k8, cy[k], av[k]);
                else r = fold_sub(dg, k8, cy[k], av[k]);
                up[k * lda] = r;
                sp[k] = r;
            }
        }
    }
    __syncthreads();   // staged tile complete
    if (ok) {
        // lower entries A'[x, y], y < x: one 256-byte row segment per warp store
        for (int i = warp; i < TR; i += TTHREADS / 32) {
            const int64_t xr = r0 + i, y = c0 + lane;
            if (xr < Ln && y < xr) Anv[xr * lda + y] = stage[i * (TC + 1) + lane];
        }
    }
    tile_teardown(ts, st, nullptr);
}

// ------------------------------------------------- K = R11^-1 R12, blocked
// Backward substitution in blocks of 32 rows, k = nblk-1 .. 0:
//     X_k = U_k^{-1} B_k             (U_k: the k-th 32 x 32 diagonal block
//                                     of R11, inverted in FP64 beforehand)
//     B_i -= R[i, block k] X_k       for every row i < 32 k.
// The updates are products of depth 32 on the tensor cores from exact digit
// slices, as in the trailing update: the 32 entries of row i of R in block
// column k (power-of-two scale per row) against the 32 entries of each
// column of X_k (scale per column).  B (r x q, FP64 in memory) is updated in
// double-float and stored back exactly (48 significant bits fit FP64);
// X_k = U_k^{-1} B_k runs in double-float on the FP32 pipes.  Step k is two
// launches: ksolve_prep_kernel (the digits of R's block column k for the
// rows above it, and X_k with its digits) and ksolve_update_kernel.

// Blocks [0, nrb): one warp per row i < rows_r (digits of R[i, 32k ..]);
// blocks [nrb, ..): one warp per column c < q (X_k[:, c], written to B,
// and its digits).
__global__ void __launch_bounds__(256)
ksolve_prep_kernel(const double *__restrict__ R, int64_t ldr, const double *__restrict__ DinvF,
                   int64_t r, double *__restrict__ B, int64_t ldb, int64_t q, int64_t k,
                   int64_t rows_r, int64_t nrb, __nv_bfloat16 *__restrict__ GR,
                   float *__restrict__ gsR, int64_t Rcap, __nv_bfloat16 *__restrict__ GX,
                   float *__restrict__ gsX, int64_t Qcap) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c0 = k * 32;
    const int nbk = (int)(r - c0 < 32 ? r - c0 : 32);
    if (blockIdx.x < nrb) {
        const int64_t i = (int64_t)blockIdx.x * 8 + warp;
        if (i >= rows_r) return;
        const F2 v = lane < nbk ? d2df(R[i * ldr + c0 + lane]) : F2{0.f, 0.f};
        warp_digits(v, GR + i * 32 + lane, Rcap * 32, gsR + i);
        return;
    }
    const int64_t c = (int64_t)(blockIdx.x - nrb) * 8 + warp;
    if (c >= q) return;
    // lane a holds B[c0 + a, c]; lane l forms X[l] = sum_a Uinv[l, a] B[a]
    const F2 bv = lane < nbk ? d2df(B[(c0 + lane) * ldb + c]) : F2{0.f, 0.f};
    const double *ui = DinvF + k * 1024 + lane * 32;
    float sh = 0.f, sl = 0.f;
#pragma unroll 8
    for (int a2 = 0; a2 < 32; a2++) {
        const F2 ba{__shfl_sync(0xffffffffu, bv.h, a2), __shfl_sync(0xffffffffu, bv.l, a2)};
        df_acc_prod(sh, sl, d2df(ui[a2]), ba);
    }
    const F2 x = lane < nbk ? df_renorm(sh, sl) : F2{0.f, 0.f};
    if (lane < nbk) B[(c0 + lane) * ldb + c] = f2d(x.h) + f2d(x.l);
    warp_digits(x, GX + c * 32 + lane, Qcap * 32, gsX + c);
}

// Tiles of 128 rows (< rows) x 32 columns (< q) of B: B -= R[:, block k] X_k.
// The tile of B is staged in shared memory (row-wise coalesced loads and
// stores) while the copies and MMAs run.
__global__ void __launch_bounds__(TTHREADS, 2)
ksolve_update_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     double *__restrict__ B, int64_t ldb, int64_t rows, int64_t q,
                     const float *__restrict__ gsR, const float *__restrict__ gsX, int *flag) {
    const int64_t nnt = (q + TC - 1) / TC;
    const int64_t r0 = (int64_t)(blockIdx.x / nnt) * TR, c0 = (int64_t)(blockIdx.x % nnt) * TC;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm, *sB = sm + A_BYTES;
    double *stage = reinterpret_cast<double *>(sm + KS_STAGE_OFF);   // [TR][TC + 1]
    __shared__ __align__(8) TileSmem ts;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    tile_setup(ts);
    if (threadIdx.x == 0) tile_load(ts, &tmA, &tmB, sA, sB, (int)r0, (int)c0);
    const bool cin = c0 + lane < q;
    for (int i = warp; i < TR; i += TTHREADS / 32)
        if (r0 + i < rows && cin) stage[i * (TC + 1) + lane] = B[(r0 + i) * ldb + c0 + lane];
    if (threadIdx.x == 0) tile_mma(ts, sA, sB);
    const bool ok = tile_wait(ts);
    __syncthreads();   // staged tile of B visible
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t x = r0 + quarter * 32 + lane;
    if (ok && x < rows) {
        const float sx = gsR[x];
        double *sp = stage + (quarter * 32 + lane) * (TC + 1) + half * 16;
#pragma unroll
        for (int ps = 0; ps < 2; ps++) {
            uint32_t dg[NDIAG][8];
            tile_ld8(ts, quarter, half * 16 + ps * 8, dg);
#pragma unroll
            for (int k8 = 0; k8 < 8; k8++) {
                const int kk = ps * 8 + k8;
                const int64_t y = c0 + half * 16 + kk;
                if (y >= q) break;
                const F2 v = fold_sub(dg, k8, sx * gsX[y], d2df(sp[kk]));
                sp[kk] = f2d(v.h) + f2d(v.l);
            }
        }
    }
    __syncthreads();   // updated tile complete
    if (ok)
        for (int i = warp; i < TR; i += TTHREADS / 32)
            if (r0 + i < rows && cin) B[(r0 + i) * ldb + c0 + lane] = stage[i * (TC + 1) + lane];
    tile_teardown(ts, nullptr, flag);
}

}  // namespace

int64_t trail_tc_rows(int64_t L) { return (L + TR - 1) / TR * TR; }

namespace {
struct KsWs {
    __nv_bfloat16 *GR, *GX;
    float *gsR, *gsX;
    int64_t Rcap, Qcap;
};
KsWs ksolve_carve(Arena &a, int64_t r, int64_t q) {
    KsWs w;
    w.Rcap = (r + TR - 1) / TR * TR;
    w.Qcap = (q + TC - 1) / TC * TC;
    w.GR = a.take<__nv_bfloat16>(NPLANE * w.Rcap * 32);
    w.GX = a.take<__nv_bfloat16>(NPLANE * w.Qcap * 32);
    w.gsR = a.take<float>(w.Rcap);
    w.gsX = a.take<float>(w.Qcap);
    return w;
}
}  // namespace

size_t ksolve_tc_bytes(int64_t r, int64_t q) {
    Arena a;
    ksolve_carve(a, r, q);
    return a.used + 256;
}

void ksolve_tc(cudaStream_t s, const double *R, int64_t ldr, const double *DinvF, int64_t r,
               double *B, int64_t ldb, int64_t q, void *ws, int *flag) {
    static const bool attr = [] {
        ELM_CUDA(cudaFuncSetAttribute(ksolve_update_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TRAIL_SMEM));
        return true;
    }();
    (void)attr;
    if (r <= 0 || q <= 0) return;
    Arena a;
    a.base = (char *)ws;
    a.cap = ksolve_tc_bytes(r, q);
    const KsWs w = ksolve_carve(a, r, q);
    // rows beyond r and columns beyond q are never written back; zero their
    // digits once so that no stale bits reach the tensor cores
    ELM_CUDA(cudaMemsetAsync(w.GR, 0, sizeof(__nv_bfloat16) * NPLANE * w.Rcap * 32, s));
    ELM_CUDA(cudaMemsetAsync(w.GX, 0, sizeof(__nv_bfloat16) * NPLANE * w.Qcap * 32, s));
    const CUtensorMap ma = make_map_planes(w.GR, w.Rcap, NPLANE, TR, NDIG);
    const CUtensorMap mb = make_map_planes(w.GX, w.Qcap, NPLANE, TC, NPLANE);
    const int64_t nblk = (r + 31) / 32, nnt = (q + TC - 1) / TC, nxb = (q + 7) / 8;
    for (int64_t k = nblk - 1; k >= 0; k--) {
        const int64_t rows = 32 * k, nrb = (rows + 7) / 8;
        ksolve_prep_kernel<<<(unsigned)(nrb + nxb), 256, 0, s>>>(
            R, ldr, DinvF, r, B, ldb, q, k, rows, nrb, w.GR, w.gsR, w.Rcap, w.GX, w.gsX, w.Qcap);
        ELM_CHECK_LAUNCH();
        if (rows == 0) continue;
        const int64_t nmt = (rows + TR - 1) / TR;
        ksolve_update_kernel<<<(unsigned)(nmt * nnt), TTHREADS, TRAIL_SMEM, s>>>(
            ma, mb, B, ldb, rows, q, w.gsR, w.gsX, flag);
        ELM_CHECK_LAUNCH();
    }
}

namespace {
template <bool F64>
void trailing_tc_launch(cudaStream_t s, const double *A, double *An, int64_t lda, const double *P,
                        int64_t ldp, const int32_t *rem, FactorState *st, __nv_bfloat16 *G,
                        float *gs, int64_t Lcap, int64_t Lup) {
    using S = Scheme<F64>;
    static const bool attr = [] {   // once per process and scheme, thread-safely
        ELM_CUDA(cudaFuncSetAttribute(trailing_tc_kernel<F64>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TRAIL_SMEM));
        return true;
    }();
    (void)attr;
    const CUtensorMap ma = make_map_planes(G, Lcap, S::NPLANE, TR, S::NDIG);
    const CUtensorMap mb = make_map_planes(G, Lcap, S::NPLANE, TC, S::NPLANE);
    const int64_t rows = trail_tc_rows(Lup);   // rows any tile reads
    trail_digits_kernel<F64><<<(unsigned)(rows / 8), 256, 0, s>>>(P, ldp, rem, st, G, gs, Lcap,
                                                                  rows);
    ELM_CHECK_LAUNCH();
    const int64_t nrb = rows / TR;
    trailing_tc_kernel<F64><<<(unsigned)(2 * nrb * (nrb + 1)), TTHREADS, TRAIL_SMEM, s>>>(
        ma, mb, A, An, lda, rem, gs, st);
    ELM_CHECK_LAUNCH();
}
}  // namespace

int trail_tc_planes() { return MAX_PLANES; }

void trailing_tc(cudaStream_t s, const double *A, double *An, int64_t lda, const double *P,
                 int64_t ldp, const int32_t *rem, FactorState *st, __nv_bfloat16 *G, float *gs,
                 int64_t Lcap, int64_t Lup, bool f64) {
    if (Lup <= 0) return;
    if (Lcap % TR || Lup > Lcap) throw ElmError(ELM_ERR_ARG, "trailing update: bad sizes");
    if (f64) trailing_tc_launch<true>(s, A, An, lda, P, ldp, rem, st, G, gs, Lcap, Lup);
    else trailing_tc_launch<false>(s, A, An, lda, P, ldp, rem, st, G, gs, Lcap, Lup);
}

}  // namespace elm
