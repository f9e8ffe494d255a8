// Trailing update of the mixed form's pivoted factorisation on the tensor
// cores (Eq. 6; Algorithm 1, steps 3-4).  After a panel of up to 32 pivots
// every remaining entry of the active matrix becomes
//     A'[x, y] = A[rem x, rem y] - sum_t P[t, rem x] P[t, rem y],
// with rem the compaction map of the unpivoted columns.  A and the panel
// rows P hold double-float pairs (h + l, two floats in eight bytes).
//
// Digits.  The 32 panel entries of each remaining column x are scaled by a
// power of two s_x >= their largest magnitude and split into six signed
// 8-bit digits, integers |a_j| <= 128 (exact in bf16):
//     P[t, x] / s_x = sum_{j<6} a_j 2^(-7-8j) + r,   |r| <= 2^-48.
// Products.  For a digit pair (i, j) one tcgen05 MMA (kind::f16, bf16
// operands, FP32 accumulator in tensor memory) sums the 32 products
// |a_i b_j| <= 2^14 of a pair: at most 2^19 per pair and six pairs share the
// weight 2^(-14-8d) of diagonal d = i + j, so every accumulator stays an
// integer below 2^22 and the FP32 accumulation is exact in any order.
// Pairs with i + j <= 6 are kept (26 of 36); the others weigh below 2^-48
// of s_x s_y.  The drain folds the seven exact diagonal sums into a
// double-float value (TwoSum, FP32 pipes), scales it by s_x s_y and
// subtracts it from the double-float entry of A: about 2^-46 relative to
// s_x s_y, like the double-float update it replaces, in about 45 FP32
// instructions per entry instead of 32 products of 10.
// Symmetry.  The integer sums are symmetric in (x, y) and the scales are per
// column, so bitwise-equal columns stay bitwise equal (ties in the pivot
// search resolve as in the double-float update) and A' is exactly
// symmetric; each lower tile also writes its mirror.
//
// Layout of the digit planes: G[c][p][32] bf16, p < Lcap (compacted column
// index, Lcap a multiple of 128), K = 32 panel rows (zero past the panel's
// pivots).  Plane c = 6 - j holds digit j (c = 1..6); plane 0 is all zeros
// and stands for a seventh digit of the B operand, so that for every A
// digit i the pairs (i, 6-i..0) form one MMA over B planes i..6 whose
// diagonal d lands at tensor-memory column (6 - d) 32, with every MMA
// starting at column 0.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "df_arith.cuh"
#include "elm_internal.cuh"
#include "tc_ptx.cuh"

namespace elm {

namespace {

using df::F2;
using namespace tcx;

static_assert(TRAIL_TC_K == 32, "one 64-byte K row of bf16 digits per plane");
constexpr int TR = 128;                    // tile rows (TMEM lanes)
constexpr int TC = 32;                     // tile columns
constexpr int NDIG = 6;                    // digits per panel entry
constexpr int NDIAG = NDIG + 1;            // kept diagonals d = 0..6
constexpr int NPLANE = NDIG + 1;           // digit planes incl. the zero plane
constexpr uint32_t A_PLANE = TR * 64;      // bytes of one A plane (128 rows x 32 bf16)
constexpr uint32_t B_PLANE = TC * 64;      // bytes of one B plane
constexpr uint32_t A_BYTES = NDIG * A_PLANE;
constexpr uint32_t B_BYTES = NPLANE * B_PLANE;
constexpr uint32_t TMEM_COLS = 256;        // NDIAG x 32 = 224 used
constexpr int TTHREADS = 256;              // two warps per TMEM lane quarter
// Dynamic shared memory: the operands (62 KB) and, once the MMAs are done,
// the transposed output tile.  Asking for 100 KB keeps at most two CTAs on
// an SM, whose tensor memory holds two allocations of 256 columns.
constexpr size_t TRAIL_SMEM = 100 * 1024;
constexpr uint64_t TRAIL_WAIT_NS = 2000000000ull;
// kind::f16, bf16 x bf16 -> f32, K-major operands, M = 128 (N set per MMA)
constexpr uint32_t IDESC_M128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TR >> 4) << 24);
static_assert(NDIAG * TC <= (int)TMEM_COLS, "diagonals exceed the allocation");
static_assert((NPLANE - 0) * TC <= 256, "widest MMA above N = 256");
static_assert(A_BYTES + B_BYTES + 1024 <= TRAIL_SMEM, "operands exceed shared memory");
static_assert((size_t)TR * (TC + 1) * 8 + 1024 <= TRAIL_SMEM, "output tile exceeds shared memory");

__device__ __forceinline__ float rint_small(float x) {   // |x| < 2^22: nearest integer
    return __fadd_rn(__fadd_rn(x, 12582912.f), -12582912.f);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One warp per compacted column p < rows: scale and digits of its panel
// entries P[t, rem p], t < steps (zero beyond, and for p >= Ln).
__global__ void __launch_bounds__(256)
trail_digits_kernel(const F2 *__restrict__ P, int64_t ldp, const int32_t *__restrict__ rem,
                    const FactorState *__restrict__ st, __nv_bfloat16 *__restrict__ G,
                    float *__restrict__ gs, int64_t Lcap, int64_t rows) {
    const FactorState s = *st;
    if (s.done) return;
    const int64_t Ln = s.Lr;
    const int steps = (int)s.steps;
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= rows) return;
    F2 v{0.f, 0.f};
    if (p < Ln && lane < steps) v = P[(int64_t)lane * ldp + rem[p]];
    // smallest power of two >= the largest |h| of the column (1 for a zero
    // column; a denormal maximum rounds up to 2^-126)
    const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(v.h)));
    uint32_t sb = (m + 0x7fffffu) & 0xff800000u;
    if (sb == 0u) sb = 0x3f800000u;
    const float inv = __uint_as_float((254u << 23) - sb);   // 1 / s, exact
    // x = v / s, |x| <= 1 + 2^-24; digit j carries weight 2^(-7-8j)
    float rh = v.h * inv * 128.f, rl = v.l * inv * 128.f;
    __nv_bfloat16 *g = G + p * 32 + lane;
    const int64_t pstride = Lcap * 32;
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
    if (lane == 0) gs[p] = __uint_as_float(sb);
}

// Lower tiles of 128 rows x 32 columns: row block rb holds column blocks
// 0 .. 4 rb + 3.  Warp 0 allocates tensor memory; thread 0 issues the two
// TMA copies (all A planes of the tile's rows, all B planes of its columns)
// and the twelve MMAs; all eight warps prefetch their entries of A, then
// drain (warp w: TMEM lanes 32 (w mod 4) .., columns 16 (w / 4) ..).
__global__ void __launch_bounds__(TTHREADS, 2)
trailing_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const F2 *__restrict__ A, F2 *__restrict__ An, int64_t lda,
                   const int32_t *__restrict__ rem, const float *__restrict__ gs,
                   FactorState *st) {
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
    uint8_t *sA = sm, *sB = sm + A_BYTES;
    F2 *stage = reinterpret_cast<F2 *>(sm);   // [TR][TC + 1], after the MMAs
    __shared__ __align__(8) uint64_t full_bar, mma_bar;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(&full_bar, 1);
        mbar_init(&mma_bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    volatile int *abort = &abort_sh;

    if (threadIdx.x == 0) {
        mbar_expect_tx(&full_bar, A_BYTES + B_BYTES);
        tma_3d(&tmA, &full_bar, sA, 0, (int)r0, 1);   // planes 1..6: A digits 5..0
        tma_3d(&tmB, &full_bar, sB, 0, (int)c0, 0);   // planes 0..6: B digits "6", 5..0
    }

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
    F2 av[16];
    float cy[16];   // s_x s_y, a product of two powers of two
#pragma unroll
    for (int k = 0; k < 16; k++) {
        av[k] = F2{0.f, 0.f};
        cy[k] = 0.f;
        if (k < kv) {
            av[k] = A[(int64_t)rem[yb + k] * lda + rx];
            cy[k] = sx * gs[yb + k];
        }
    }

    if (threadIdx.x == 0) {
        if (mbar_wait(&full_bar, 0, abort, TRAIL_WAIT_NS)) {
            tc_fence_after();
            const uint64_t da0 = desc_sw64(su32(sA)), db0 = desc_sw64(su32(sB));
            // A digit i (smem plane 5 - i) against B planes i..6 (digits
            // 6 - i .. 0): diagonal d = i + (6 - c) at column (6 - d) 32.
            // i = 0 reaches every column and comes first.
#pragma unroll
            for (int i = 0; i < NDIG; i++) {
                const uint64_t da = da0 + (uint64_t)(((NDIG - 1 - i) * A_PLANE) >> 4);
                const uint64_t db = db0 + (uint64_t)((i * B_PLANE) >> 4);
                const uint32_t idesc = IDESC_M128 | ((uint32_t)(((NPLANE - i) * TC) >> 3) << 17);
#pragma unroll
                for (int kk = 0; kk < 2; kk++)   // K = 32: two steps of 16
                    mma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (i == 0 && kk == 0) ? 0u : 1u);
            }
        }
        mma_commit(&mma_bar);   // arrives once every MMA issued above has completed
    }
    const bool ok = mbar_wait(&mma_bar, 0, abort, TRAIL_WAIT_NS) && !*abort;
    tc_fence_after();

    if (ok) {
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        F2 *up = An + yb * lda + x;                                   // upper entries
        F2 *sp = stage + (quarter * 32 + lane) * (TC + 1) + half * 16;   // lower, staged
#pragma unroll
        for (int ps = 0; ps < 2; ps++) {
            uint32_t dg[NDIAG][8];
#pragma unroll
            for (int d = 0; d < NDIAG; d++)
                tmem_ld8(tl + (uint32_t)((NDIAG - 1 - d) * TC + half * 16 + ps * 8), dg[d]);
            tmem_wait_ld();
#pragma unroll
            for (int d = 0; d < NDIAG; d++) reg_fence8(dg[d]);
#pragma unroll
            for (int k8 = 0; k8 < 8; k8++) {
                const int k = ps * 8 + k8;
                if (k >= kv) break;
                // sum_d D_d 2^(-14-8d): the two leading pairs exactly by TwoSum,
                // the three smallest terms (below 2^-24) in FP32
                float h1, l1, h2, l2, h, e;
                two_sum(__uint_as_float(dg[0][k8]) * 0x1p-14f, __uint_as_float(dg[1][k8]) * 0x1p-22f, h1, l1);
                two_sum(__uint_as_float(dg[2][k8]) * 0x1p-30f, __uint_as_float(dg[3][k8]) * 0x1p-38f, h2, l2);
                const float tail = __uint_as_float(dg[4][k8]) * 0x1p-46f +
                                   (__uint_as_float(dg[5][k8]) * 0x1p-54f +
                                    __uint_as_float(dg[6][k8]) * 0x1p-62f);
                two_sum(h1, h2, h, e);
                const float l = (((l1 + l2) + e) + tail) * cy[k];
                h *= cy[k];
                // A - (h + l), renormalised
                float sh, se;
                two_sum(av[k].h, -h, sh, se);
                se += av[k].l - l;
                const float rh = sh + se;
                const F2 r{rh, se - (rh - sh)};
                up[k * lda] = r;
                sp[k] = r;
            }
        }
    }
    tc_fence_before();
    __syncthreads();   // staged tile complete; every tensor-memory read done
    if (ok) {
        // lower entries A'[x, y], y < x: one 256-byte row segment per warp store
        for (int i = warp; i < TR; i += TTHREADS / 32) {
            const int64_t xr = r0 + i, y = c0 + lane;
            if (xr < Ln && y < xr) An[xr * lda + y] = stage[i * (TC + 1) + lane];
        }
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
    if (threadIdx.x == 0 && *abort) {
        // let the copies land before the CTA's shared memory is released
        const uint64_t t0 = gtime();
        while (!mbar_try(&full_bar, 0) && gtime() - t0 < TRAIL_WAIT_NS) {
        }
        atomicOr(&st->flags, 2);
    }
}

}  // namespace

int64_t trail_tc_rows(int64_t L) { return (L + TR - 1) / TR * TR; }

void trailing_tc(cudaStream_t s, const double *A, double *An, int64_t lda, const double *P,
                 int64_t ldp, const int32_t *rem, FactorState *st, __nv_bfloat16 *G, float *gs,
                 int64_t Lcap, int64_t Lup) {
    static const bool attr = [] {   // once per process, thread-safely
        ELM_CUDA(cudaFuncSetAttribute(trailing_tc_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TRAIL_SMEM));
        return true;
    }();
    (void)attr;
    if (Lup <= 0) return;
    if (Lcap % TR || Lup > Lcap)
        throw ElmError(ELM_ERR_ARG, "trailing update: bad sizes");
    const CUtensorMap ma = make_map_planes(G, Lcap, NPLANE, TR, NDIG);
    const CUtensorMap mb = make_map_planes(G, Lcap, NPLANE, TC, NPLANE);
    const int64_t rows = trail_tc_rows(Lup);   // rows any tile reads
    trail_digits_kernel<<<(unsigned)(rows / 8), 256, 0, s>>>((const F2 *)P, ldp, rem, st, G, gs,
                                                             Lcap, rows);
    ELM_CHECK_LAUNCH();
    const int64_t nrb = rows / TR;
    trailing_tc_kernel<<<(unsigned)(2 * nrb * (nrb + 1)), TTHREADS, TRAIL_SMEM, s>>>(
        ma, mb, (const F2 *)A, (F2 *)An, lda, rem, gs, st);
    ELM_CHECK_LAUNCH();
}

}  // namespace elm
