// Mixed-precision dense products on the 5th-generation tensor cores.
//
// The hidden-layer pre-activation X W (Eq. 1, Eq. 3) and the Gram blocks
// H^T H, H^T T (Eqs. 9-13) are computed from exact integer-digit slices:
// every operand row is scaled by a power of two into [-1, 1] and split into
// P signed digits of B bits,
//     v = sum_p d_p 2^(-(B-1) - B(p-1)),   |d_p| <= 2^(B-1),
// each digit an integer held exactly in bf16.  For a pair of digit planes
// (p, q) the tcgen05 MMA (kind::f16, bf16 operands, FP32 accumulator in
// tensor memory) sums products |d_p d_q| <= 2^(2B-2); over a K chunk of
// 2^(24-2B+2) / 4 elements (256 for B = 8, 1024 for B = 7) the partial sums
// stay below 2^24, so the FP32 accumulation is exact.  Pairs with the same
// weight 2^(-B(p+q-2)) share one accumulator ("diagonal" t = p + q), and
// the pairs of one A plane with consecutive B planes form one MMA of width
// up to 256 (B planes stored in descending order, diagonal t at TMEM column
// (TMAX - t) 64).  After each chunk the drain warps fold the diagonals, as
// exact integers, into a per-element int64 fixed-point running sum kept in
// tensor memory; the epilogue converts it to FP64 once (the hidden layer,
// one chunk deep, forms its pre-activation directly as a double-float
// pair).  So the only roundings are the final conversion and, for
// diagonals holding more than four pairs (weight at most 2^(-4B) of the
// leading one), the FP32 accumulator itself.  Pairs with p + q > TMAX are
// dropped.
//
// Kernel layout (persistent, 128 x 64 output tiles, 320 threads):
//   warp 0      TMA producer: digit tiles of A (128 rows) and B (64 rows),
//               32 K-elements per stage, 64-byte swizzle, STAGES-deep ring
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warps 2..9  drains and the epilogue (two warps per TMEM lane quarter,
//               32 columns each)
// Every mbarrier wait is bounded by wall-clock time; on expiry the kernel
// sets an error flag, stops issuing work and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <vector>

#include "elm_internal.cuh"
#include "oz_tiles.cuh"
#include "tc_ptx.cuh"

namespace elm {

namespace {

constexpr int BM = 128;         // tile rows (A rows, TMEM lanes)
constexpr int BN = 64;          // tile columns (B rows)
constexpr int SK = 32;          // K elements per stage (64 bytes of bf16)

// K stages per exact chunk for B-bit digits: products <= 2^(2B-2), and four
// pairs of a diagonal over a chunk must stay <= 2^24.
template <int DBITS>
__host__ __device__ constexpr int chunk_slabs() {
    return (1 << (24 - 2 * (DBITS - 1) - 2)) / SK;
}
constexpr int NTHREADS = 320;   // warp 0 TMA, warp 1 MMA, warps 2..9 drains/epilogue
constexpr int NEPI = 256;       // drain/epilogue threads: two warps per TMEM lane quarter
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s bound on any single wait

using namespace tcx;

// Instruction descriptor: kind::f16, bf16 x bf16 -> f32, both K-major,
// M = 128; the N field (bits 17-22, N / 8) is set per MMA.
constexpr uint32_t IDESC_M = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BM >> 4) << 24);

// ---------------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two floats with the error-free transformations
// of Knuth (TwoSum) and Dekker (FastTwoSum, TwoProduct via FMA): about 48
// significant bits from FP32 instructions.
struct dfl {
    float h, l;
};

// Two small integers (|d| <= 256, held in floats) as packed bf16: such a
// float has at most 8 significant bits, so its bf16 encoding is exactly its
// upper 16 bits -- integer operations, no conversion instruction.
__device__ __forceinline__ uint32_t pack_bf16_int(float lo, float hi) {
    return (__float_as_uint(lo) >> 16) | (__float_as_uint(hi) & 0xffff0000u);
}
// Nearest integer, ties to even, of |x| < 2^22 on the FP32 add pipe: in
// x + 1.5 2^23 the unit is the last mantissa bit, so the add rounds x to an
// integer and the subtraction is exact.  Same result as rintf, which issues
// on the narrower conversion (XU) pipe.
__device__ __forceinline__ float rint_digit(float x) {
    return __fadd_rn(__fadd_rn(x, 12582912.f), -12582912.f);
}
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    dfl s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, s.l + x.l + y.l);
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, fmaf(x.l, y.h, e));
    return fast_two_sum(p, e);
}

// Logistic function of a double-float argument from a table of sigma and
// sigma' (double-float) at z_k = -40 + k / 64, k = 0 .. 5120, and the Taylor
// expansion to fourth order in delta = u - z_k (|delta| <= 2^-7):
//   sigma(u) = s0 + s1 d + s2 d^2/2 + s3 d^3/6 + s4 d^4/24 + O(d^5),
// with the derivatives of the logistic function written through s = sigma:
//   s1 = s (1 - s), s2 = s1 (1 - 2 s), s3 = s1 (1 - 6 s + 6 s^2),
//   s4 = s2 (1 - 12 s + 12 s^2).
// The fifth-order remainder is below 1e-13; terms after the linear one are
// at most 2^-15 and are evaluated in FP32.  Outside [-40, 40] sigma is 0 or
// 1 to within 5e-18.
constexpr int SIG_N = 5121;
__device__ __forceinline__ dfl sigmoid_df(dfl u, const float4 *__restrict__ tab) {
    if (u.h <= -40.f) return {0.f, 0.f};
    if (u.h >= 40.f) return {1.f, 0.f};
    int k = __float2int_rn((u.h + 40.f) * 64.f);
    k = k < 0 ? 0 : (k > SIG_N - 1 ? SIG_N - 1 : k);
    const float z0 = (float)k * 0.015625f - 40.f;   // exact
    const dfl d = two_sum(u.h - z0, u.l);           // u.h - z0 is exact
    const float4 t = __ldg(tab + k);
    const dfl lin = df_mul({t.z, t.w}, d);
    const float s = t.x, s1 = t.z;
    const float a2 = s1 * fmaf(-2.f, s, 1.f);
    const float q6 = fmaf(6.f * s, s - 1.f, 1.f);
    const float q12 = fmaf(12.f * s, s - 1.f, 1.f);
    const float a3 = s1 * q6, a4 = a2 * q12;
    const float dh = d.h;
    const float hot =
        dh * dh * fmaf(dh, fmaf(dh, a4 * (1.f / 24.f), a3 * (1.f / 6.f)), 0.5f * a2);
    const dfl h = df_add({t.x, t.y}, lin);
    return fast_two_sum(h.h, h.l + hot);
}

// Epilogue of the fused hidden layer: H = a g(z + b) from the exact
// pre-activation, written as Gram digit planes.
struct ActParams {
    const double *b, *a;    // bias and output scale (a may be NULL)
    int act;                // ELM_ACT_*
    int64_t L, m;           // hidden width; rows L .. L+m-1 belong to targets
    __nv_bfloat16 *planes;  // Gram digit planes: blocks of kb samples, [block][plane][row][kb]
    int64_t plane_stride;   // Lp * kb
    int64_t kb;             // samples per block (gram_kblk)
    int64_t blk_stride;     // GRAM_PH * Lp * kb
    const double *hs;       // Gram row scales (pow2_ceil(a_j))
    const float4 *tab;      // sigmoid table (s0 hi/lo, s1 hi/lo) on a 2^-6 grid
    const float *csf;       // per-sample scales as floats
    const float4 *rowc;     // per hidden row: {rowf, 1/hs, b hi, b lo}, {a hi, a lo, scaled, 0}
    double *Ht;             // optional FP64 H^T (row j, column i)
    float2 *Hdf;            // optional H as double-float pairs, sample-major: [n * ldhd + m]
    int64_t ldhd;
    int64_t ldh;
};

struct OzParams {
    int64_t a_rows;     // rows per A digit plane
    int64_t b_rows;     // rows per B digit plane
    int64_t K;          // padded K (multiple of SK)
    int64_t m_valid;    // output rows to write
    int64_t n_valid;    // output columns to write
    int64_t ntile_m;    // tiles along M
    int gram;           // 1: lower-triangular tile set, mirrored writes
    double out_scale;
    const double *rscale;  // per output row (A row) power-of-two scale
    const double *cscale;  // per output column (B row) scale
    double *out;
    int64_t ldo;
    int *err;
    int64_t ntiles;     // tiles in the tile set
    int64_t whole;      // tiles below this run over the whole K range, one CTA each
    long long *part;    // EPI == 0: int64 partial sums of the tiles from `whole` on
    uint64_t wait_ns;   // bound of each pipeline wait (0: WAIT_NS)
    int accumulate;     // EPI == 0, whole tiles: add to the output instead of storing
    int64_t n_base;     // non-Gram tiles: first B row (column) of the tile set
    int64_t kblk;       // > 0: operand planes stored in blocks of kblk K elements
                        // ([block][row][kblk], 3-D tensor maps); 0: one block of K
    ActParams ap;       // used when the kernel's EPI != 0
};

// Fused hidden-layer epilogue for one row (neuron j = m) and 32 samples
// n0 .. n0+31, from the pre-activation V (double-float, in units of
// 2^(-2(B-1) - B(TMAX-2)) * ws[m] * xs[n]) held in registers: z -> h =
// a_j g(z + b_j) -> GRAM_PH digits of h / hs[j] on the 2^-34 grid.  All
// arithmetic per element is FP32 / double-float.
constexpr int GRAM_PH_ = 5, GRAM_BITS_ = 7;
struct RowAct {
    bool live, skip, scaled;
    float rowf, inv_hs;
    dfl bj, aj;
};
// Per-row constants of the epilogue, formed once per hidden row (FP64
// work, so not once per tile): rowf = out_scale rscale 2^(-B (TMAX - 2)),
// 1 / hs, the bias b and the output scale a as double-float pairs.
template <int DBITS, int TMAX>
__global__ void rowconst_kernel(double out_scale, const double *__restrict__ rscale,
                                const double *__restrict__ b, const double *__restrict__ a,
                                const double *__restrict__ hs, int64_t L, int64_t Lp,
                                float4 *__restrict__ rowc) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Lp) return;
    float4 c0 = make_float4(0.f, 1.f, 0.f, 0.f), c1 = make_float4(1.f, 0.f, 0.f, 0.f);
    if (m < L) {
        c0.x = (float)ldexp(out_scale * rscale[m], -DBITS * (TMAX - 2));
        c0.y = (float)(1.0 / hs[m]);
        const double bv = b[m];
        c0.z = (float)bv;
        c0.w = (float)(bv - (double)c0.z);
        if (a) {
            const double av = a[m];
            c1.x = (float)av;
            c1.y = (float)(av - (double)c1.x);
            c1.z = 1.f;
        }
    }
    rowc[2 * m] = c0;
    rowc[2 * m + 1] = c1;
}
__device__ __forceinline__ RowAct row_setup(const OzParams &P, int64_t m) {
    const ActParams &A = P.ap;
    RowAct r{};
    r.skip = m >= A.L && m < A.L + A.m;            // target rows: written by the slicer
    r.live = m < A.L;
    r.aj = {1.f, 0.f};
    r.inv_hs = 1.f;
    if (r.live) {
        const float4 c0 = A.rowc[2 * m], c1 = A.rowc[2 * m + 1];
        r.rowf = c0.x;
        r.inv_hs = c0.y;
        r.bj = {c0.z, c0.w};
        r.aj = {c1.x, c1.y};
        r.scaled = c1.z != 0.f;
    }
    return r;
}
// 8 samples n0 .. n0+7 of one row; HT: also write FP64 H^T (a compile-time
// switch, so the training form issues no FP64 conversion for it)
template <bool HT>
__device__ __forceinline__ void hidden_emit8(const OzParams &P, const RowAct &R, int64_t m,
                                             int64_t n0, const dfl *V) {
    const ActParams &A = P.ap;
    if (R.skip) return;
    float dg[GRAM_PH_][8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int64_t n = n0 + i;
        const bool on = R.live && n < P.n_valid;
        const float f = on ? R.rowf * A.csf[n] : 0.f;   // two exact power-of-two products
        dfl z{V[i].h * f, V[i].l * f};
        z = df_add(z, R.bj);
        dfl hv;
        if (A.act == ELM_ACT_TANH) {                    // tanh u = 2 sigma(2u) - 1
            dfl sg = sigmoid_df({2.f * z.h, 2.f * z.l}, A.tab);
            hv = df_add({2.f * sg.h, 2.f * sg.l}, {-1.f, 0.f});
        } else {
            hv = sigmoid_df(z, A.tab);
        }
        if (R.scaled) hv = df_mul(hv, R.aj);
        if (HT && on) A.Ht[m * A.ldh + n] = (double)hv.h + (double)hv.l;
        if (on && A.Hdf) A.Hdf[n * A.ldhd + m] = make_float2(hv.h, hv.l);   // lanes: consecutive m
        hv.h = on ? hv.h * R.inv_hs : 0.f;   // the digit planes hold H / hs
        hv.l = on ? hv.l * R.inv_hs : 0.f;
        // balanced digits of h~ on the 2^-34 grid, most significant first:
        // d = rint(r 2^B), r <- r 2^B - d, carried in double-float
        float rh = hv.h * (float)(1 << (GRAM_BITS_ - 1));
        float rl = hv.l * (float)(1 << (GRAM_BITS_ - 1));
#pragma unroll
        for (int p = 0; p < GRAM_PH_; p++) {
            const float d = rint_digit(rh);
            dg[p][i] = d;
            const dfl r = two_sum(rh - d, rl);            // rh - d is exact
            rh = r.h * (float)(1 << GRAM_BITS_);
            rl = r.l * (float)(1 << GRAM_BITS_);
        }
    }
    const int64_t blk = n0 / A.kb;      // n0 .. n0+7 lie in one block
    __nv_bfloat16 *row = A.planes + blk * A.blk_stride + m * A.kb + (n0 - blk * A.kb);
#pragma unroll
    for (int p = 0; p < GRAM_PH_; p++) {
        uint4 v;
        v.x = pack_bf16_int(dg[p][0], dg[p][1]);
        v.y = pack_bf16_int(dg[p][2], dg[p][3]);
        v.z = pack_bf16_int(dg[p][4], dg[p][5]);
        v.w = pack_bf16_int(dg[p][6], dg[p][7]);
        *(uint4 *)(row + (int64_t)p * A.plane_stride) = v;
    }
}

__device__ __forceinline__ void tile_coords(const OzParams &P, int64_t t, int64_t &m0,
                                            int64_t &n0) {
    if (P.gram) {
        // lower tiles in super-blocks (oz_tiles.cuh); ntile_m is the row blocks
        int64_t J, cb;
        gram_tile(t, P.ntile_m, J, cb);
        m0 = J * BM;
        n0 = cb * BN;
    } else {
        m0 = (t % P.ntile_m) * BM;
        n0 = P.n_base + (t / P.ntile_m) * BN;
    }
}

// Work of one CTA: the tiles b, b + G, ... below P.whole over their whole K
// range, then a contiguous share of the remaining tiles' K chunks (tile
// after tile), so the last, partial wave of tiles is spread over every CTA.
// Chunk boundaries keep each piece's running sums exact; the pieces of a
// split tile are added as int64 (order-independent) into P.part.
struct WorkIter {
    int64_t t_next, pos, pos_end;
};
__device__ __forceinline__ WorkIter work_begin(const OzParams &P, int nchunk) {
    WorkIter w;
    const int64_t G = gridDim.x, R = (P.ntiles - P.whole) * nchunk;
    w.t_next = blockIdx.x;
    w.pos = R * (int64_t)blockIdx.x / G;
    w.pos_end = R * ((int64_t)blockIdx.x + 1) / G;
    return w;
}
__device__ __forceinline__ bool work_next(const OzParams &P, int nchunk, WorkIter &w,
                                          int64_t &t, int &c_lo, int &c_hi) {
    if (w.t_next < P.whole) {
        t = w.t_next;
        c_lo = 0;
        c_hi = nchunk;
        w.t_next += gridDim.x;
        return true;
    }
    if (w.pos >= w.pos_end) return false;
    t = P.whole + w.pos / nchunk;
    c_lo = (int)(w.pos % nchunk);
    const int64_t left = w.pos_end - w.pos;
    c_hi = left < nchunk - c_lo ? c_lo + (int)left : nchunk;
    w.pos += c_hi - c_lo;
    return true;
}

// A batched launch: several problems (the same digit scheme, any sizes) in
// one persistent grid.  Unit u in [first[j], first[j+1]) is tile
// u - first[j] of problem j, over its whole K range (no split tiles).  The
// problems' parameters and tensor maps (A then B) sit in global memory; a
// tensor map there must be 64-byte aligned and written before the launch.
struct OzBatch {
    const OzParams *params;   // [nprob]
    const CUtensorMap *maps;  // [2 nprob]
    const int64_t *first;     // [nprob + 1]
    int nprob;                // 0: single-problem launch (the kernel's P, tmA, tmB)
    int *err;
    uint64_t wait_ns;
};

// What one role of the kernel works on next: the unit's parameters, tensor
// maps, tile, chunk range and K extent.
struct Unit {
    const OzParams *P;
    const CUtensorMap *ma, *mb;
    int64_t t;
    int c_lo, c_hi, nslab, nchunk;
};
struct Walk {
    WorkIter wi;   // single problem
    int64_t u;     // batched: next unit of this CTA
};

// Persistent kernel: CTA b processes tiles b, b + G, b + 2G, ... (G = grid
// size) of one problem, or units b, b + G, ... of a batch of problems.  The TMA ring and all barrier phases run on across tiles, so the
// producer prefetches the next tile while the epilogue of the last one runs;
// the epilogue copies its final values out of tensor memory into registers
// and releases it before doing the output arithmetic, so the next tile's
// MMAs overlap that arithmetic.
template <int PA, int PB, int TMAX, int STAGES, int DBITS, int EPI, int TMIN = 2,
          int CHUNK = 0, bool BAT = false>
__global__ void __launch_bounds__(NTHREADS, 1)
ozaki_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const __grid_constant__ OzParams P, const __grid_constant__ OzBatch B) {
    // K stages per exact chunk (CHUNK = 0: four pairs per diagonal)
    constexpr int CHUNK_SLABS = CHUNK ? CHUNK : chunk_slabs<DBITS>();
    constexpr int ND = TMAX - TMIN + 1;          // diagonals t = TMIN..TMAX
    constexpr uint32_t A_BYTES = BM * SK * 2;    // 8 KB per plane
    constexpr uint32_t B_BYTES = BN * SK * 2;    // 4 KB per plane
    constexpr uint32_t STAGE_BYTES = PA * A_BYTES + PB * B_BYTES;
    // columns: ND accumulators, then the low and high 32-bit words of the
    // int64 running sums (used when K spans several chunks)
    constexpr uint32_t LO_COL = ND * BN, HI_COL = ND * BN + BN;
    constexpr uint32_t USED = ND * BN + 2 * BN;
    constexpr uint32_t TMEM_COLS = USED <= 128 ? 128 : (USED <= 256 ? 256 : 512);
    static_assert(USED <= 512, "too many diagonals for tensor memory");

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, mma_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a batched launch (BAT) reads each unit's parameters from global
    // memory; a single launch reads P from the parameter space directly
    constexpr bool batched = BAT;
    // pipeline waits use the caller's bound; the waits that only let this
    // CTA's own copies and MMAs finish before it exits keep WAIT_NS
    const uint64_t wns = batched ? B.wait_ns : P.wait_ns;
    const uint64_t lim = wns ? wns : WAIT_NS;
    // every role walks the same sequence of units
    auto walk_begin = [&]() {
        Walk w;
        w.u = blockIdx.x;
        if (!batched) {
            const int nslab = (int)(P.K / SK);
            w.wi = work_begin(P, (nslab + CHUNK_SLABS - 1) / CHUNK_SLABS);
        }
        return w;
    };
    auto walk_next = [&](Walk &w, Unit &U) {
        if (!batched) {
            U.P = &P;
            U.ma = &tmA;
            U.mb = &tmB;
            U.nslab = (int)(P.K / SK);
            U.nchunk = (U.nslab + CHUNK_SLABS - 1) / CHUNK_SLABS;
            return work_next(P, U.nchunk, w.wi, U.t, U.c_lo, U.c_hi);
        }
        if (w.u >= B.first[B.nprob]) return false;
        int lo = 0, hi = B.nprob - 1;      // the problem holding unit w.u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.first[mid] <= w.u) lo = mid;
            else hi = mid - 1;
        }
        U.P = B.params + lo;
        U.ma = B.maps + 2 * lo;
        U.mb = B.maps + 2 * lo + 1;
        U.t = w.u - B.first[lo];
        U.nslab = (int)(U.P->K / SK);
        U.nchunk = (U.nslab + CHUNK_SLABS - 1) / CHUNK_SLABS;
        U.c_lo = 0;
        U.c_hi = U.nchunk;
        w.u += gridDim.x;
        return true;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, NEPI);
        mbar_init(&mma_done, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_base_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    volatile int *abort = &abort_sh;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- producer
            int64_t g = 0, issued = 0;
            Unit U;
            Walk wk = walk_begin();
            while (!*abort && walk_next(wk, U)) {
                int64_t m0, n0;
                const OzParams &Pp = BAT ? *U.P : P;
                tile_coords(Pp, U.t, m0, n0);
                const int s_hi = U.c_hi * CHUNK_SLABS < U.nslab ? U.c_hi * CHUNK_SLABS : U.nslab;
                const int64_t a_rows = Pp.a_rows, b_rows = Pp.b_rows;
                const int kb = (int)(Pp.kblk ? Pp.kblk : Pp.K);
                for (int s = U.c_lo * CHUNK_SLABS; s < s_hi; s++, g++) {
                    const int st = (int)(g % STAGES);
                    if (g >= STAGES &&
                        !mbar_wait(&empty_bar[st], (uint32_t)(((g / STAGES) - 1) & 1), abort, lim))
                        break;
                    uint8_t *base = smem + (size_t)st * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[st], STAGE_BYTES);
                    const int kz = (s * SK) / kb, kx = s * SK - kz * kb;   // block, offset
#pragma unroll
                    for (int p = 0; p < PA; p++)
                        tma_3d(U.ma, &full_bar[st], base + p * A_BYTES, kx,
                               (int)(p * a_rows + m0), kz);
#pragma unroll
                    for (int q = 0; q < PB; q++)   // digit q + 1, stored in descending order
                        tma_3d(U.mb, &full_bar[st], base + PA * A_BYTES + (PB - 1 - q) * B_BYTES,
                               kx, (int)(q * b_rows + n0), kz);
                    issued = g + 1;
                }
            }
            if (*abort) {
                // let copies already issued land before the CTA exits
                for (int64_t g2 = (issued > STAGES ? issued - STAGES : 0); g2 < issued; g2++) {
                    const uint64_t t0 = gtime();
                    while (!mbar_try(&full_bar[g2 % STAGES], (uint32_t)((g2 / STAGES) & 1)) &&
                           gtime() - t0 < WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issue
            int64_t g = 0, gc = 0;
            Unit U;
            Walk wk = walk_begin();
            while (!*abort && walk_next(wk, U)) {
                const int s_hi = U.c_hi * CHUNK_SLABS < U.nslab ? U.c_hi * CHUNK_SLABS : U.nslab;
                for (int s = U.c_lo * CHUNK_SLABS; s < s_hi && !*abort; s++, g++) {
                    const int st = (int)(g % STAGES);
                    const bool first = (s % CHUNK_SLABS) == 0;
                    // accumulators free again once the previous chunk is read
                    if (first && gc > 0 && !mbar_wait(&acc_empty, (uint32_t)((gc - 1) & 1), abort, lim))
                        break;
                    if (!mbar_wait(&full_bar[st], (uint32_t)((g / STAGES) & 1), abort, lim)) break;
                    tc_fence_after();
                    // one descriptor per stage; planes and K steps are compile-time
                    // offsets in its 16-byte start-address field (smem < 256 KB)
                    const uint64_t da0 = desc_sw64(su32(smem + (size_t)st * STAGE_BYTES));
                    const uint64_t db0 = da0 + (uint64_t)((PA * A_BYTES) >> 4);
                    // A plane p against the B planes q = min(PB, TMAX-p) ..
                    // max(1, TMIN-p) (diagonals t = p + q in TMIN..TMAX) in MMAs of
                    // width up to 256: B planes are stored in descending order and
                    // diagonal t's accumulator sits at column (TMAX - t) BN, so a
                    // group starts at column 0 (and, past four planes, continues at
                    // column 256 with width 64 or 128): A is read once per group
                    // instead of once per pair, and every accumulator address is a
                    // multiple of its MMA width.  p = 1 reaches every diagonal and
                    // comes first, so it alone starts the chunk's accumulators.
                    static_assert(PB >= TMAX - 1 && TMIN >= 2,
                                  "plane 1 must reach every diagonal");
                    static_assert(TMAX - TMIN + 1 <= 8, "at most two MMA groups per plane");
#pragma unroll
                    for (int p = 1; p <= PA && p < TMAX; p++) {
                        const int q_top = PB < TMAX - p ? PB : TMAX - p;
                        const int q_lo = TMIN - p > 1 ? TMIN - p : 1;
#pragma unroll
                        for (int g = 0; q_top - 4 * g >= q_lo; g++) {
                            const int q_hi = q_top - 4 * g;
                            const int nq = q_hi - q_lo + 1 < 4 ? q_hi - q_lo + 1 : 4;
                            const uint32_t col = (uint32_t)((TMAX - p - q_hi) * BN);
                            const uint32_t idesc = IDESC_M | ((uint32_t)((BN * nq) >> 3) << 17);
                            const uint64_t da = da0 + (uint64_t)(((p - 1) * A_BYTES) >> 4);
                            const uint64_t db = db0 + (uint64_t)(((PB - q_hi) * B_BYTES) >> 4);
#pragma unroll
                            for (int kk = 0; kk < SK / 16; kk++) {
                                const uint32_t acc = (first && p == 1 && kk == 0) ? 0u : 1u;
                                mma_bf16(tmem + col, da + 2 * kk, db + 2 * kk, idesc, acc);
                            }
                        }
                    }
                    mma_commit(&empty_bar[st]);
                    if ((s % CHUNK_SLABS) == CHUNK_SLABS - 1 || s == s_hi - 1) {
                        mma_commit(&acc_full);
                        gc++;
                    }
                }
            }
            // every MMA issued so far has completed once this barrier flips;
            // tensor memory is freed only after that
            mma_commit(&mma_done);
            const uint64_t t0 = gtime();
            while (!mbar_try(&mma_done, 0) && gtime() - t0 < WAIT_NS) {
            }
        }
    } else {
        // ------------------------------------------------ drains and epilogue
        const int quarter = warp & 3;
        const int c0 = ((warp - 2) >> 2) * 32;       // this warp's 32 columns of the tile
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
        int64_t gc = 0;
        bool ok = true;
        Unit U;
        Walk wk = walk_begin();
        while (ok && walk_next(wk, U)) {
            // batched mode: the unit's parameters copied once into this
            // thread's own memory, which the epilogue's global stores cannot
            // alias (read through U.P, every field would be reloaded after
            // each store)
            OzParams Pb;
            if (BAT) Pb = *U.P;
            const OzParams &Pu = BAT ? Pb : P;
            const int64_t t = U.t;
            const int c_lo = U.c_lo, c_hi = U.c_hi;
            const bool direct = (EPI != 0) && U.nchunk == 1;
            int64_t m0, n0;
            tile_coords(Pu, t, m0, n0);
            const int64_t m = m0 + quarter * 32 + lane;
            long long run[32];     // EPI == 0: final sums of this warp's 32 columns
            for (int c = c_lo; c < c_hi; c++, gc++) {
                // warp-uniform decision: TMEM loads below are warp-collective
                ok = __all_sync(0xffffffffu, mbar_wait(&acc_full, (uint32_t)(gc & 1), abort, lim));
                if (!ok) break;
                tc_fence_after();
                const bool last = c == c_hi - 1;
                // Each TMEM load is issued before the arithmetic on the previous
                // one (two register buffers), so its latency overlaps that work.
                const auto diag_addr = [&](int k) {   // k = h ND + (t - 2)
                    return lane_base + (uint32_t)((TMAX - TMIN - k % ND) * BN + (k / ND) * 16);
                };
                uint32_t wb[2][16];
                if (direct) {
                    // V = sum_t acc_t 2^(B (TMAX - t)): Horner from the leading
                    // diagonal in double-float, parked in the (otherwise unused)
                    // running-sum columns as (hi, lo) floats
                    dfl V[16];
                    tmem_ld16(diag_addr(0), wb[0]);
                    tmem_wait_ld();
                    reg_fence16(wb[0]);
#pragma unroll
                    for (int k = 0; k < 2 * ND; k++) {
                        if (k + 1 < 2 * ND) tmem_ld16(diag_addr(k + 1), wb[(k + 1) & 1]);
                        const uint32_t *w = wb[k & 1];
                        const float sc = (float)(1 << DBITS);
                        if (k % ND == 0) {
#pragma unroll
                            for (int i = 0; i < 16; i++) V[i] = {__uint_as_float(w[i]), 0.f};
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; i++)
                                V[i] = df_add({V[i].h * sc, V[i].l * sc}, {__uint_as_float(w[i]), 0.f});
                        }
                        if (k % ND == ND - 1) {
                            const int h = k / ND;
                            uint32_t s0[16], s1[16];
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                s0[i] = __float_as_uint(V[i].h);
                                s1[i] = __float_as_uint(V[i].l);
                            }
                            tmem_st16_async(lane_base + LO_COL + h * 16, s0);
                            tmem_st16_async(lane_base + HI_COL + h * 16, s1);
                        }
                        if (k + 1 < 2 * ND) {
                            tmem_wait_ld();
                            reg_fence16(wb[(k + 1) & 1]);
                        }
                    }
                    tmem_wait_st();
                } else {
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        long long *r = run + h * 16;
                        if (c == c_lo) {
#pragma unroll
                            for (int i = 0; i < 16; i++) r[i] = 0;
                        } else {
                            tmem_ld16(lane_base + LO_COL + h * 16, wb[0]);
                            tmem_ld16(lane_base + HI_COL + h * 16, wb[1]);
                            tmem_wait_ld();
                            reg_fence16(wb[0]);
                            reg_fence16(wb[1]);
#pragma unroll
                            for (int i = 0; i < 16; i++)
                                r[i] = (long long)(((unsigned long long)wb[1][i] << 32) | wb[0][i]);
                        }
                        tmem_ld16(diag_addr(h * ND), wb[0]);
                        tmem_wait_ld();
                        reg_fence16(wb[0]);
#pragma unroll
                        for (int td = TMIN; td <= TMAX; td++) {
                            const int k = td - TMIN;
                            if (td < TMAX) tmem_ld16(diag_addr(h * ND + k + 1), wb[(k + 1) & 1]);
                            const uint32_t *w = wb[k & 1];
                            // accumulators are exact integers below 2^25
                            const long long mult = 1ll << (DBITS * (TMAX - td));
#pragma unroll
                            for (int i = 0; i < 16; i++)
                                r[i] += (long long)__float2int_rn(__uint_as_float(w[i])) * mult;
                            if (td < TMAX) {
                                tmem_wait_ld();
                                reg_fence16(wb[(k + 1) & 1]);
                            }
                        }
                        if (!last || EPI != 0) {
                            // the previous stores from these registers have completed
                            tmem_wait_st();
                            uint32_t *w0 = wb[0], *w1 = wb[1];
                            if (last) {
                                // EPI != 0 over several chunks: park V as (hi, lo) floats
#pragma unroll
                                for (int i = 0; i < 16; i++) {
                                    const float vh = __ll2float_rn(r[i]);
                                    w0[i] = __float_as_uint(vh);
                                    w1[i] = __float_as_uint(__ll2float_rn(r[i] - __float2ll_rn(vh)));
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; i++) {
                                    w0[i] = (uint32_t)((unsigned long long)r[i]);
                                    w1[i] = (uint32_t)((unsigned long long)r[i] >> 32);
                                }
                            }
                            tmem_st16_async(lane_base + LO_COL + h * 16, w0);
                            tmem_st16_async(lane_base + HI_COL + h * 16, w1);
                        }
                    }
                    tmem_wait_st();
                }
                tc_fence_before();
                mbar_arrive(&acc_empty);   // MMAs may overwrite the accumulators now
            }
            if (!ok || *abort) break;
            // ---------------------------------------------------- output
            if (EPI == 0 && t >= Pu.whole) {
                // a piece of a split tile (all of it, possibly): exact int64 adds,
                // column-major in the tile so a warp's 32 lanes (rows) hit
                // consecutive addresses; gram_tail_kernel writes the tile
                long long *pt = Pu.part + (t - Pu.whole) * (BM * BN) + (int64_t)c0 * BM +
                                quarter * 32 + lane;
#pragma unroll
                for (int i = 0; i < 32; i++)
                    atomicAdd(reinterpret_cast<unsigned long long *>(pt + i * BM),
                              (unsigned long long)run[i]);
            } else if (EPI == 0) {
                const double unit = ldexp(1.0, -DBITS * (TMAX - 2));
                if (m < Pu.m_valid) {
                    const double rs = Pu.out_scale * unit * Pu.rscale[m];
                    double *out = Pu.out;
                    const int64_t ldo = Pu.ldo, n_valid = Pu.n_valid;
                    const bool gram = Pu.gram != 0, accum = Pu.accumulate != 0;
                    const double *cscale = Pu.cscale;
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const int64_t n = n0 + c0 + i;
                        if (n >= n_valid || (gram && n > m)) continue;
                        double v = (double)run[i] * rs * cscale[n];
                        if (accum) v += out[m * ldo + n];
                        out[m * ldo + n] = v;
                        if (gram && n < m) out[n * ldo + m] = v;   // lanes: consecutive m
                    }
                }
            } else {
                // the running-sum columns are this warp's until its next drain
                const RowAct ra = row_setup(Pu, m);
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    uint32_t w0[16], w1[16];
                    tmem_ld16(lane_base + LO_COL + h * 16, w0);
                    tmem_ld16(lane_base + HI_COL + h * 16, w1);
                    tmem_wait_ld();
                    dfl V[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) V[i] = {__uint_as_float(w0[i]), __uint_as_float(w1[i])};
                    hidden_emit8<EPI == 2>(Pu, ra, m, n0 + c0 + h * 16, V);
                    hidden_emit8<EPI == 2>(Pu, ra, m, n0 + c0 + h * 16 + 8, V + 8);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
    if (threadIdx.x == 0 && *abort) atomicExch(batched ? B.err : P.err, 1);
}

// Split tiles of the Gram: FP64 values from the int64 sums of their pieces,
// with the same expression as the whole-tile epilogue (bitwise the same
// result).  grid = (BM BN / 256, split tiles); element e is column-major.
template <int DBITS, int TMAX>
__global__ void gram_tail_kernel(const OzParams P) {
    const int64_t k = blockIdx.y;
    const int e = blockIdx.x * 256 + threadIdx.x;
    int64_t m0, n0;
    tile_coords(P, P.whole + k, m0, n0);
    const int64_t m = m0 + e % BM, n = n0 + e / BM;
    if (m >= P.m_valid || n >= P.n_valid || (P.gram && n > m)) return;
    const double unit = ldexp(1.0, -DBITS * (TMAX - 2));
    const double rs = P.out_scale * unit * P.rscale[m];
    const double v = (double)P.part[k * (BM * BN) + e] * rs * P.cscale[n];
    P.out[m * P.ldo + n] = v;
    if (P.gram && n < m) P.out[n * P.ldo + m] = v;
}

// ------------------------------------------------------------ digit slicing
// v in [-1, 1] -> PD digits of B bits, v ~= sum_p d_p 2^(-(B-1) - B(p-1)),
// |d_p| <= 2^(B-1); exact FP64 arithmetic, round-to-nearest digits.
template <int PD, int DBITS>
__device__ __forceinline__ void split_digits(double v, float *d) {
    double x = v * (double)(1 << (DBITS - 1));
#pragma unroll
    for (int p = 0; p < PD; p++) {
        double r = rint(x);
        d[p] = (float)r;
        x = (x - r) * (double)(1 << DBITS);
    }
}

// Balanced base-2^B digits of the integer q (|q| <= 2^(B-1+B(PD-1))),
// most significant first: d[0] in [-2^(B-1), 2^(B-1)], the others in
// [-2^(B-1), 2^(B-1)).
template <int PD, int DBITS>
__device__ __forceinline__ void int_digits(long long q, float *d) {
    constexpr long long H = 1ll << (DBITS - 1), M = (1ll << DBITS) - 1;
#pragma unroll
    for (int p = PD - 1; p >= 1; p--) {
        const long long r = ((q + H) & M) - H;
        d[p] = (float)r;
        q = (q - r) >> DBITS;
    }
    d[0] = (float)q;
}

// Smallest power of two 2^e with |v| <= 2^e (1 for v == 0).
__device__ __forceinline__ double pow2_ceil(double v) {
    v = fabs(v);
    if (!(v > 0.0) || !isfinite(v)) return 1.0;
    int e;
    double m = frexp(v, &e);  // v = m 2^e, m in [0.5, 1)
    if (m == 0.5) e -= 1;
    return ldexp(1.0, e);
}

// X (N x n, row stride ldx) -> PD planes of Np x nK bf16 (row i, col k),
// rows scaled by xs[i] = pow2_ceil(max_k |X[i, k]|).  One warp per row.
template <int PD, int DBITS, typename XT>
__global__ void digits_rows_kernel(const XT *__restrict__ X, int64_t N, int64_t n, int64_t ldx,
                                   int64_t Np, int64_t nK, __nv_bfloat16 *__restrict__ planes,
                                   double *__restrict__ xs, float *__restrict__ xsf,
                                   int32_t *__restrict__ nonfinite, int64_t i0, int64_t i1) {
    constexpr int SH = (DBITS - 1) + DBITS * (PD - 1);
    const int64_t i = i0 + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= i1) return;   // rows i0 .. i1-1 (i1 <= Np)
    double mx = 0.0;
    bool bad = false;
    if (i < N)
        for (int64_t k = lane; k < n; k += 32) {
            const double v = (double)X[i * ldx + k];
            bad |= !isfinite(v);
            mx = fmax(mx, fabs(v));
        }
    if (__any_sync(0xffffffffu, bad) && lane == 0 && nonfinite) atomicOr(nonfinite, 1);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double sc = pow2_ceil(mx);
    if (lane == 0) {
        xs[i] = sc;
        xsf[i] = (float)sc;
    }
    const double mul = ldexp(1.0 / sc, SH);  // exact: powers of two
    for (int64_t k = lane; k < nK; k += 32) {
        float d[PD];
        const long long q = (i < N && k < n) ? __double2ll_rn((double)X[i * ldx + k] * mul) : 0;
        int_digits<PD, DBITS>(q, d);
#pragma unroll
        for (int p = 0; p < PD; p++)
            planes[(int64_t)p * Np * nK + i * nK + k] = __float2bfloat16_rn(d[p]);
    }
}

// FP32 X: the same digits from FP32 arithmetic only.  x~ = x / xs[i] is
// exact (power of two); d = rint(64 x~), r = 64 x~ - d is exact, then
// d_p = rint(128 r), r <- 128 r - d_p: every step is exact in FP32 because
// r keeps at most 24 significant bits.  8 consecutive k per thread, one
// 16-byte store per plane.
template <int PD, int DBITS>
__global__ void digits_rows_f32_kernel(const float *__restrict__ X, int64_t N, int64_t n,
                                       int64_t ldx, int64_t Np, int64_t nK,
                                       __nv_bfloat16 *__restrict__ planes,
                                       double *__restrict__ xs, float *__restrict__ xsf,
                                       int32_t *__restrict__ nonfinite, int64_t i0, int64_t i1) {
    const int64_t i = i0 + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= i1) return;   // rows i0 .. i1-1 (i1 <= Np)
    float mx = 0.f;
    bool bad = false;
    if (i < N)
        for (int64_t k = lane; k < n; k += 32) {
            const float v = X[i * ldx + k];
            bad |= !isfinite(v);
            mx = fmaxf(mx, fabsf(v));
        }
    if (__any_sync(0xffffffffu, bad) && lane == 0 && nonfinite) atomicOr(nonfinite, 1);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double sc = pow2_ceil((double)mx);
    if (lane == 0) {
        xs[i] = sc;
        xsf[i] = (float)sc;
    }
    const float inv = (float)(1.0 / sc);
    for (int64_t k0 = (int64_t)lane * 8; k0 < nK; k0 += 256) {
        float d[PD][8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int64_t k = k0 + e;
            float r = (i < N && k < n) ? X[i * ldx + k] * inv * (float)(1 << (DBITS - 1)) : 0.f;
#pragma unroll
            for (int p = 0; p < PD; p++) {
                const float dp = rint_digit(r);
                d[p][e] = dp;
                r = (r - dp) * (float)(1 << DBITS);
            }
        }
#pragma unroll
        for (int p = 0; p < PD; p++) {
            uint4 v;
            v.x = pack_bf16_int(d[p][0], d[p][1]);
            v.y = pack_bf16_int(d[p][2], d[p][3]);
            v.z = pack_bf16_int(d[p][4], d[p][5]);
            v.w = pack_bf16_int(d[p][6], d[p][7]);
            *(uint4 *)(planes + (int64_t)p * Np * nK + i * nK + k0) = v;
        }
    }
}

// Column scales of W: ws[j] = pow2_ceil(max_k |W[k, j]|), 1 for padding.
__global__ void col_scale_kernel(const double *__restrict__ W, int64_t n, int64_t L, int64_t ldw,
                                 int64_t Lp, double *__restrict__ ws) {
    // 32 columns per block, 8 row groups
    __shared__ double red[8][33];
    const int cj = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + cj;
    double mx = 0.0;
    if (j < L)
        for (int64_t k = rg; k < n; k += 8) mx = fmax(mx, fabs(W[k * ldw + j]));
    red[rg][cj] = mx;
    __syncthreads();
    if (rg == 0 && j < Lp) {
        for (int r = 1; r < 8; r++) mx = fmax(mx, red[r][cj]);
        ws[j] = j < L ? pow2_ceil(mx) : 1.0;
    }
}

// W digits, one thread per (j, 8 consecutive k); FP64 value split into a
// double-float pair once, digits from FP32 arithmetic.
template <int PD, int DBITS>
__global__ void digits_cols_par_kernel(const double *__restrict__ W, int64_t n, int64_t L,
                                       int64_t ldw, int64_t Lp, int64_t nK,
                                       __nv_bfloat16 *__restrict__ planes,
                                       const double *__restrict__ ws) {
    const int64_t kb = nK / 8;
    const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e0 >= Lp * kb) return;
    const int64_t j = e0 / kb, k0 = (e0 % kb) * 8;
    const double inv = 1.0 / ws[j];
    float d[PD][8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int64_t k = k0 + e;
        const double v = (j < L && k < n) ? W[k * ldw + j] * inv * (double)(1 << (DBITS - 1)) : 0.0;
        float rh = (float)v;
        float rl = (float)(v - (double)rh);
#pragma unroll
        for (int p = 0; p < PD; p++) {
            const float dp = rint_digit(rh);
            d[p][e] = dp;
            const dfl r = two_sum(rh - dp, rl);   // rh - dp is exact
            rh = r.h * (float)(1 << DBITS);
            rl = r.l * (float)(1 << DBITS);
        }
    }
#pragma unroll
    for (int p = 0; p < PD; p++) {
        uint4 v;
        v.x = pack_bf16_int(d[p][0], d[p][1]);
        v.y = pack_bf16_int(d[p][2], d[p][3]);
        v.z = pack_bf16_int(d[p][4], d[p][5]);
        v.w = pack_bf16_int(d[p][6], d[p][7]);
        *(uint4 *)(planes + (int64_t)p * Lp * nK + j * nK + k0) = v;
    }
}

// Gram row scales: hs[j] = pow2_ceil(a_j) for hidden rows, 1 for padding
// rows, 0 for target rows (filled in by the target slicer).
__global__ void hs_kernel(const double *__restrict__ a, int64_t L, int64_t m, int64_t Lp,
                          double *__restrict__ hs) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Lp) return;
    hs[j] = j < L ? (a ? pow2_ceil(a[j]) : 1.0) : (j < L + m ? 0.0 : 1.0);
}

// Sigmoid table: sigma(z_k) and sigma'(z_k) as double-float pairs.
__global__ void sigmoid_table_kernel(float4 *__restrict__ tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= SIG_N) return;
    const double z = -40.0 + (double)k / 64.0;
    const double s0 = 1.0 / (1.0 + exp(-z));
    const double s1 = s0 * (1.0 - s0);
    const float s0h = (float)s0, s1h = (float)s1;
    tab[k] = make_float4(s0h, (float)(s0 - (double)s0h), s1h, (float)(s1 - (double)s1h));
}

// max_i |T[i, c]| into hs[L + c] (set to 0 by hs_kernel): non-negative
// doubles order like their 64-bit patterns, so an integer atomicMax keeps
// the largest.  Blocks of 32 columns x 8 row phases, grid-strided rows.
__global__ void t_colmax_kernel(const double *__restrict__ T, int64_t ldt, int64_t N, int64_t m,
                                int64_t L, double *__restrict__ hs) {
    __shared__ double red[8][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    double mx = 0.0;
    if (c < m)
        for (int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y; i < N; i += (int64_t)gridDim.y * 8)
            mx = fmax(mx, fabs(T[i * ldt + c]));
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && c < m) {
        for (int y = 1; y < 8; y++) mx = fmax(mx, red[y][threadIdx.x]);
        if (mx > 0.0)
            atomicMax(reinterpret_cast<unsigned long long *>(hs + L + c),
                      (unsigned long long)__double_as_longlong(mx));
    }
}
// T (N x m) -> digit plane rows L + c (column c of T), scaled by
// hs[L + c] = pow2_ceil(max_i |T[i, c]|); thread per sample, grid.y = c.
// Block (0, c) writes the scale back over the maximum; a block that reads
// it afterwards gets the same scale (pow2_ceil is idempotent).
template <int PD, int DBITS>
__global__ void t_digits_kernel(const double *__restrict__ T, int64_t ldt, int64_t N, int64_t L,
                                int64_t Lp, int64_t Np, int64_t kb, __nv_bfloat16 *__restrict__ planes,
                                double *__restrict__ hs) {
    const int64_t c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double sc = pow2_ceil(hs[L + c]);
    __syncthreads();   // every thread of block (0, c) has read before the write-back
    if (blockIdx.x == 0 && threadIdx.x == 0) hs[L + c] = sc;
    if (i >= Np) return;
    float d[PD];
    split_digits<PD, DBITS>(i < N ? T[i * ldt + c] * (1.0 / sc) : 0.0, d);
#pragma unroll
    for (int p = 0; p < PD; p++)
        planes[(i / kb) * PD * Lp * kb + ((int64_t)p * Lp + L + c) * kb + i % kb] =
            __float2bfloat16_rn(d[p]);
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // initialised once, thread-safely (a throwing initialiser is retried)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        ELM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                  cudaEnableDefault, &q));
        if (!p || q != cudaDriverEntryPointSuccess)
            throw ElmError(ELM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// 2-D bf16 map over `rows` x `K` (row-major), box 32 x box_rows, 64-B swizzle.
// 3-D bf16 map over K blocks of kb elements (kb = 0: one block of K):
// [block][rows][kb] row-major, box 32 x box_rows x 1, 64-B swizzle.
CUtensorMap make_map(const __nv_bfloat16 *base, int64_t rows, int64_t K, int box_rows,
                     int64_t kb = 0) {
    if (kb <= 0) kb = K;
    if (((uintptr_t)base & 15) || (kb * 2) % 16 || kb % SK)
        throw ElmError(ELM_ERR_ARG, "digit planes misaligned for TMA");
    CUtensorMap m;
    const int64_t nblk = (K + kb - 1) / kb;
    cuuint64_t dims[3] = {(cuuint64_t)kb, (cuuint64_t)rows, (cuuint64_t)nblk};
    cuuint64_t strides[2] = {(cuuint64_t)(kb * 2), (cuuint64_t)(rows * kb * 2)};
    cuuint32_t box[3] = {(cuuint32_t)SK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)base, dims, strides,
                             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw ElmError(ELM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

int sm_count() {
    static const int sms = [] {
        int dev = 0, n = 0;
        ELM_CUDA(cudaGetDevice(&dev));
        ELM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        return n;
    }();
    return sms;
}

// Dynamic shared memory of an ozaki_kernel instance, set up once per process.
template <int PA, int PB, int TMAX, int STAGES, int DBITS, int EPI, int TMIN = 2, int CHUNK = 0,
          bool BAT = false>
size_t ozaki_smem() {
    constexpr size_t stage = (size_t)PA * BM * SK * 2 + (size_t)PB * BN * SK * 2;
    const size_t smem = STAGES * stage + 1024;
    static const bool attr = [&] {   // once per variant, thread-safely
        ELM_CUDA(cudaFuncSetAttribute(ozaki_kernel<PA, PB, TMAX, STAGES, DBITS, EPI, TMIN, CHUNK, BAT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)attr;
    return smem;
}

template <int PA, int PB, int TMAX, int STAGES, int DBITS, int EPI, int TMIN = 2, int CHUNK = 0>
void launch_ozaki(cudaStream_t s, const __nv_bfloat16 *A, const __nv_bfloat16 *B, OzParams P,
                  int64_t ntiles) {
    const size_t smem = ozaki_smem<PA, PB, TMAX, STAGES, DBITS, EPI, TMIN, CHUNK>();
    auto k = ozaki_kernel<PA, PB, TMAX, STAGES, DBITS, EPI, TMIN, CHUNK>;
    const int sms = sm_count();
    CUtensorMap ma = make_map(A, PA * P.a_rows, P.K, BM, P.kblk);
    CUtensorMap mb = make_map(B, PB * P.b_rows, P.K, BN, P.kblk);
    P.ntiles = ntiles;
    // only the Gram epilogue handles split tiles
    if (EPI != 0 || !P.part || P.whole > ntiles || P.whole < 0) P.whole = ntiles;
    // split tiles spread over every SM; otherwise one CTA per tile at most
    const int64_t grid = (ntiles < sms && P.whole == ntiles) ? ntiles : sms;
    k<<<(unsigned)grid, NTHREADS, smem, s>>>(ma, mb, P, OzBatch{});
    ELM_CHECK_LAUNCH();
}

}  // namespace

CUtensorMap make_map_f64(const double *base, int64_t rows, int64_t cols, int64_t ld, int bx,
                         int by) {
    if (((uintptr_t)base & 15) || (ld * 8) % 16)
        throw ElmError(ELM_ERR_ARG, "matrix misaligned for TMA");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
    cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void *)base, dims, strides,
                             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw ElmError(ELM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

// 3-D bf16 map over digit planes [planes][rows][32] (64-byte rows, 64-B
// swizzle), box 32 x box_rows x box_planes.
CUtensorMap make_map_planes(const __nv_bfloat16 *base, int64_t rows, int planes, int box_rows,
                            int box_planes) {
    if ((uintptr_t)base & 15) throw ElmError(ELM_ERR_ARG, "digit planes misaligned for TMA");
    CUtensorMap m;
    cuuint64_t dims[3] = {(cuuint64_t)SK, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(SK * 2), (cuuint64_t)(rows * SK * 2)};
    cuuint32_t box[3] = {(cuuint32_t)SK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)base, dims, strides,
                             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw ElmError(ELM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

// Digit counts, digit widths and kept pairs (p + q <= TMAX) of the two
// products.  Pre-activation: 6 digits of 7 bits (operand grid 2^-41; one
// exact chunk for up to 1024 inputs).  Gram: 5 digits of 7 bits (H on a
// 2^-34 grid, chunks of 1024 samples).
constexpr int HID_PX = 6, HID_PW = 6, HID_TMAX = 7, HID_BITS = 7;
constexpr int GRAM_PH = GRAM_PH_, GRAM_TMAX = 6, GRAM_BITS = GRAM_BITS_;
// the mixed form's size limits (mixed_limits.h) hold for these schemes
static_assert(HID_PX == HID_PW, "the pair count per diagonal assumes equal digit counts");
static_assert(chunk_slabs<GRAM_BITS>() * SK == MIXED_CHUNK &&
                  chunk_slabs<HID_BITS>() * SK == MIXED_CHUNK,
              "exact chunk length");
static_assert(sums_fit(chunk_bound(GRAM_PH, 2, GRAM_TMAX, GRAM_BITS, MIXED_CHUNK),
                       MIXED_MAX_ROWS, MIXED_CHUNK),
              "Gram running sums exceed int64 within MIXED_MAX_ROWS");
static_assert(sums_fit(chunk_bound(HID_PW, 2, HID_TMAX, HID_BITS, MIXED_CHUNK),
                       MIXED_MAX_INPUTS, MIXED_CHUNK),
              "hidden-layer running sums exceed int64 within MIXED_MAX_INPUTS");

int64_t oz_pad(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

OzHidWs oz_hid_carve(Arena &ar, int64_t N, int64_t n, int64_t L, int64_t m) {
    const int64_t Np = oz_pad(N, BN), nK = oz_pad(n, SK), Lp = oz_pad(L + m, BM);
    OzHidWs w;
    w.xp = ar.take<__nv_bfloat16>(HID_PX * Np * nK);
    w.wp = ar.take<__nv_bfloat16>(HID_PW * Lp * nK);
    w.xs = ar.take<double>(Np);
    w.xsf = ar.take<float>(Np);
    w.ws = ar.take<double>(Lp);
    w.tab = ar.take<float4>(SIG_N);
    w.rowc = ar.take<float4>(2 * Lp);
    return w;
}

// Samples per block of the Gram digit planes.  The planes are stored as
// [block][plane][row][kb]: with one block of all N samples, a row of a plane
// lies N * 2 bytes from the next, and for N of a few hundred thousand the
// Gram kernel's loads of a tile's rows spread over so many pages that it
// slows down by up to 2x (measured: 40000 samples with the rows 320K or 512K
// samples apart, 1.23x and 1.83x the time of the rows 40K apart).
constexpr int64_t GRAM_KBLK = 65536;
int64_t gram_kblk(int64_t Np) { return Np > GRAM_KBLK ? GRAM_KBLK : Np; }

size_t oz_gram_planes_bytes(int64_t N, int64_t L, int64_t m) {
    const int64_t Np = oz_pad(N, BN), kb = gram_kblk(Np), nblk = (Np + kb - 1) / kb;
    return (size_t)nblk * GRAM_PH * oz_pad(L + m, BM) * kb * 2;
}

// H = a g(X W + b) on the tensor cores, emitted directly as the Gram digit
// planes (rows < L and padding rows; target rows are left to oz_t_digits),
// with the row scales hs and, if Ht != NULL, FP64 H^T; the digit slicer of X
// also records a non-finite X in *nonfinite (when given).
void oz_hidden(cudaStream_t s, const OzHidWs &w, const void *X, int xdt, int64_t N, int64_t n,
               int64_t ldx, const double *W, int64_t ldw, const double *b, const double *a,
               int act, int64_t L, int64_t m, __nv_bfloat16 *planes, double *hs, double *Ht,
               int64_t ldh, int *err, void *Hdf, int32_t *nonfinite, const OzRowChunks *chunks,
               uint64_t wait_ns, int stages) {
    const int64_t Np = oz_pad(N, BN), nK = oz_pad(n, SK), Lp = oz_pad(L + m, BM);
    col_scale_kernel<<<(unsigned)((Lp + 31) / 32), 256, 0, s>>>(W, n, L, ldw, Lp, w.ws);
    ELM_CHECK_LAUNCH();
    digits_cols_par_kernel<HID_PW, HID_BITS>
        <<<(unsigned)((Lp * (nK / 8) + 255) / 256), 256, 0, s>>>(W, n, L, ldw, Lp, nK, w.wp, w.ws);
    ELM_CHECK_LAUNCH();
    hs_kernel<<<(unsigned)((Lp + 255) / 256), 256, 0, s>>>(a, L, m, Lp, hs);
    ELM_CHECK_LAUNCH();
    sigmoid_table_kernel<<<(SIG_N + 255) / 256, 256, 0, s>>>(w.tab);
    ELM_CHECK_LAUNCH();
    rowconst_kernel<HID_BITS, HID_TMAX><<<(unsigned)((Lp + 255) / 256), 256, 0, s>>>(
        ldexp(1.0, -2 * (HID_BITS - 1)), w.ws, b, a, hs, L, Lp, w.rowc);
    ELM_CHECK_LAUNCH();
    OzParams P{};
    P.a_rows = Lp;
    P.b_rows = Np;
    P.K = nK;
    P.m_valid = L;
    P.n_valid = N;
    P.ntile_m = Lp / BM;
    P.gram = 0;
    P.out_scale = ldexp(1.0, -2 * (HID_BITS - 1));
    P.rscale = w.ws;
    P.cscale = w.xs;
    P.out = nullptr;
    P.ldo = 0;
    P.err = err;
    P.wait_ns = wait_ns;
    P.ap.b = b;
    P.ap.a = a;
    P.ap.act = act;
    P.ap.L = L;
    P.ap.m = m;
    P.ap.planes = planes;
    P.ap.kb = gram_kblk(Np);
    P.ap.plane_stride = Lp * P.ap.kb;
    P.ap.blk_stride = GRAM_PH * Lp * P.ap.kb;
    P.ap.hs = hs;
    P.ap.tab = w.tab;
    P.ap.csf = w.xsf;
    P.ap.rowc = w.rowc;
    P.ap.Ht = Ht;
    P.ap.Hdf = (float2 *)Hdf;
    P.ap.ldhd = L;
    P.ap.ldh = ldh;
    // the samples in row windows (one window, or the caller's chunks as their
    // copies land): digits of the window's X rows, then its tiles
    const int nc = chunks ? chunks->count : 1;
    for (int c = 0; c < nc; c++) {
        const int64_t r0 = chunks ? chunks->row[c] : 0;
        const int64_t r1 = chunks ? (c + 1 < nc ? chunks->row[c + 1] : Np) : Np;
        if (r1 <= r0) continue;
        if (chunks && chunks->ready[c]) ELM_CUDA(cudaStreamWaitEvent(s, chunks->ready[c], 0));
        const unsigned g = (unsigned)((r1 - r0 + 7) / 8);
        if (xdt == ELM_F64)
            digits_rows_kernel<HID_PX, HID_BITS, double><<<g, 256, 0, s>>>(
                (const double *)X, N, n, ldx, Np, nK, w.xp, w.xs, w.xsf, nonfinite, r0, r1);
        else
            digits_rows_f32_kernel<HID_PX, HID_BITS><<<g, 256, 0, s>>>(
                (const float *)X, N, n, ldx, Np, nK, w.xp, w.xs, w.xsf, nonfinite, r0, r1);
        ELM_CHECK_LAUNCH();
        const int64_t tiles = (Lp / BM) * ((r1 - r0) / BN);
        P.n_base = r0;
        P.whole = tiles;   // no split tiles
        // (two pipeline stages: an autotuner choice; three by default)
        if (Ht)
            launch_ozaki<HID_PW, HID_PX, HID_TMAX, 3, HID_BITS, 2>(s, w.wp, w.xp, P, tiles);
        else if (stages == 2)
            launch_ozaki<HID_PW, HID_PX, HID_TMAX, 2, HID_BITS, 1>(s, w.wp, w.xp, P, tiles);
        else
            launch_ozaki<HID_PW, HID_PX, HID_TMAX, 3, HID_BITS, 1>(s, w.wp, w.xp, P, tiles);
    }
}

// Target rows L .. L+m-1 of the Gram digit planes.
void oz_t_digits(cudaStream_t s, const double *T, int64_t ldt, int64_t N, int64_t L, int64_t m,
                 __nv_bfloat16 *planes, double *hs) {
    if (m <= 0) return;
    const int64_t Np = oz_pad(N, BN), Lp = oz_pad(L + m, BM);
    const int64_t ry = (N + 7) / 8 < 512 ? (N + 7) / 8 : 512;
    t_colmax_kernel<<<dim3((unsigned)((m + 31) / 32), (unsigned)(ry > 0 ? ry : 1)), dim3(32, 8), 0,
                      s>>>(T, ldt, N, m, L, hs);
    ELM_CHECK_LAUNCH();
    t_digits_kernel<GRAM_PH, GRAM_BITS><<<dim3((unsigned)((Np + 255) / 256), (unsigned)m), 256, 0,
                                          s>>>(T, ldt, N, L, Lp, Np, gram_kblk(Np), planes, hs);
    ELM_CHECK_LAUNCH();
}

// G (Lt x Lt FP64, both triangles, Lt = L + m) = Gram of the augmented rows
// [H^T; T^T] from the digit planes.
size_t oz_gram_part_bytes() { return (size_t)sm_count() * BM * BN * sizeof(long long); }

void oz_gram(cudaStream_t s, const __nv_bfloat16 *planes, const double *hs, int64_t N,
             int64_t L, int64_t m, double *G, int64_t ldg, int *err, long long *part,
             uint64_t wait_ns, int stages) {
    const int64_t Np = oz_pad(N, BN), Lp = oz_pad(L + m, BM);
    const int64_t nJ = Lp / BM, ntiles = nJ * (nJ + 1);
    const int64_t sms = sm_count();
    OzParams P{};
    // A last, partial wave of at most half the SMs' worth of tiles is split
    // by K chunks over every CTA.  (Split pieces start at unrelated K
    // offsets and lose the L2 sharing of tiles that stream K in step:
    // measured on a 272-tile Gram, 4x the DRAM reads for a 1.5 % gain.)
    const int64_t tail = ntiles % sms;
    P.whole = (part && tail != 0 && 2 * tail <= sms) ? ntiles - tail : ntiles;
    P.part = part;
    P.a_rows = Lp;
    P.b_rows = Lp;
    P.K = Np;
    P.kblk = gram_kblk(Np);
    P.m_valid = L + m;
    P.n_valid = L + m;
    P.ntile_m = nJ;
    P.gram = 1;
    P.out_scale = ldexp(1.0, -2 * (GRAM_BITS - 1));
    P.rscale = hs;
    P.cscale = hs;
    P.out = G;
    P.ldo = ldg;
    P.err = err;
    P.wait_ns = wait_ns;
    if (P.whole < ntiles)
        ELM_CUDA(cudaMemsetAsync(part, 0, (size_t)(ntiles - P.whole) * BM * BN * sizeof(long long),
                                 s));
    if (stages == 2)
        launch_ozaki<GRAM_PH, GRAM_PH, GRAM_TMAX, 2, GRAM_BITS, 0>(s, planes, planes, P, ntiles);
    else
        launch_ozaki<GRAM_PH, GRAM_PH, GRAM_TMAX, 3, GRAM_BITS, 0>(s, planes, planes, P, ntiles);
    if (P.whole < ntiles) {
        P.ntiles = ntiles;
        gram_tail_kernel<GRAM_BITS, GRAM_TMAX>
            <<<dim3(BM * BN / 256, (unsigned)(ntiles - P.whole)), 256, 0, s>>>(P);
        ELM_CHECK_LAUNCH();
    }
}

// ------------------------------------------------------ FP64-accurate Gram
// [H^T H, H^T T] of an FP64 matrix A = [H^T; T^T] ((L + m) x N, row-major)
// on the tensor cores, as accurate as an FP64 Gram.  Each row is split into
// EX_PH = 8 balanced digits of 7 bits on a 2^-55 grid of its power-of-two
// scale (the FP64 value, rounded once at 2^-56 of the row's maximum), and
// every digit-pair product of weight above 2^-68 (p + q <= 9) is summed
// exactly: diagonals 2..5 (10 pairs, at most four per diagonal, K chunks of
// 1024) in one launch, diagonals 6..9 (26 pairs, at most eight per diagonal,
// K chunks of 512, so every FP32 partial sum stays within 8 * 2^12 * 512 =
// 2^24) in a second launch that adds its FP64 result to the first.  The
// dropped pairs weigh at most 2^-56 relative, the FP64 conversions 2^-53.
constexpr int EX_PH = 8, EX_BITS = 7;
// the two bands below hold their int64 running sums up to EXACT_MAX_K
static_assert(sums_fit(chunk_bound(4, 2, 5, EX_BITS, chunk_slabs<EX_BITS>() * SK), EXACT_MAX_K,
                       chunk_slabs<EX_BITS>() * SK) &&
                  sums_fit(chunk_bound(EX_PH, 6, 9, EX_BITS, 16 * SK), EXACT_MAX_K, 16 * SK),
              "FP64-accurate bands exceed int64 within EXACT_MAX_K");

size_t oz_exact_planes_bytes(int64_t N, int64_t L, int64_t m) {
    return (size_t)EX_PH * oz_pad(L + m, BM) * oz_pad(N, BN) * 2;
}

void oz_gram_exact(cudaStream_t s, const double *A, int64_t lda, int64_t N, int64_t L, int64_t m,
                   __nv_bfloat16 *planes, double *hs, float *hsf, double *G, int64_t ldg, int *err,
                   int32_t *nonfinite, uint64_t wait_ns) {
    const int64_t Np = oz_pad(N, BN), Lp = oz_pad(L + m, BM);
    const int64_t nJ = Lp / BM, ntiles = nJ * (nJ + 1);
    digits_rows_kernel<EX_PH, EX_BITS, double><<<(unsigned)((Lp + 7) / 8), 256, 0, s>>>(
        A, L + m, N, lda, Lp, Np, planes, hs, hsf, nonfinite, 0, Lp);
    ELM_CHECK_LAUNCH();
    OzParams P{};
    P.whole = ntiles;
    P.part = nullptr;
    P.a_rows = Lp;
    P.b_rows = Lp;
    P.K = Np;
    P.m_valid = L + m;
    P.n_valid = L + m;
    P.ntile_m = nJ;
    P.gram = 1;
    P.out_scale = ldexp(1.0, -2 * (EX_BITS - 1));
    P.rscale = hs;
    P.cscale = hs;
    P.out = G;
    P.ldo = ldg;
    P.err = err;
    P.wait_ns = wait_ns;
    P.accumulate = 0;
    launch_ozaki<4, 4, 5, 3, EX_BITS, 0, 2, 0>(s, planes, planes, P, ntiles);
    P.accumulate = 1;
    launch_ozaki<8, 8, 9, 2, EX_BITS, 0, 6, 16>(s, planes, planes, P, ntiles);
}

// ------------------------------------------- FP64-accurate hidden product
// Pre-activations of the FP64 form on the tensor cores: W^T (one row per
// neuron) and X (one row per sample) split like the rows of the exact Gram
// (EX_PH digits of EX_BITS bits on a 2^-55 grid of the row's power-of-two
// scale); the rectangular tile walk of the hidden layer, and the exact
// Gram's two bands of diagonals (2-5, then 6-9 added onto the FP64 sums).
struct OzExactHidWs {
    double *wt;                    // W^T, L x n
    __nv_bfloat16 *wp, *xp;        // digit planes of W^T and X
    double *wsc, *xsc;             // row scales
    float *wscf, *xscf;
};
OzExactHidWs oz_hidden_exact_carve(Arena &ar, int64_t N, int64_t n, int64_t L) {
    const int64_t Np = oz_pad(N, BN), nK = oz_pad(n, SK), Lp = oz_pad(L, BM);
    OzExactHidWs w;
    w.wt = ar.take<double>(L * n);
    w.wp = ar.take<__nv_bfloat16>(EX_PH * Lp * nK);
    w.xp = ar.take<__nv_bfloat16>(EX_PH * Np * nK);
    w.wsc = ar.take<double>(Lp);
    w.xsc = ar.take<double>(Np);
    w.wscf = ar.take<float>(Lp);
    w.xscf = ar.take<float>(Np);
    return w;
}

// ------------------------------------------------------------ batched launch
// The hidden layer and the Gram of several problems as one launch each: the
// slicing kernels run per problem, then one persistent grid walks the tiles
// of every problem (ozaki_kernel with an OzBatch).  Whole tiles only.
namespace {

template <int PA, int PB, int TMAX, int STAGES, int DBITS, int EPI>
void launch_ozaki_batch(cudaStream_t s, const std::vector<OzParams> &ps,
                        const std::vector<CUtensorMap> &maps, const std::vector<int64_t> &first,
                        char *dev, int *err, uint64_t wait_ns) {
    const int64_t count = (int64_t)ps.size();
    const int64_t units = first[count];
    if (units <= 0) return;
    const size_t smem = ozaki_smem<PA, PB, TMAX, STAGES, DBITS, EPI, 2, 0, true>();
    // device copies: maps (64-byte aligned), parameters, unit offsets
    CUtensorMap *dmaps = reinterpret_cast<CUtensorMap *>(dev);
    const size_t mbytes = (sizeof(CUtensorMap) * maps.size() + 255) / 256 * 256;
    OzParams *dps = reinterpret_cast<OzParams *>(dev + mbytes);
    const size_t pbytes = (sizeof(OzParams) * ps.size() + 255) / 256 * 256;
    int64_t *dfirst = reinterpret_cast<int64_t *>(dev + mbytes + pbytes);
    ELM_CUDA(cudaMemcpyAsync(dmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                             cudaMemcpyHostToDevice, s));
    ELM_CUDA(cudaMemcpyAsync(dps, ps.data(), sizeof(OzParams) * ps.size(), cudaMemcpyHostToDevice,
                             s));
    ELM_CUDA(cudaMemcpyAsync(dfirst, first.data(), sizeof(int64_t) * first.size(),
                             cudaMemcpyHostToDevice, s));
    OzBatch B{};
    B.params = dps;
    B.maps = dmaps;
    B.first = dfirst;
    B.nprob = (int)count;
    B.err = err;
    B.wait_ns = wait_ns;
    const int64_t sms = sm_count();
    const int64_t grid = units < sms ? units : sms;
    CUtensorMap none{};
    ozaki_kernel<PA, PB, TMAX, STAGES, DBITS, EPI, 2, 0, true><<<(unsigned)grid, NTHREADS, smem,
                                                                 s>>>(none, none, OzParams{}, B);
    ELM_CHECK_LAUNCH();
}

}  // namespace

size_t oz_hidden_exact_bytes(int64_t N, int64_t n, int64_t L) {
    Arena m;
    oz_hidden_exact_carve(m, N, n, L);
    return m.used;
}

void oz_hidden_exact(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n, int64_t ldx,
                     const double *W, int64_t ldw, int64_t L, char *ws, double *Ht, int64_t ldh,
                     int *err, int32_t *nonfinite, uint64_t wait_ns) {
    if (N <= 0 || L <= 0) return;
    const int64_t Np = oz_pad(N, BN), nK = oz_pad(n, SK), Lp = oz_pad(L, BM);
    Arena ar;
    ar.base = ws;
    ar.cap = oz_hidden_exact_bytes(N, n, L);
    const OzExactHidWs w = oz_hidden_exact_carve(ar, N, n, L);
    transpose_f64(s, W, n, L, ldw, w.wt, n);
    digits_rows_kernel<EX_PH, EX_BITS, double><<<(unsigned)((Lp + 7) / 8), 256, 0, s>>>(
        w.wt, L, n, n, Lp, nK, w.wp, w.wsc, w.wscf, nonfinite, 0, Lp);
    ELM_CHECK_LAUNCH();
    if (xdt == ELM_F64)
        digits_rows_kernel<EX_PH, EX_BITS, double><<<(unsigned)((Np + 7) / 8), 256, 0, s>>>(
            (const double *)X, N, n, ldx, Np, nK, w.xp, w.xsc, w.xscf, nonfinite, 0, Np);
    else
        digits_rows_kernel<EX_PH, EX_BITS, float><<<(unsigned)((Np + 7) / 8), 256, 0, s>>>(
            (const float *)X, N, n, ldx, Np, nK, w.xp, w.xsc, w.xscf, nonfinite, 0, Np);
    ELM_CHECK_LAUNCH();
    const int64_t ntiles = (Lp / BM) * (Np / BN);
    OzParams P{};
    P.whole = ntiles;
    P.part = nullptr;
    P.a_rows = Lp;
    P.b_rows = Np;
    P.K = nK;
    P.m_valid = L;
    P.n_valid = N;
    P.ntile_m = Lp / BM;
    P.n_base = 0;
    P.gram = 0;
    P.out_scale = ldexp(1.0, -2 * (EX_BITS - 1));
    P.rscale = w.wsc;
    P.cscale = w.xsc;
    P.out = Ht;
    P.ldo = ldh;
    P.err = err;
    P.wait_ns = wait_ns;
    P.accumulate = 0;
    launch_ozaki<4, 4, 5, 3, EX_BITS, 0, 2, 0>(s, w.wp, w.xp, P, ntiles);
    P.accumulate = 1;
    launch_ozaki<8, 8, 9, 2, EX_BITS, 0, 6, 16>(s, w.wp, w.xp, P, ntiles);
}

size_t oz_batch_bytes(int64_t count) {
    const size_t mbytes = (sizeof(CUtensorMap) * 2 * count + 255) / 256 * 256;
    const size_t pbytes = (sizeof(OzParams) * count + 255) / 256 * 256;
    const size_t fbytes = (sizeof(int64_t) * (count + 1) + 255) / 256 * 256;
    return 2 * (mbytes + pbytes + fbytes);    // the hidden layer's, then the Gram's
}

void oz_hidden_gram_batch(cudaStream_t s, const OzBatchItem *it, int64_t count, void *dev,
                          int *err, uint64_t wait_ns, cudaEvent_t after_hidden) {
    if (count <= 0) return;
    std::vector<OzParams> ph, pg;
    std::vector<CUtensorMap> mh, mg;
    std::vector<int64_t> fh(1, 0), fg(1, 0);
    for (int64_t i = 0; i < count; i++) {
        const OzBatchItem &q = it[i];
        const int64_t Np = oz_pad(q.N, BN), nK = oz_pad(q.n, SK), Lp = oz_pad(q.L + q.m, BM);
        const OzHidWs &w = q.hw;
        // the slicing and per-row kernels of oz_hidden, whole X at once
        col_scale_kernel<<<(unsigned)((Lp + 31) / 32), 256, 0, s>>>(q.W, q.n, q.L, q.ldw, Lp, w.ws);
        ELM_CHECK_LAUNCH();
        digits_cols_par_kernel<HID_PW, HID_BITS>
            <<<(unsigned)((Lp * (nK / 8) + 255) / 256), 256, 0, s>>>(q.W, q.n, q.L, q.ldw, Lp, nK,
                                                                      w.wp, w.ws);
        ELM_CHECK_LAUNCH();
        hs_kernel<<<(unsigned)((Lp + 255) / 256), 256, 0, s>>>(q.a, q.L, q.m, Lp, q.hs);
        ELM_CHECK_LAUNCH();
        sigmoid_table_kernel<<<(SIG_N + 255) / 256, 256, 0, s>>>(w.tab);
        ELM_CHECK_LAUNCH();
        rowconst_kernel<HID_BITS, HID_TMAX><<<(unsigned)((Lp + 255) / 256), 256, 0, s>>>(
            ldexp(1.0, -2 * (HID_BITS - 1)), w.ws, q.b, q.a, q.hs, q.L, Lp, w.rowc);
        ELM_CHECK_LAUNCH();
        const unsigned g = (unsigned)((Np + 7) / 8);
        if (q.xdt == ELM_F64)
            digits_rows_kernel<HID_PX, HID_BITS, double><<<g, 256, 0, s>>>(
                (const double *)q.X, q.N, q.n, q.ldx, Np, nK, w.xp, w.xs, w.xsf, q.nonfinite, 0,
                Np);
        else
            digits_rows_f32_kernel<HID_PX, HID_BITS><<<g, 256, 0, s>>>(
                (const float *)q.X, q.N, q.n, q.ldx, Np, nK, w.xp, w.xs, w.xsf, q.nonfinite, 0,
                Np);
        ELM_CHECK_LAUNCH();
        OzParams P{};
        P.a_rows = Lp;
        P.b_rows = Np;
        P.K = nK;
        P.m_valid = q.L;
        P.n_valid = q.N;
        P.ntile_m = Lp / BM;
        P.gram = 0;
        P.out_scale = ldexp(1.0, -2 * (HID_BITS - 1));
        P.rscale = w.ws;
        P.cscale = w.xs;
        P.err = err;
        P.wait_ns = wait_ns;
        P.ap.b = q.b;
        P.ap.a = q.a;
        P.ap.act = q.act;
        P.ap.L = q.L;
        P.ap.m = q.m;
        P.ap.planes = q.planes;
        P.ap.kb = gram_kblk(Np);
        P.ap.plane_stride = Lp * P.ap.kb;
        P.ap.blk_stride = GRAM_PH * Lp * P.ap.kb;
        P.ap.hs = q.hs;
        P.ap.tab = w.tab;
        P.ap.csf = w.xsf;
        P.ap.rowc = w.rowc;
        P.ap.Ht = nullptr;
        P.ap.Hdf = (float2 *)q.Hdf;
        P.ap.ldhd = q.L;
        P.ap.ldh = 0;
        const int64_t tiles = (Lp / BM) * (Np / BN);
        P.ntiles = tiles;
        P.whole = tiles;
        P.n_base = 0;
        ph.push_back(P);
        mh.push_back(make_map(w.wp, HID_PW * Lp, nK, BM));
        mh.push_back(make_map(w.xp, HID_PX * Np, nK, BN));
        fh.push_back(fh.back() + tiles);
        // the target rows of the Gram digit planes
        oz_t_digits(s, q.T, q.ldt, q.N, q.L, q.m, q.planes, q.hs);
        // the Gram's parameters
        const int64_t nJ = Lp / BM, gt = nJ * (nJ + 1);
        OzParams G{};
        G.whole = gt;
        G.ntiles = gt;
        G.part = nullptr;
        G.a_rows = Lp;
        G.b_rows = Lp;
        G.K = Np;
        G.kblk = gram_kblk(Np);
        G.m_valid = q.L + q.m;
        G.n_valid = q.L + q.m;
        G.ntile_m = nJ;
        G.gram = 1;
        G.out_scale = ldexp(1.0, -2 * (GRAM_BITS - 1));
        G.rscale = q.hs;
        G.cscale = q.hs;
        G.out = q.G;
        G.ldo = q.ldg;
        G.err = err;
        G.wait_ns = wait_ns;
        pg.push_back(G);
        mg.push_back(make_map(q.planes, GRAM_PH * Lp, Np, BM, G.kblk));
        mg.push_back(make_map(q.planes, GRAM_PH * Lp, Np, BN, G.kblk));
        fg.push_back(fg.back() + gt);
    }
    char *d = (char *)dev;
    const size_t half = oz_batch_bytes(count) / 2;
    launch_ozaki_batch<HID_PW, HID_PX, HID_TMAX, 3, HID_BITS, 1>(s, ph, mh, fh, d, err, wait_ns);
    if (after_hidden) ELM_CUDA(cudaEventRecord(after_hidden, s));
    launch_ozaki_batch<GRAM_PH, GRAM_PH, GRAM_TMAX, 3, GRAM_BITS, 0>(s, pg, mg, fg, d + half, err,
                                                                   wait_ns);
}

}  // namespace elm
