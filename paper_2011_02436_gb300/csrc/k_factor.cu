// Rank-revealing factorisation of the Gram matrix (Eq. 6; Algorithm 1
// steps 3-4) and the triangular solves of the full-rank route to H^+.
//
// Diagonal-pivoted Cholesky of the equilibrated Gram matrix, blocked in
// panels of nb pivots:
//   * the panel runs on one thread-block cluster (8 or 16 CTAs).  Each CTA
//     owns a slice of the active columns and keeps their updated diagonal
//     and the panel rows in shared memory.  Per pivot: every CTA publishes
//     its local argmax, one hardware cluster barrier, every CTA reads the
//     candidates through distributed shared memory and takes the same
//     decision (largest diagonal, ties to the lowest original index).  No
//     spin-waits: the only waits are cluster barriers.
//   * the trailing update A' = A - P^T P (P: the panel rows) runs on the
//     whole GPU and at the same time compacts the active matrix (pivoted
//     columns drop out), so every panel works on a dense (L-k) x (L-k)
//     matrix and no row/column swaps are ever performed.
// Pivot rows are kept in original column order (Rrow) and gathered into
// pivot order, unscaled, at the end.
#include <cooperative_groups.h>
#include <math.h>
#include <type_traits>

#include <stdio.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "df_arith.cuh"
#include "elm_internal.cuh"

namespace cg = cooperative_groups;

namespace elm {

namespace {
using namespace df;

constexpr int FT = 256;       // threads per CTA in the panel / solves
constexpr int MAXNB = 64;     // largest panel width of the data structures
constexpr int PNB = 24;       // largest panel width of the FP64 pivot kernel
// largest panel width of the double-float pivot kernel: a wider panel costs
// each pivot a longer dot product with the pivot column but saves trailing
// passes over the active matrix (factor phase of the sparse-pixel Gram,
// L = 2000: 5.62 / 5.21 / 5.16 / 5.42 ms at widths 16 / 24 / 32 / 48; of the
// rank-deficient one, L = 6000: 41.4 / 36.7 / 35.3 / 35.1 ms)
constexpr int PNB_DF = 32;
constexpr int TSTAGE = 32;    // panel rows staged at a time by the trailing updates
constexpr int MAXCPT = 8;     // panel columns per thread: wmax <= MAXCPT * FT

// Order key of a double as an unsigned integer (larger key = larger value,
// NaN below everything): comparisons then use the integer pipes, not the
// FP64 pipe, which issues about two lanes per clock per SM on GB300.
__device__ __forceinline__ unsigned long long dkey(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) return 0ull;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// 1/sqrt(v) to FP64 accuracy for v > 0 within the float exponent range.
// The seed y0 = rsqrtf(v) (about 22 bits) is formed with integer moves
// instead of FP64 conversions (each FP64 instruction costs one 64-cycle
// issue slot per SM sub-partition on GB300); then one third-order step of
// the iteration for v^{-1/2}:  r = 1 - v y0^2 (exact product: y0 has 24
// significant bits),  y1 = y0 + y0 r (1/2 + 3/8 r), whose truncation error
// is about (5/16) r^3 < 2^-62 relative.
__device__ __forceinline__ double rsqrt64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)(b >> 52) - 1023;                       // v > 0
    const uint32_t fb = ((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
    const unsigned long long db =
        ((unsigned long long)(((yb >> 23) & 0xffu) - 127 + 1023) << 52) |
        ((unsigned long long)(yb & 0x7fffffu) << 29);
    const double y0 = __longlong_as_double((long long)db);
    const double r = fma(-v, y0 * y0, 1.0);
    return fma(y0 * r, fma(0.375, r, 0.5), y0);
}

// 1/sqrt(v), v > 0: float seed y0, then the third-order step
// y0 + y0 r (1/2 + 3/8 r) with r = 1 - v y0^2 formed in double-float
// (y0^2 is exact as a TwoProduct).
__device__ __forceinline__ F2 df_rsqrt(F2 v) {
    const float y0 = rsqrtf(v.h);
    const float q = y0 * y0;
    const float qe = fmaf(y0, y0, -q);
    const F2 r = df_add(F2{1.f, 0.f}, df_neg(df_mul(v, F2{q, qe})));
    const float rr = r.h + r.l;
    return df_renorm(y0, y0 * rr * fmaf(0.375f, rr, 0.5f));
}
// order key of a normalised pair (lexicographic on the float keys of h, l)
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long dfkey(F2 v) {
    if (v.h != v.h) return 0ull;   // NaN below everything
    return ((unsigned long long)fkey(v.h) << 32) | fkey(v.l);
}

// Arithmetic of the pivot panel: FP64, or double-float for the mixed form
// (whose Gram matrix is itself accurate to about 2^-34).  Values travel in
// eight bytes either way.
template <bool DF>
struct PanelArith;
template <>
struct PanelArith<false> {
    using T = double;
    static __device__ __forceinline__ T load(const double *A, int64_t i) { return A[i]; }
    static __device__ __forceinline__ T of(double v) { return v; }
    static __device__ __forceinline__ unsigned long long key(T v) { return dkey(v); }
    static __device__ __forceinline__ T rsqrt(T v) { return rsqrt64(v); }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T scale_diff(T a, T acc, T r) { return (a - acc) * r; }
    static __device__ __forceinline__ T sub_sq(T d, T v) { return fma(-v, v, d); }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ double to_double(T v) { return v; }
};
template <>
struct PanelArith<true> {
    using T = F2;
    static __device__ __forceinline__ T load(const double *A, int64_t i) {
        return reinterpret_cast<const F2 *>(A)[i];
    }
    static __device__ __forceinline__ T of(double v) { return d2df(v); }
    static __device__ __forceinline__ unsigned long long key(T v) { return dfkey(v); }
    static __device__ __forceinline__ T rsqrt(T v) { return df_rsqrt(v); }
    static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
    static __device__ __forceinline__ T scale_diff(T a, T acc, T r) {
        return df_mul(df_add(a, df_neg(acc)), r);
    }
    static __device__ __forceinline__ T sub_sq(T d, T v) {
        float h = d.h, l = d.l;
        df_acc_prod(h, l, v, df_neg(v));
        return df_renorm(h, l);
    }
    static __device__ __forceinline__ T zero() { return F2{0.f, 0.f}; }
    static __device__ __forceinline__ double to_double(T v) { return f2d(v.h) + f2d(v.l); }
};

// Equilibration scales s_j = 1/sqrt(S_jj) (0 if S_jj <= 0), dS = diag(S),
// act = identity, and the factorisation state; one thread per column.
__global__ void equil_scale_kernel(const double *__restrict__ S, int64_t lds, int64_t L,
                                   double *__restrict__ sc, double *__restrict__ dS,
                                   int32_t *__restrict__ act, FactorState *st) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < L) {
        const double dj = S[j * lds + j];
        sc[j] = dj > 0.0 ? 1.0 / sqrt(dj) : 0.0;
        dS[j] = dj;
        act[j] = (int32_t)j;
    }
    if (j == 0) {
        st->k = 0;
        st->Lr = L;
        st->rank = L;
        st->done = 0;
        st->steps = 0;
        st->flags = 0;
        st->stop_val = 0.0;
    }
}
// S -> A = diag(s) S diag(s) (row j = blockIdx.y), as FP64 or double-float
template <bool DF>
__global__ void equil_kernel(const double *__restrict__ S, int64_t lds, int64_t L,
                             const double *__restrict__ sc, double *__restrict__ A, int64_t lda,
                             FactorState *st) {
    const int64_t j = blockIdx.y, l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    if (l < L) {
        const double v = S[j * lds + l];
        bad = !isfinite(v);
        const double a = (v * sc[j]) * sc[l];
        if (DF) reinterpret_cast<F2 *>(A)[j * lda + l] = d2df(a);
        else A[j * lda + l] = a;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->flags, 1);
}

// ------------------------------------------------------------ panel
// A pivot candidate as published to the cluster: the CTA's largest unpivoted
// updated diagonal, its original and active index, and that column's entries
// in the panel rows so far.
struct __align__(16) Slot {
    double val;
    long long idx;        // (orig << 32) | x, x = -1 when the CTA has none
    double pcol[MAXNB];
};
constexpr int MAXCS = 16;
constexpr uint64_t PANEL_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t mapa(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// 8-byte store into a peer's shared memory, counted by that peer's mbarrier
__device__ __forceinline__ void st_async64(uint32_t raddr, uint64_t v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(
                     raddr),
                 "l"(v), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}
// shared memory of this CTA -> shared memory of a peer (cluster addresses
// of the destination and of the peer's mbarrier)
__device__ __forceinline__ void bulk_s2c(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "r"(su32(src)), "r"(bytes), "r"(bar)
        : "memory");
}
// one tile of a 2-D tensor map into this CTA's shared memory
__device__ __forceinline__ void tma2d_g2s(const CUtensorMap *tm, uint64_t *bar, void *dst, int x,
                                          int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"((uint64_t)tm), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (mbar_try(b, parity)) return true;
        if (gtime() - t0 > PANEL_WAIT_NS) return false;
    }
}



// Bytes of one candidate message carrying `t` panel entries, and of one
// exchange.
__device__ __forceinline__ uint32_t msg_bytes(int t) {
    return 16u + 8u * (uint32_t)t;
}
__device__ __forceinline__ uint32_t exch_bytes(int CS, int t) {
    return (uint32_t)CS * msg_bytes(t);
}

// One panel of up to nb pivots on a cluster.  A: active matrix (Lr x Lr,
// full symmetric, lda), act: active -> original index.  Writes the panel
// rows P (active index space, row stride ldp), the pivot rows Rrow (original
// column order), perm, the compaction map rem / act_next and the state.
// Per pivot every CTA sends its local candidate (with the candidate
// column's panel entries) into every peer's shared memory with st.async;
// each CTA waits on its own transaction-counted mbarrier (double-buffered
// slots), so no cluster-wide barrier sits inside the pivot loop.  Waits are
// bounded; on expiry the state's flag bit 1 is set.
template <int CPT, bool DF>
__global__ void __launch_bounds__(FT)
panel_kernel(const double *__restrict__ A, int64_t lda, const int32_t *__restrict__ act,
             double *__restrict__ P, int64_t ldp, double *__restrict__ Rrow, int64_t ldr,
             int32_t *__restrict__ perm, int32_t *__restrict__ rem,
             int32_t *__restrict__ act_next, FactorState *st, int64_t L, int nb,
             int64_t wmax, double tau) {
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int cr = (int)cluster.block_rank();
    __shared__ Slot slots[2][MAXCS];
    __shared__ __align__(8) uint64_t xbar[2];
    __shared__ unsigned long long wred_k[FT / 32];
    __shared__ uint32_t wred_o[FT / 32];
    __shared__ int32_t s_cnt;
    __shared__ int64_t s_off, s_tot;
    __shared__ int s_timeout;
    extern __shared__ double dyn[];

    const FactorState s0 = *st;
    if (s0.done) return;  // uniform over the cluster
    const int64_t Lr = s0.Lr, k0 = s0.k;
    const int64_t Wd = (Lr + CS - 1) / CS;
    const int64_t x0 = (int64_t)cr * Wd;
    const int64_t nloc = x0 < Lr ? (Lr - x0 < Wd ? Lr - x0 : Wd) : 0;
    using AR = PanelArith<DF>;
    using T = typename AR::T;
    T *Ps = reinterpret_cast<T *>(dyn);        // nb x wmax
    T *d = Ps + (int64_t)nb * wmax;            // wmax
    T *Pg = reinterpret_cast<T *>(P);          // panel rows (global)
    T *Rg = reinterpret_cast<T *>(Rrow);       // pivot rows (global)
    int32_t *piv = (int32_t *)(d + wmax);      // wmax
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
        s_timeout = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(&xbar[0], exch_bytes(CS, 0));   // filled by the first exchange
        mbar_expect(&xbar[1], exch_bytes(CS, 1));   // filled after pivot 0
    }
    // this thread's peer (tid mod 16) for the sends: its slot cr and barrier
    uint32_t rslot0[2], rbar0[2];
    for (int b2 = 0; b2 < 2; b2++) {
        const int peer = (int)(threadIdx.x & (MAXCS - 1)) < CS ? (int)(threadIdx.x & (MAXCS - 1)) : 0;
        rslot0[b2] = mapa(su32(&slots[b2][cr]), peer);
        rbar0[b2] = mapa(su32(&xbar[b2]), peer);
    }
    // this thread's columns xl = tid + i FT: diagonal, pivoted flag and
    // original index live in registers (d is mirrored in shared memory for
    // the message of the CTA's candidate)
    T dreg[CPT];
    int32_t areg[CPT];
    bool preg[CPT];
#pragma unroll
    for (int i = 0; i < CPT; i++) {
        const int64_t xl = threadIdx.x + (int64_t)i * FT;
        dreg[i] = AR::zero();
        areg[i] = 0;
        preg[i] = true;
        if (xl < nloc) {
            dreg[i] = AR::load(A, (x0 + xl) * lda + x0 + xl);
            areg[i] = act[x0 + xl];
            preg[i] = false;
            d[xl] = dreg[i];
            piv[xl] = 0;
        }
    }
    cluster.sync();   // every peer's barriers are initialised and armed

    // Candidates travel as (order key of the diagonal, ord = orig << 14 |
    // x): larger key first, equal keys to the lower original index.  Both
    // fit integer registers, so a comparison costs no FP64 issue slot.
    auto pbetter = [](unsigned long long ka, uint32_t oa, unsigned long long kb, uint32_t ob) {
        return ka > kb || (ka == kb && oa < ob);
    };
    // warp-wide best by three hardware reductions: the largest key (high
    // word, then low word among the lanes holding that high word), then
    // the smallest ord among the lanes holding that key
    auto warp_best = [&](unsigned long long &k, uint32_t &o) {
        const uint32_t kh = (uint32_t)(k >> 32), kl = (uint32_t)k;
        const uint32_t mh = __reduce_max_sync(0xffffffffu, kh);
        const uint32_t ml = __reduce_max_sync(0xffffffffu, kh == mh ? kl : 0u);
        const unsigned long long mk = ((unsigned long long)mh << 32) | ml;
        o = __reduce_min_sync(0xffffffffu, k == mk ? o : 0xffffffffu);
        k = mk;
    };
    // send this CTA's best (k, o) -- every thread passes its own -- with
    // the column's first `t` panel entries to every peer's slot `cr` of
    // buffer `buf`
    // (all threads pass their own best)
    auto publish = [&](int t, int buf, unsigned long long k, uint32_t o) {
        warp_best(k, o);
        if (lane == 0) {
            wred_k[warp] = k;
            wred_o[warp] = o;
        }
        __syncthreads();
        k = lane < FT / 32 ? wred_k[lane] : 0ull;
        o = lane < FT / 32 ? wred_o[lane] : 0xffffffffu;
        warp_best(k, o);
        const bool any = k != 0ull;
        const int32_t bx = any ? (int32_t)(o & 0x3fffu) : -1;
        const int64_t xl = any ? bx - x0 : 0;
        // thread (peer = tid mod 16, f = tid / 16 + 16 j): f = 0 value, f = 1
        // index, f >= 2 panel entry f - 2
        const int nf = 2 + t;
        const int peer = threadIdx.x & (MAXCS - 1);
        if (peer >= CS) return;
        const uint32_t rslot = buf ? rslot0[1] : rslot0[0], rbar = buf ? rbar0[1] : rbar0[0];
        for (int f = threadIdx.x >> 4; f < nf; f += FT / MAXCS) {
            uint64_t v;
            if (f == 0) v = any ? *reinterpret_cast<const uint64_t *>(&d[xl]) : 0ull;
            else if (f == 1) v = any ? (((uint64_t)(o >> 14) << 32) | (uint32_t)bx) : ~0ull;
            else v = any ? *reinterpret_cast<const uint64_t *>(&Ps[(int64_t)(f - 2) * Wd + xl]) : 0ull;
            st_async64(rslot + 8 * f, v, rbar);
        }
    };

    {
        unsigned long long k = 0ull;
        uint32_t o = 0xffffffffu;
#pragma unroll
        for (int i = 0; i < CPT; i++) {
            const int64_t xl = threadIdx.x + (int64_t)i * FT;
            if (preg[i]) continue;
            const unsigned long long k2 = AR::key(dreg[i]);
            const uint32_t o2 = ((uint32_t)areg[i] << 14) | (uint32_t)(x0 + xl);
            if (pbetter(k2, o2, k, o)) {
                k = k2;
                o = o2;
            }
        }
        publish(0, 0, k, o);
    }

    const unsigned long long tau_key = AR::key(AR::of(tau));
    const int tmax = (int)(nb < Lr ? nb : Lr);
    int steps = 0;
    bool done = false;
    for (int t = 0; t < tmax; t++) {
        const int buf = t & 1;
        if (!mbar_wait(&xbar[buf], (uint32_t)((t >> 1) & 1))) {
            s_timeout = 1;
            break;
        }
        // every warp reduces the CS candidates itself (no broadcast needed)
        unsigned long long bk = 0ull;
        uint32_t bo = 0xffffffffu;
        if (lane < CS) {
            const Slot &sl = slots[buf][lane];
            const int32_t sx = (int32_t)(sl.idx & 0xffffffff);
            if (sx >= 0) {
                bk = AR::key(*reinterpret_cast<const T *>(&sl.val));
                bo = ((uint32_t)(sl.idx >> 32) << 14) | (uint32_t)sx;
            }
        }
        warp_best(bk, bo);
        if (!(bk > tau_key)) {   // largest remaining diagonal <= tau (or none, or NaN)
            if (cr == 0 && threadIdx.x == 0) {
                double sv = 0.0;
                if (bk != 0ull)
                    sv = AR::to_double(*reinterpret_cast<const T *>(
                        &slots[buf][(int)((int64_t)(bo & 0x3fffu) / Wd)].val));
                st->stop_val = sv;
            }
            done = true;
            break;
        }
        const int64_t q = bo & 0x3fffu;
        const int bi = (int)(q / Wd);
        const T bval = *reinterpret_cast<const T *>(&slots[buf][bi].val);
        const T *ucol = reinterpret_cast<const T *>(slots[buf][bi].pcol);
        const int64_t aq0 = q * lda + x0;
        // this thread's entries of row q first: the load latency overlaps
        // the reciprocal square root
        T aq[CPT];
#pragma unroll
        for (int i = 0; i < CPT; i++) {
            const int64_t xl = threadIdx.x + (int64_t)i * FT;
            aq[i] = xl < nloc ? AR::load(A, aq0 + xl) : AR::zero();
        }
        // only warps that own columns spend FP64 issue slots
        T rinv = AR::zero(), rkk = AR::zero();
        if ((int64_t)(warp * 32) < nloc) {
            rinv = AR::rsqrt(bval);
            rkk = AR::mul(bval, rinv);
        }
        // the pivot column's panel entries, the same for every thread
        T uc[PNB];
        if constexpr (!DF) {
#pragma unroll
            for (int s2 = 0; s2 < PNB; s2++) uc[s2] = s2 < t ? ucol[s2] : AR::zero();
        }
        unsigned long long nk = 0ull;   // best candidate for the next pivot
        uint32_t no = 0xffffffffu;
#pragma unroll
        for (int i = 0; i < CPT; i++) {
            const int64_t xl = threadIdx.x + (int64_t)i * FT;
            if (xl >= nloc) continue;
            const int64_t x = x0 + xl;
            T v;
            if (x == q) {
                v = rkk;
                preg[i] = true;
                piv[xl] = 1;
                perm[k0 + t] = areg[i];
            } else if (preg[i]) {
                v = AR::zero();
            } else {
                T acc;
                if constexpr (DF) {
                    // double-float: short dependent steps, so a plain loop with
                    // its loads unrolled four ahead keeps the FP32 pipe busy
                    float ah = 0.f, al = 0.f;
                    const T *pcol = Ps + xl;
                    int s2 = 0;
                    for (; s2 + 4 <= t; s2 += 4) {
                        const F2 u0 = ucol[s2], u1 = ucol[s2 + 1], u2 = ucol[s2 + 2], u3 = ucol[s2 + 3];
                        const F2 p0 = pcol[(int64_t)s2 * Wd], p1 = pcol[(int64_t)(s2 + 1) * Wd];
                        const F2 p2 = pcol[(int64_t)(s2 + 2) * Wd], p3 = pcol[(int64_t)(s2 + 3) * Wd];
                        df_acc_prod(ah, al, u0, p0);
                        df_acc_prod(ah, al, u1, p1);
                        df_acc_prod(ah, al, u2, p2);
                        df_acc_prod(ah, al, u3, p3);
                    }
                    for (; s2 < t; s2++) df_acc_prod(ah, al, ucol[s2], pcol[(int64_t)s2 * Wd]);
                    acc = df_renorm(ah, al);
                } else {
                    // FP64: each step is a 64-cycle issue slot; load the column's
                    // panel entries first, then run exactly t chained FMAs
                    // (a jump into an unrolled chain: terms t-1 down to 0)
                    T pc[PNB];
#pragma unroll
                    for (int s2 = 0; s2 < PNB; s2++)
                        pc[s2] = s2 < t ? Ps[(int64_t)s2 * Wd + xl] : AR::zero();
                    double a1 = 0.0;
                    auto term = [&](double a2, double b2) { a1 = fma(a2, b2, a1); };
                    switch (t) {
                    case 24: term(uc[23], pc[23]); [[fallthrough]];
                    case 23: term(uc[22], pc[22]); [[fallthrough]];
                    case 22: term(uc[21], pc[21]); [[fallthrough]];
                    case 21: term(uc[20], pc[20]); [[fallthrough]];
                    case 20: term(uc[19], pc[19]); [[fallthrough]];
                    case 19: term(uc[18], pc[18]); [[fallthrough]];
                    case 18: term(uc[17], pc[17]); [[fallthrough]];
                    case 17: term(uc[16], pc[16]); [[fallthrough]];
                    case 16: term(uc[15], pc[15]); [[fallthrough]];
                    case 15: term(uc[14], pc[14]); [[fallthrough]];
                    case 14: term(uc[13], pc[13]); [[fallthrough]];
                    case 13: term(uc[12], pc[12]); [[fallthrough]];
                    case 12: term(uc[11], pc[11]); [[fallthrough]];
                    case 11: term(uc[10], pc[10]); [[fallthrough]];
                    case 10: term(uc[9], pc[9]); [[fallthrough]];
                    case 9: term(uc[8], pc[8]); [[fallthrough]];
                    case 8: term(uc[7], pc[7]); [[fallthrough]];
                    case 7: term(uc[6], pc[6]); [[fallthrough]];
                    case 6: term(uc[5], pc[5]); [[fallthrough]];
                    case 5: term(uc[4], pc[4]); [[fallthrough]];
                    case 4: term(uc[3], pc[3]); [[fallthrough]];
                    case 3: term(uc[2], pc[2]); [[fallthrough]];
                    case 2: term(uc[1], pc[1]); [[fallthrough]];
                    case 1: term(uc[0], pc[0]); [[fallthrough]];
                    default: break;
                    }
                    acc = a1;
                }
                v = AR::scale_diff(aq[i], acc, rinv);
                const T dn = AR::sub_sq(dreg[i], v);
                dreg[i] = dn;
                d[xl] = dn;
                const unsigned long long k2 = AR::key(dn);
                const uint32_t o2 = ((uint32_t)areg[i] << 14) | (uint32_t)x;
                if (pbetter(k2, o2, nk, no)) {
                    nk = k2;
                    no = o2;
                }
            }
            Ps[(int64_t)t * Wd + xl] = v;
            Pg[(int64_t)t * ldp + x] = v;
            Rg[(k0 + t) * ldr + areg[i]] = v;
        }
        __syncthreads();   // this CTA's slice updated; slots[buf] fully read
        // re-arm this buffer for its next use (filled after pivot t + 1) before
        // sending anything that lets a peer get there
        if (threadIdx.x == 0 && t + 2 < tmax) mbar_expect(&xbar[buf], exch_bytes(CS, t + 2));
        steps = t + 1;
        if (t + 1 < tmax) publish(t + 1, buf ^ 1, nk, no);
    }
    if (s_timeout && threadIdx.x == 0) atomicOr(&st->flags, 2);

    // Compaction: unpivoted active columns keep their relative order.
    if (threadIdx.x < 32) {
        int32_t cnt = 0;
        for (int64_t b0 = 0; b0 < nloc; b0 += 32) {
            int64_t xl = b0 + threadIdx.x;
            bool f = xl < nloc && !piv[xl];
            cnt += __popc(__ballot_sync(0xffffffffu, f));
        }
        if (threadIdx.x == 0) s_cnt = cnt;
    }
    cluster.sync();
    if (threadIdx.x == 0) {
        int64_t off = 0, tot = 0;
        for (int c = 0; c < CS; c++) {
            int32_t v = *cluster.map_shared_rank(&s_cnt, c);
            if (c < cr) off += v;
            tot += v;
        }
        s_off = off;
        s_tot = tot;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t pos = s_off;
        for (int64_t b0 = 0; b0 < nloc; b0 += 32) {
            int64_t xl = b0 + threadIdx.x;
            bool f = xl < nloc && !piv[xl];
            unsigned mask = __ballot_sync(0xffffffffu, f);
            if (f) {
                int64_t p = pos + __popc(mask & ((1u << threadIdx.x) - 1u));
                int32_t o = act[x0 + xl];
                rem[p] = (int32_t)(x0 + xl);
                act_next[p] = o;
                if (done) perm[k0 + steps + p] = o;
            }
            pos += __popc(mask);
        }
    }
    if (cr == 0 && threadIdx.x == 0) {
        st->k = k0 + steps;
        st->Lr = s_tot;
        st->steps = steps;
        if (done || k0 + steps >= L) {
            st->done = 1;
            st->rank = k0 + steps;
        }
    }
    cluster.sync();  // keep shared memory alive until every peer has read it
}

// A_next[x', y'] = A[rem x', rem y'] - sum_t P[t, rem x'] P[t, rem y'] on
// lower 32 x 32 tiles, mirrored to the upper triangle.  Small tiles keep
// the grid wide when the active matrix has shrunk to a few hundred rows.
constexpr int TT = 32;
__global__ void __launch_bounds__(256)
trailing_kernel(const double *__restrict__ A, double *__restrict__ An, int64_t lda,
                const double *__restrict__ P, int64_t ldp, const int32_t *__restrict__ rem,
                const FactorState *__restrict__ st) {
    const FactorState s = *st;
    if (s.done) return;
    const int64_t Lr = s.Lr;
    const int steps = (int)s.steps;
    int64_t t = blockIdx.x;
    // lower-triangle tile (J, I) of block t: float estimate, exact integer fix
    int64_t J = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (J * (J + 1) / 2 > t) J--;
    while ((J + 1) * (J + 2) / 2 <= t) J++;
    const int64_t I = t - J * (J + 1) / 2;
    const int64_t r0 = J * TT, c0 = I * TT;
    if (r0 >= Lr) return;
    __shared__ double Pr[TSTAGE][TT + 1];
    __shared__ double Pc[TSTAGE][TT + 1];
    __shared__ int32_t rr_[TT], rc_[TT];
    if (threadIdx.x < TT) {
        int64_t x = r0 + threadIdx.x, y = c0 + threadIdx.x;
        rr_[threadIdx.x] = x < Lr ? rem[x] : -1;
        rc_[threadIdx.x] = y < Lr ? rem[y] : -1;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            int a = rr_[ty + 16 * p], b = rc_[tx + 16 * q];
            acc[p][q] = (a >= 0 && b >= 0) ? A[(int64_t)a * lda + b] : 0.0;
        }
    for (int t0 = 0; t0 < steps; t0 += TSTAGE) {   // panel rows TSTAGE at a time
        const int nt = steps - t0 < TSTAGE ? steps - t0 : TSTAGE;
        if (t0 > 0) __syncthreads();
        for (int e = threadIdx.x; e < TSTAGE * TT; e += 256) {
            int tt = e / TT, k = e % TT;
            Pr[tt][k] = (tt < nt && rr_[k] >= 0) ? P[(int64_t)(t0 + tt) * ldp + rr_[k]] : 0.0;
            Pc[tt][k] = (tt < nt && rc_[k] >= 0) ? P[(int64_t)(t0 + tt) * ldp + rc_[k]] : 0.0;
        }
        __syncthreads();
        for (int tt = 0; tt < nt; tt++) {
            const double u0 = Pr[tt][ty], u1 = Pr[tt][ty + 16];
            const double v0 = Pc[tt][tx], v1 = Pc[tt][tx + 16];
            acc[0][0] = fma(-u0, v0, acc[0][0]);
            acc[0][1] = fma(-u0, v1, acc[0][1]);
            acc[1][0] = fma(-u1, v0, acc[1][0]);
            acc[1][1] = fma(-u1, v1, acc[1][1]);
        }
    }
#pragma unroll
    for (int p = 0; p < 2; p++) {
        int64_t x = r0 + ty + 16 * p;
        if (x >= Lr) continue;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            int64_t y = c0 + tx + 16 * q;
            if (y >= Lr) continue;
            An[x * lda + y] = acc[p][q];
            if (J != I) An[y * lda + x] = acc[p][q];
        }
    }
}

// The same update in the mixed form, on the FP32 pipes: A, An and the
// panel rows hold double-float pairs, and each product P[t, x] P[t, y]
// (TwoProduct by FMA, cross terms included) is subtracted with TwoSum:
// about 2^-44 relative per element, against 24 FP64 FMAs that each take a
// 64-cycle issue slot.
__device__ __forceinline__ void df_sub_prod(float &sh, float &sl, const F2 a, const F2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float s = sh - p;
    const float bb = s - sh;
    const float err = (sh - (s - bb)) + (-p - bb);
    sl = sl + (err - e);
    sh = s;
}
__global__ void __launch_bounds__(256)
trailing_df_kernel(const F2 *__restrict__ A, F2 *__restrict__ An, int64_t lda,
                   const F2 *__restrict__ P, int64_t ldp, const int32_t *__restrict__ rem,
                   const FactorState *__restrict__ st) {
    const FactorState s = *st;
    if (s.done) return;
    const int64_t Lr = s.Lr;
    const int steps = (int)s.steps;
    int64_t t = blockIdx.x;
    // lower-triangle tile (J, I) of block t: float estimate, exact integer fix
    int64_t J = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (J * (J + 1) / 2 > t) J--;
    while ((J + 1) * (J + 2) / 2 <= t) J++;
    const int64_t I = t - J * (J + 1) / 2;
    const int64_t r0 = J * TT, c0 = I * TT;
    if (r0 >= Lr) return;
    __shared__ F2 Pr[TSTAGE][TT + 1];
    __shared__ F2 Pc[TSTAGE][TT + 1];
    __shared__ int32_t rr_[TT], rc_[TT];
    if (threadIdx.x < TT) {
        int64_t x = r0 + threadIdx.x, y = c0 + threadIdx.x;
        rr_[threadIdx.x] = x < Lr ? rem[x] : -1;
        rc_[threadIdx.x] = y < Lr ? rem[y] : -1;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float ah[2][2], al[2][2];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            int a = rr_[ty + 16 * p], b = rc_[tx + 16 * q];
            const F2 v = (a >= 0 && b >= 0) ? A[(int64_t)a * lda + b] : F2{0.f, 0.f};
            ah[p][q] = v.h;
            al[p][q] = v.l;
        }
    for (int t0 = 0; t0 < steps; t0 += TSTAGE) {   // panel rows TSTAGE at a time
        const int nt = steps - t0 < TSTAGE ? steps - t0 : TSTAGE;
        if (t0 > 0) __syncthreads();
        for (int e = threadIdx.x; e < TSTAGE * TT; e += 256) {
            int tt = e / TT, k = e % TT;
            Pr[tt][k] = (tt < nt && rr_[k] >= 0) ? P[(int64_t)(t0 + tt) * ldp + rr_[k]]
                                                 : F2{0.f, 0.f};
            Pc[tt][k] = (tt < nt && rc_[k] >= 0) ? P[(int64_t)(t0 + tt) * ldp + rc_[k]]
                                                 : F2{0.f, 0.f};
        }
        __syncthreads();
        for (int tt = 0; tt < nt; tt++) {
            const F2 u0 = Pr[tt][ty], u1 = Pr[tt][ty + 16];
            const F2 v0 = Pc[tt][tx], v1 = Pc[tt][tx + 16];
            df_sub_prod(ah[0][0], al[0][0], u0, v0);
            df_sub_prod(ah[0][1], al[0][1], u0, v1);
            df_sub_prod(ah[1][0], al[1][0], u1, v0);
            df_sub_prod(ah[1][1], al[1][1], u1, v1);
        }
    }
#pragma unroll
    for (int p = 0; p < 2; p++) {
        int64_t x = r0 + ty + 16 * p;
        if (x >= Lr) continue;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            int64_t y = c0 + tx + 16 * q;
            if (y >= Lr) continue;
            const float sh = ah[p][q] + al[p][q];
            const F2 v{sh, al[p][q] - (sh - ah[p][q])};
            An[x * lda + y] = v;
            if (J != I) An[y * lda + x] = v;
        }
    }
}

// Active columns above which the mixed form's trailing update runs on the
// tensor cores (exact digit slices, one launch pair per panel).
constexpr int64_t TRAIL_TC_MIN = 256;

// R[i, pos] = Rrow[i, perm pos] sqrt(dS[perm pos]) for i < rank, pos >= i;
// Rt = R^T.  32 x 32 tiles transposed through shared memory.
template <bool DF>
__global__ void finalize_kernel(const double *__restrict__ Rrow, int64_t ldrr,
                                const int32_t *__restrict__ perm,
                                const double *__restrict__ dS,
                                const FactorState *__restrict__ st, int64_t L,
                                double *__restrict__ R, double *__restrict__ Rt, int64_t ld) {
    __shared__ double tile[32][33];
    const int64_t r = st->rank;
    const int64_t i0 = (int64_t)blockIdx.y * 32, p0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        int64_t i = i0 + yy, pos = p0 + tx;
        double v = 0.0;
        if (i < r && pos < L && pos >= i) {
            int32_t o = perm[pos];
            double dd = dS[o];
            const double rv = PanelArith<DF>::to_double(
                reinterpret_cast<const typename PanelArith<DF>::T *>(Rrow)[i * ldrr + o]);
            v = rv * (dd > 0.0 ? sqrt(dd) : 0.0);
        }
        if (i < L) R[i * ld + pos] = v;   // columns L .. ld-1: zero padding
        tile[yy][tx] = v;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        int64_t pos = p0 + yy, i = i0 + tx;
        if (pos < L) Rt[pos * ld + i] = tile[tx][yy];
    }
}

// ------------------------------------------------------- triangular solves
// Both directions are one kernel over a "coefficient" matrix C whose row i
// holds the coefficients of x_i in every equation: C = R for R^T x = b
// (top block first), C = R^T for R x = b (bottom block first).  Either way
// the entries one step needs are contiguous row segments of C.
constexpr int TB_ = 32;       // rows per diagonal block

// Inverse U^{-1} of each TB_ x TB_ diagonal block U of the leading r x r
// block of R, zero outside the block's nb x nb part (last block: nb < TB_).
// Stored per block k as DinvF[k][a][c] = U^{-1}[a][c] (for R^T x = b the
// block's equation matrix is U^T, so lane c of a solve reads column c of
// (U^T)^{-1}, i.e. row-major entries [a][c] of U^{-1}) and DinvB[k][a][c] =
// U^{-1}[c][a].  One warp per block; lane c solves U x = e_c by back
// substitution with x in registers.
__global__ void __launch_bounds__(32)
diag_inv_kernel(const double *__restrict__ R, int64_t ldr, int64_t r,
                double *__restrict__ DinvF, double *__restrict__ DinvB) {
    __shared__ double U[TB_][TB_ + 1];
    __shared__ double rd[TB_];
    const int64_t k = blockIdx.x, i0 = k * TB_;
    const int nb = (int)(r - i0 < TB_ ? r - i0 : TB_);
    const int lane = threadIdx.x;
    for (int a = 0; a < TB_; a++)
        U[a][lane] = (a < nb && lane < nb) ? R[(i0 + a) * ldr + i0 + lane] : 0.0;
    __syncwarp();
    rd[lane] = lane < nb ? 1.0 / U[lane][lane] : 0.0;
    __syncwarp();
    double x[TB_];
#pragma unroll
    for (int i = TB_ - 1; i >= 0; i--) {
        double v = (i == lane) ? 1.0 : 0.0;
#pragma unroll
        for (int l = i + 1; l < TB_; l++) v = fma(-U[i][l], x[l], v);
        x[i] = (i < nb && lane < nb) ? v * rd[i] : 0.0;
    }
    double *F = DinvF + k * TB_ * TB_, *Bk = DinvB + k * TB_ * TB_;
#pragma unroll
    for (int i = 0; i < TB_; i++) F[i * TB_ + lane] = x[i];
#pragma unroll
    for (int i = 0; i < TB_; i++) Bk[lane * TB_ + i] = x[i];
}

constexpr int NDG = 4;   // inverse-block buffers (fetched two steps ahead)

constexpr int MAXSLOT = 2 * MAXCS;   // solution slots: two per cluster rank

// shared memory of trsm_kernel in bytes: mbarriers (512 B), then the own
// blocks of B, the solution slots, the partial sums of the split dot
// products, the inverse diagonal blocks and the update slabs
__host__ __device__ constexpr size_t trsm_smem_bytes(int nown, int nsl, int CB) {
    return 512 + 8 * ((size_t)nown * TB_ * CB + (size_t)MAXSLOT * TB_ * CB + 8 * (size_t)TB_ * CB +
                      (size_t)NDG * TB_ * TB_ + 2 * (size_t)nsl * TB_ * TB_);
}

// Blocked triangular solve on one thread-block cluster per group of CB
// right-hand-side columns (Algorithm 1 step 9 through the factor of Eq. 6).
// Diagonal blocks of TB_ rows are dealt round-robin to the CTAs of the
// cluster; each CTA keeps its blocks of B in shared memory.  Step s solves
// block k_s: its owner applies the block's precomputed inverse (all eight
// warps, the 32-term dot products split four ways per SM sub-partition)
// and sends the solution with one bulk copy per peer into that peer's
// slot s mod 2CS, completing on the peer's mbarrier; every CTA then updates
// its remaining rows.  No cluster barrier sits in the loop: a CTA waits
// only for the solution it needs, and the owner of step s+1 first updates
// and solves its own block (look-ahead) before its other rows.  A slot is
// rewritten 2CS steps later: every CTA owns a step among the CS before
// that and sends its solution only after finishing step s, so the new
// data cannot arrive before every receiver has consumed the old.
// The inverse blocks and the slabs of C arrive by bulk copies issued ahead.
// Waits are bounded; on expiry *tflag is set.
template <bool REV, int CB, bool DF = false>
__global__ void __launch_bounds__(FT)
trsm_kernel(const __grid_constant__ CUtensorMap tmC, const double *__restrict__ C, int64_t ldc,
            const double *__restrict__ Dinv, int64_t r, double *__restrict__ B, int64_t ldb,
            int64_t q, int nown, int nsl, int *tflag) {
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int cr = (int)cluster.block_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c0 = (int64_t)(blockIdx.x / CS) * CB;
    const int nc = (int)(q - c0 < CB ? q - c0 : CB);
    const int64_t nblk = (r + TB_ - 1) / TB_;
    constexpr uint32_t XBYTES = TB_ * CB * 8;
    // values of B and of the solution: FP64, or double-float pairs (DF, the
    // mixed form), eight bytes either way; R and the inverse blocks stay FP64
    using V = typename std::conditional<DF, F2, double>::type;
    extern __shared__ __align__(128) unsigned char tsm[];
    uint64_t *bar_sl = (uint64_t *)tsm;                 // 2: slab buffers
    uint64_t *bar_dg = bar_sl + 2;                      // NDG: inverse-block buffers
    uint64_t *bar_x = bar_dg + NDG;                     // MAXSLOT: solution slots
    V *bs = (V *)(tsm + 512);                           // nown x TB_ x CB
    V *xb = bs + (size_t)nown * TB_ * CB;               // MAXSLOT x TB_ x CB
    V *part = xb + (size_t)MAXSLOT * TB_ * CB;          // 8 x TB_ x CB
    const int NS = 2 * CS;                              // slots in use
    double *dg = (double *)(part + 8 * TB_ * CB);       // NDG x TB_ x TB_
    double *sl = dg + (size_t)NDG * TB_ * TB_;          // 2 x nsl x TB_ x TB_
    __shared__ int s_abort;

    auto blk = [&](int64_t s) { return REV ? nblk - 1 - s : s; };
    auto owner_of = [&](int64_t s) { return (int)(blk(s) % CS); };
    auto rows = [&](int64_t k) { return (int)(r - k * TB_ < TB_ ? r - k * TB_ : TB_); };
    // own block k2 takes part in the update of step k
    auto later = [&](int64_t k2, int64_t k) { return k2 < nblk && (REV ? k2 < k : k2 > k); };
    // The slab window holds the nsl own blocks that take part in the most
    // steps: a block is updated by every step before it (R^T x = b) or after
    // it (R x = b), so the last of this CTA's blocks, or the first.
    const int nmine = (int)((nblk - cr + CS - 1) / CS);
    const int wlo = REV ? 0 : (nmine > nsl ? nmine - nsl : 0);
    auto in_win = [&](int kl) { return kl >= wlo && kl < wlo + nsl; };

    // warp 1: inverse block of step s into dg[s % NDG] (if owned; else an
    // empty phase, so every buffer's phase count follows the step count)
    auto fill_diag = [&](int64_t s) {
        if (s >= nblk) return;
        const int64_t k = blk(s);
        const int buf = (int)(s % NDG);
        if (lane == 0) {
            if ((int)(k % CS) == cr) {
                mbar_expect(&bar_dg[buf], TB_ * TB_ * 8);
                bulk_g2s(dg + (size_t)buf * TB_ * TB_, Dinv + k * TB_ * TB_, TB_ * TB_ * 8,
                         &bar_dg[buf]);
            } else {
                mbar_arrive(&bar_dg[buf]);
            }
        }
    };
    // thread 0: the 32 x 32 tiles of C coupling block k_s with the own
    // blocks to update (those inside the window) into sl[s & 1], one
    // tensor-map copy per tile (rows past r read as zero)
    auto fill_slab = [&](int64_t s) {
        if (s >= nblk || threadIdx.x != 0) return;
        const int64_t k = blk(s);
        const int buf = (int)(s & 1);
        int cnt = 0;
        for (int kl = wlo; kl < wlo + nsl; kl++) cnt += later((int64_t)kl * CS + cr, k) ? 1 : 0;
        if (!cnt) {
            mbar_arrive(&bar_sl[buf]);
            return;
        }
        mbar_expect(&bar_sl[buf], (uint32_t)cnt * TB_ * TB_ * 8);
        for (int kl = wlo; kl < wlo + nsl; kl++) {
            const int64_t k2 = (int64_t)kl * CS + cr;
            if (!later(k2, k)) continue;
            tma2d_g2s(&tmC, &bar_sl[buf], sl + ((size_t)buf * nsl + (kl - wlo)) * TB_ * TB_,
                      (int)(k2 * TB_), (int)(k * TB_));
        }
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (!s_abort && !mbar_wait(bar, parity)) s_abort = 1;
    };
    // coefficient of x_{k_s*TB_+a} in equation k2*TB_+jj
    auto coef = [&](int64_t s, int kl, int a, int jj) {
        const int64_t k = blk(s), k2 = (int64_t)kl * CS + cr;
        return in_win(kl) ? sl[(((size_t)(s & 1) * nsl + (kl - wlo)) * TB_ + a) * TB_ + jj]
                          : C[(k * TB_ + a) * ldc + k2 * TB_ + jj];
    };

    // owner of step s: x = Dinv_k b_k with all warps (warp: column warp %
    // CB, a quarter warp / CB of the terms), then send to every peer
    auto solve_send = [&](int64_t s) {
        const int64_t k = blk(s);
        const int slot = (int)(s % NS);
        V *xs = xb + (size_t)slot * TB_ * CB;
        V *xk = bs + (size_t)(k / CS) * TB_ * CB;
        wait(&bar_dg[s % NDG], (uint32_t)((s / NDG) & 1));
        {
            constexpr int NQ = 8 / CB, AQ = TB_ / NQ;
            const int c = warp % CB, qi = warp / CB;
            const double *D = dg + (size_t)(s % NDG) * TB_ * TB_;
            if constexpr (DF) {
                float ph = 0.f, pl = 0.f;
#pragma unroll
                for (int a = qi * AQ; a < qi * AQ + AQ; a++)
                    df_acc_prod(ph, pl, d2df(D[a * TB_ + lane]), xk[a * CB + c]);
                part[(qi * TB_ + lane) * CB + c] = df_renorm(ph, pl);
            } else {
                double p = 0.0;
#pragma unroll
                for (int a = qi * AQ; a < qi * AQ + AQ; a++)
                    p = fma(D[a * TB_ + lane], xk[a * CB + c], p);
                part[(qi * TB_ + lane) * CB + c] = p;
            }
        }
        __syncthreads();
        if (threadIdx.x < TB_ * CB) {
            constexpr int NQ = 8 / CB;
            V v = part[threadIdx.x];
#pragma unroll
            for (int qi = 1; qi < NQ; qi++) {
                if constexpr (DF) v = df_add(v, part[qi * TB_ * CB + threadIdx.x]);
                else v += part[qi * TB_ * CB + threadIdx.x];
            }
            xs[threadIdx.x] = v;
            xk[threadIdx.x] = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (warp == 0 && lane < CS && lane != cr)
            bulk_s2c(mapa(su32(xs), lane), xs, XBYTES, mapa(su32(&bar_x[slot]), lane));
    };
    // own block kl with the solution of step s, terms split over all warps
    auto update_block = [&](int64_t s, const V *xs, int kl) {
        const int nb = rows(blk(s));
        const int64_t j = ((int64_t)kl * CS + cr) * TB_ + lane;
        if constexpr (DF) {
            float ah[CB], al[CB];
#pragma unroll
            for (int c = 0; c < CB; c++) ah[c] = al[c] = 0.f;
#pragma unroll
            for (int a = warp * 4; a < warp * 4 + 4; a++) {
                if (a >= nb) break;
                const F2 rv = d2df(coef(s, kl, a, lane));
#pragma unroll
                for (int c = 0; c < CB; c++) df_acc_prod(ah[c], al[c], rv, xs[a * CB + c]);
            }
#pragma unroll
            for (int c = 0; c < CB; c++) part[(warp * TB_ + lane) * CB + c] = df_renorm(ah[c], al[c]);
        } else {
            double acc[CB];
#pragma unroll
            for (int c = 0; c < CB; c++) acc[c] = 0.0;
#pragma unroll
            for (int a = warp * 4; a < warp * 4 + 4; a++) {
                if (a >= nb) break;
                const double rv = coef(s, kl, a, lane);
#pragma unroll
                for (int c = 0; c < CB; c++) acc[c] = fma(rv, xs[a * CB + c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < CB; c++) part[(warp * TB_ + lane) * CB + c] = acc[c];
        }
        __syncthreads();
        if (threadIdx.x < TB_ * CB && ((int64_t)kl * CS + cr) * TB_ + threadIdx.x / CB < r) {
            V v = part[threadIdx.x];
#pragma unroll
            for (int w = 1; w < 8; w++) {
                if constexpr (DF) v = df_add(v, part[w * TB_ * CB + threadIdx.x]);
                else v += part[w * TB_ * CB + threadIdx.x];
            }
            V &dst = bs[(size_t)kl * TB_ * CB + threadIdx.x];
            if constexpr (DF) dst = df_add(dst, df_neg(v));
            else dst -= v;
        }
        (void)j;
        __syncthreads();
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 + NDG + MAXSLOT; i++) mbar_init(&bar_sl[i], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int64_t e = threadIdx.x; e < (int64_t)nown * TB_ * CB; e += FT) {
        const int kl = (int)(e / (TB_ * CB)), a = (int)((e / CB) % TB_), c = (int)(e % CB);
        const int64_t k = (int64_t)kl * CS + cr, i = k * TB_ + a;
        const double bv = (k < nblk && i < r && c < nc) ? B[i * ldb + c0 + c] : 0.0;
        if constexpr (DF) bs[e] = d2df(bv);
        else bs[e] = bv;
    }
    __syncthreads();
    // arm the receive slots for steps 0 .. 2CS-1, then let peers send
    if (threadIdx.x < NS && threadIdx.x < nblk && owner_of(threadIdx.x) != cr)
        mbar_expect(&bar_x[threadIdx.x], XBYTES);
    cluster.sync();
    if (warp == 1)
        for (int i = 0; i < NDG - 1; i++) fill_diag(i);
    fill_slab(0);
    if (nblk > 0 && owner_of(0) == cr) solve_send(0);

    for (int64_t s = 0; s < nblk; s++) {
        const int64_t k = blk(s);
        const int slot = (int)(s % NS);
        const bool mine = owner_of(s) == cr;
        const V *xs = xb + (size_t)slot * TB_ * CB;
        if (!mine) wait(&bar_x[slot], (uint32_t)((s / NS) & 1));
        wait(&bar_sl[s & 1], (uint32_t)((s >> 1) & 1));
        __syncthreads();
        int skip = -1;
        if (s + 1 < nblk && owner_of(s + 1) == cr) {   // look-ahead
            skip = (int)(blk(s + 1) / CS);
            update_block(s, xs, skip);
            solve_send(s + 1);
        }
        if (!s_abort) {
            const int nb = rows(k);
            for (int e = threadIdx.x; e < nown * TB_; e += FT) {
                const int kl = e / TB_, a2 = e % TB_;
                const int64_t k2 = (int64_t)kl * CS + cr;
                if (kl == skip || k2 * TB_ + a2 >= r || !later(k2, k)) continue;
                V *bb = bs + (size_t)kl * TB_ * CB + (size_t)a2 * CB;
                if constexpr (DF) {
                    // b -= R coefficient * x in double-float (TwoProduct, TwoSum)
                    float ah[CB], al[CB];
#pragma unroll
                    for (int c = 0; c < CB; c++) {
                        ah[c] = bb[c].h;
                        al[c] = bb[c].l;
                    }
                    if (in_win(kl)) {
                        const double *sp = sl + (((size_t)(s & 1) * nsl + (kl - wlo)) * TB_) * TB_ + a2;
#pragma unroll 4
                        for (int a = 0; a < nb; a++) {
                            const F2 rv = d2df(sp[a * TB_]);
#pragma unroll
                            for (int c = 0; c < CB; c++) df_sub_prod(ah[c], al[c], rv, xs[a * CB + c]);
                        }
                    } else {
                        const double *cp = C + k * TB_ * ldc + k2 * TB_ + a2;
#pragma unroll 4
                        for (int a = 0; a < nb; a++) {
                            const F2 rv = d2df(cp[a * ldc]);
#pragma unroll
                            for (int c = 0; c < CB; c++) df_sub_prod(ah[c], al[c], rv, xs[a * CB + c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < CB; c++) bb[c] = df_renorm(ah[c], al[c]);
                } else {
                    double acc[CB];
#pragma unroll
                    for (int c = 0; c < CB; c++) acc[c] = bb[c];
                    if (in_win(kl)) {
                        const double *sp = sl + (((size_t)(s & 1) * nsl + (kl - wlo)) * TB_) * TB_ + a2;
#pragma unroll 8
                        for (int a = 0; a < nb; a++) {
                            const double rv = sp[a * TB_];
#pragma unroll
                            for (int c = 0; c < CB; c++) acc[c] = fma(-rv, xs[a * CB + c], acc[c]);
                        }
                    } else {
                        const double *cp = C + k * TB_ * ldc + k2 * TB_ + a2;
#pragma unroll 4
                        for (int a = 0; a < nb; a++) {
                            const double rv = cp[a * ldc];
#pragma unroll
                            for (int c = 0; c < CB; c++) acc[c] = fma(-rv, xs[a * CB + c], acc[c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < CB; c++) bb[c] = acc[c];
                }
            }
        }
        __syncthreads();   // slot s, slab s read; bs updated
        if (threadIdx.x == 0 && !mine && s + NS < nblk) mbar_expect(&bar_x[slot], XBYTES);
        if (!s_abort) {
            fill_slab(s + 1);
            if (warp == 1) fill_diag(s + NDG - 1);
        }
    }
    cluster.sync();   // every bulk copy between CTAs has landed
    if (s_abort) {
        // give copies from global memory already issued time to land
        // before the shared memory is released
        if (threadIdx.x == 0) {
            atomicOr(tflag, 1);
            const uint64_t t0 = gtime();
            while (gtime() - t0 < 1000000ull) {
            }
        }
        __syncthreads();
        return;
    }
    for (int64_t e = threadIdx.x; e < (int64_t)nown * TB_ * CB; e += FT) {
        const int kl = (int)(e / (TB_ * CB)), a = (int)((e / CB) % TB_), c = (int)(e % CB);
        const int64_t k = (int64_t)kl * CS + cr, i = k * TB_ + a;
        if (k < nblk && i < r && c < nc) {
            if constexpr (DF) B[i * ldb + c0 + c] = f2d(bs[e].h) + f2d(bs[e].l);
            else B[i * ldb + c0 + c] = bs[e];
        }
    }
}

// chosen cluster size (per process; devices are alike); the first caller
// probes under the lock, host threads of batched trainings share the result
std::atomic<int> g_cluster{0};
std::mutex g_cluster_mu;
// largest dynamic shared memory of a panel launch (panel_geometry's budget);
// the kernels' attribute is set to it once, so concurrent launches of
// different sizes never lower it under one another
constexpr size_t PANEL_SMEM_MAX = 200 * 1024 + 64;

int pick_cluster(size_t smem_for16, size_t smem_for8) {
    if (int c = g_cluster.load()) return c;
    std::lock_guard<std::mutex> lk(g_cluster_mu);
    if (int c = g_cluster.load()) return c;
    cudaFuncSetAttribute(panel_kernel<1, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int best = 8;
    for (int cs : {16, 8}) {
        size_t sm = cs == 16 ? smem_for16 : smem_for8;
        cudaFuncSetAttribute(panel_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(FT);
        cfg.dynamicSmemBytes = sm;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, panel_kernel<1, false>, &cfg) == cudaSuccess && n > 0) {
            best = cs;
            break;
        }
        cudaGetLastError();
    }
    g_cluster.store(best);
    return best;
}

void panel_geometry(int64_t L, int cs, int *nb, int64_t *wmax, size_t *smem, int nbmax) {
    *wmax = (L + cs - 1) / cs;
    const size_t budget = 200 * 1024;
    int64_t fit = (int64_t)((budget - (size_t)(*wmax) * 16) / ((size_t)(*wmax) * 8));
    int b = (int)(fit < nbmax ? fit : nbmax);
    if (b < 1) b = 1;
    *nb = b;
    *smem = (size_t)b * (*wmax) * 8 + (size_t)(*wmax) * 16 + 64;
}

}  // namespace

size_t factor_ws_bytes(int64_t L) {
    Arena a;
    factor_ws_carve(a, L);
    return a.used;
}

FactorWs factor_ws_carve(Arena &ar, int64_t L) {
    FactorWs w;
    w.A0 = ar.take<double>(L * L);
    w.A1 = ar.take<double>(L * L);
    w.Rrow = ar.take<double>(L * L);
    w.P = ar.take<double>((int64_t)MAXNB * L);
    w.dS = ar.take<double>(L);
    w.sc = ar.take<double>(L);
    w.act0 = ar.take<int32_t>(L);
    w.act1 = ar.take<int32_t>(L);
    w.rem = ar.take<int32_t>(L);
    w.perm = ar.take<int32_t>(L);
    w.st = ar.take<FactorState>(1);
    w.G = ar.take<__nv_bfloat16>(trail_tc_planes() * trail_tc_rows(L) * 32);
    w.gs = ar.take<float>(trail_tc_rows(L));
    return w;
}

namespace {
using PanelFn = void (*)(const double *, int64_t, const int32_t *, double *, int64_t, double *,
                         int64_t, int32_t *, int32_t *, int32_t *, FactorState *, int64_t, int,
                         int64_t, double);
struct FactorGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
};
std::mutex g_fgraph_mu;
std::map<std::string, FactorGraph> g_fgraph;
void factor_enqueue(cudaStream_t s, const double *S, int64_t lds, int64_t L, double tau,
                    const FactorWs &w, double *R, double *Rt, int64_t ldr, bool df, bool tc64,
                    int cs, int nb, int64_t wmax, size_t smem, PanelFn kpanel);
}  // namespace

void factor_pivoted(cudaStream_t s, const double *S, int64_t lds, int64_t L,
                    double tau, const FactorWs &w, double *R, double *Rt, int64_t ldr, int sms,
                    bool df, int cs_req, int nb_req, bool tc64) {
    tc64 = tc64 && !df;
    if (ldr < tri_ld(L)) throw ElmError(ELM_ERR_ARG, "factor stride below tri_ld(L)");
    if (L > ELM_MAX_L) throw ElmError(ELM_ERR_UNSUPPORTED, "L above ELM_MAX_L");
    int nb16, nb8;
    int64_t w16, w8;
    size_t sm16, sm8;
    const int nbmax = nb_req > 0 ? (nb_req < (df ? MAXNB : PNB) ? nb_req : (df ? MAXNB : PNB))
                                 : (df ? PNB_DF : PNB);
    panel_geometry(L, 16, &nb16, &w16, &sm16, nbmax);
    panel_geometry(L, 8, &nb8, &w8, &sm8, nbmax);
    // Up to 2048 columns (one column per thread on 8 CTAs) the double-float
    // panel exchanges with 7 peers instead of 15: factor phase of the
    // sparse-pixel Gram (L = 2000) 5.03 ms on 8 CTAs against 5.17 on 16; for
    // L = 6000 the 16-CTA cluster is faster (35.2 against 38.3 ms).
    const int cs_max = pick_cluster(sm16, sm8);
    const int cs = cs_req == 8 || (cs_req == 16 && cs_max == 16) ? cs_req
                   : (df && L <= 8 * FT) ? 8 : cs_max;
    int nb;
    int64_t wmax;
    size_t smem;
    panel_geometry(L, cs, &nb, &wmax, &smem, nbmax);
    if (wmax > (int64_t)MAXCPT * FT) throw ElmError(ELM_ERR_UNSUPPORTED, "L too large for the panel");
    // columns per thread, as a compile-time count
    auto kpanel = df ? (wmax <= FT ? panel_kernel<1, true>
                        : wmax <= 2 * FT ? panel_kernel<2, true>
                        : wmax <= 4 * FT ? panel_kernel<4, true> : panel_kernel<8, true>)
                     : (wmax <= FT ? panel_kernel<1, false>
                        : wmax <= 2 * FT ? panel_kernel<2, false>
                        : wmax <= 4 * FT ? panel_kernel<4, false> : panel_kernel<8, false>);
    if (smem > PANEL_SMEM_MAX) throw ElmError(ELM_ERR_UNSUPPORTED, "panel shared memory");
    cudaFuncSetAttribute(kpanel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    ELM_CUDA(cudaFuncSetAttribute(kpanel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)PANEL_SMEM_MAX));

    // The launch sequence depends only on the arguments, so it is captured
    // once into a CUDA graph per argument set and replayed: one graph launch
    // instead of two launches per panel.  (Workspaces are reused between
    // trainings of one shape, so the pointers repeat.)
    char key[320];
    snprintf(key, sizeof key, "%p %ld %ld %a %p %p %p %p %p %p %p %p %p %p %p %p %p %ld %d %d %d %d",
             (const void *)S, (long)lds, (long)L, tau, (void *)w.A0, (void *)w.A1,
             (void *)w.Rrow, (void *)w.P, (void *)w.dS, (void *)w.sc, (void *)w.act0,
             (void *)w.act1, (void *)w.rem, (void *)w.perm, (void *)w.st, (void *)R, (void *)Rt,
             (long)ldr, (int)df, (int)tc64, cs, nb);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ELM_CUDA(cudaStreamIsCapturing(s, &cap));
    bool full = false;
    FactorGraph fg{};
    {
        std::lock_guard<std::mutex> lk(g_fgraph_mu);
        auto it = g_fgraph.find(key);
        if (it != g_fgraph.end()) fg = it->second;
        full = g_fgraph.size() >= 256;   // bounded cache: further shapes run uncaptured
    }
    if (cap == cudaStreamCaptureStatusNone && (fg.exec || !full)) {
        if (fg.exec) {
            ELM_CUDA(cudaGraphLaunch(fg.exec, s));
            count_launches(fg.kernels);
            return;
        }
        // captured on a stream of this thread's own (the caller's may be the
        // legacy default stream, which cannot capture); nothing runs until
        // the graph is launched on the caller's stream
        thread_local struct CaptureStream {
            cudaStream_t s = nullptr;
            ~CaptureStream() {
                if (s) cudaStreamDestroy(s);
            }
        } tls;
        if (!tls.s) ELM_CUDA(cudaStreamCreateWithFlags(&tls.s, cudaStreamNonBlocking));
        const cudaStream_t cs_stream = tls.s;
        ELM_CUDA(cudaStreamBeginCapture(cs_stream, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            factor_enqueue(cs_stream, S, lds, L, tau, w, R, Rt, ldr, df, tc64, cs, nb, wmax, smem,
                           kpanel);
        } catch (...) {
            cudaStreamEndCapture(cs_stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        ELM_CUDA(cudaStreamEndCapture(cs_stream, &graph));
        size_t nodes = 0;
        cudaGraphGetNodes(graph, nullptr, &nodes);
        std::vector<cudaGraphNode_t> nv(nodes);
        if (nodes) cudaGraphGetNodes(graph, nv.data(), &nodes);
        for (auto nd : nv) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                fg.kernels++;
        }
        const cudaError_t ie = cudaGraphInstantiate(&fg.exec, graph, 0);
        cudaGraphDestroy(graph);
        ELM_CUDA(ie);
        {
            std::lock_guard<std::mutex> lk(g_fgraph_mu);
            auto it = g_fgraph.find(key);
            if (it != g_fgraph.end()) {   // another thread captured the same meanwhile
                cudaGraphExecDestroy(fg.exec);
                fg.exec = it->second.exec;
            } else {
                g_fgraph[key] = fg;
            }
        }
        ELM_CUDA(cudaGraphLaunch(fg.exec, s));   // the capture counted its kernels once
        return;
    }
    // inside a caller's capture, or the cache is full: enqueue directly
    factor_enqueue(s, S, lds, L, tau, w, R, Rt, ldr, df, tc64, cs, nb, wmax, smem, kpanel);
}

namespace {

void factor_enqueue(cudaStream_t s, const double *S, int64_t lds, int64_t L, double tau,
                    const FactorWs &w, double *R, double *Rt, int64_t ldr, bool df, bool tc64,
                    int cs, int nb, int64_t wmax, size_t smem, PanelFn kpanel) {
    ELM_CUDA(cudaMemsetAsync(w.st, 0, sizeof(FactorState), s));
    ELM_CUDA(cudaMemsetAsync(w.Rrow, 0, sizeof(double) * L * L, s));
    {
        equil_scale_kernel<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(S, lds, L, w.sc, w.dS,
                                                                       w.act0, w.st);
        ELM_CHECK_LAUNCH();
        const dim3 g((unsigned)((L + 255) / 256), (unsigned)L);
        if (df) equil_kernel<true><<<g, 256, 0, s>>>(S, lds, L, w.sc, w.A0, L, w.st);
        else equil_kernel<false><<<g, 256, 0, s>>>(S, lds, L, w.sc, w.A0, L, w.st);
        ELM_CHECK_LAUNCH();
    }
    const int64_t npanels = (L + nb - 1) / nb;
    for (int64_t p = 0; p < npanels; p++) {
        double *Ac = (p & 1) ? w.A1 : w.A0;
        double *An = (p & 1) ? w.A0 : w.A1;
        int32_t *ac = (p & 1) ? w.act1 : w.act0;
        int32_t *an = (p & 1) ? w.act0 : w.act1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(FT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ELM_CUDA(cudaLaunchKernelEx(&cfg, kpanel, (const double *)Ac, (int64_t)L,
                                    (const int32_t *)ac, w.P, (int64_t)L, w.Rrow, (int64_t)L,
                                    w.perm, w.rem, an, w.st, (int64_t)L, nb, wmax, tau));
        ELM_CHECK_LAUNCH();
        const int64_t Lup = L - (p + 1) * nb;
        if (Lup > 0) {
            int64_t T = (Lup + TT - 1) / TT;
            if ((df || tc64) && Lup > TRAIL_TC_MIN && nb <= TRAIL_TC_K)
                trailing_tc(s, Ac, An, L, w.P, L, w.rem, w.st, w.G, w.gs, trail_tc_rows(L), Lup,
                            /*f64=*/tc64);
            else if (df)
                trailing_df_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
                    (const F2 *)Ac, (F2 *)An, L, (const F2 *)w.P, L, w.rem, w.st);
            else
                trailing_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(Ac, An, L, w.P, L,
                                                                             w.rem, w.st);
            ELM_CHECK_LAUNCH();
        }
    }
    dim3 g((unsigned)(ldr / 32), (unsigned)((L + 31) / 32));
    if (df) finalize_kernel<true><<<g, 256, 0, s>>>(w.Rrow, L, w.perm, w.dS, w.st, L, R, Rt, ldr);
    else finalize_kernel<false><<<g, 256, 0, s>>>(w.Rrow, L, w.perm, w.dS, w.st, L, R, Rt, ldr);
    ELM_CHECK_LAUNCH();
}

}  // namespace

static std::atomic<int> g_tcluster{0};
static std::mutex g_tcluster_mu;
constexpr size_t TRSM_SMEM_MAX = 216 * 1024;   // trsm_launch's budget

template <bool REV, int CB, bool DF = false>
static void trsm_launch(cudaStream_t s, const double *C, int64_t ldc, const double *Dinv,
                        int64_t r, double *B, int64_t ldb, int64_t q, int *tflag) {
    auto k = trsm_kernel<REV, CB, DF>;
    const int64_t nblk = (r + TB_ - 1) / TB_;
    const size_t budget = TRSM_SMEM_MAX;
    int cs = g_tcluster.load() ? g_tcluster.load() : 16;
    for (;;) {
        const int nown = (int)((nblk + cs - 1) / cs);
        // slab window: as many own blocks as fit (all of them up to r of
        // about 10^4); blocks beyond it read C from global memory
        const size_t fixed = trsm_smem_bytes(nown, 0, CB);
        if (fixed > budget) {
            if (cs == 16) {
                cs = 8;
                continue;
            }
            throw ElmError(ELM_ERR_UNSUPPORTED, "rank too large for the cluster solve");
        }
        int nsl = (int)((budget - fixed) / (2 * (size_t)TB_ * TB_ * 8));
        if (nsl > nown) nsl = nown;
        const size_t smem = trsm_smem_bytes(nown, nsl, CB);
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        ELM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TRSM_SMEM_MAX));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(cs * ((q + CB - 1) / CB)));
        cfg.blockDim = dim3(FT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (!g_tcluster.load()) {
            std::lock_guard<std::mutex> lk(g_tcluster_mu);
            if (!g_tcluster.load()) {
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n == 0) {
                    cudaGetLastError();
                    if (cs == 16) {
                        cs = 8;
                        continue;
                    }
                    throw ElmError(ELM_ERR_CUDA, "no cluster configuration for the solve");
                }
                g_tcluster.store(cs);
            } else if (g_tcluster.load() != cs) {
                cs = g_tcluster.load();
                continue;
            }
        }
        const CUtensorMap tmC = make_map_f64(C, r, ldc, ldc, TB_, TB_);
        ELM_CUDA(cudaLaunchKernelEx(&cfg, k, tmC, C, ldc, Dinv, r, B, ldb, q, nown, nsl, tflag));
        ELM_CHECK_LAUNCH();
        return;
    }
}

// Right-hand sides per cluster: spread small counts over several clusters
// (each cluster's 16 SMs issue few FP64 operations per clock).
template <bool REV, bool DF = false>
static void trsm_any(cudaStream_t s, const double *C, int64_t ldc, const double *Dinv, int64_t r,
                     double *B, int64_t ldb, int64_t q, int *tflag) {
    if (r <= 0 || q <= 0) return;
    if (ldc % TB_ != 0 || ldc < ((r + TB_ - 1) / TB_) * TB_)
        throw ElmError(ELM_ERR_ARG, "triangular factor stride must be a multiple of 32");
    if (DF) {   // many right-hand sides only (forming K in the mixed form)
        trsm_launch<REV, 8, DF>(s, C, ldc, Dinv, r, B, ldb, q, tflag);
        return;
    }
    if (q <= 8) trsm_launch<REV, 1>(s, C, ldc, Dinv, r, B, ldb, q, tflag);
    else if (q <= 16) trsm_launch<REV, 2>(s, C, ldc, Dinv, r, B, ldb, q, tflag);
    else if (q <= 64) trsm_launch<REV, 4>(s, C, ldc, Dinv, r, B, ldb, q, tflag);
    else trsm_launch<REV, 8>(s, C, ldc, Dinv, r, B, ldb, q, tflag);
}

int64_t tri_ld(int64_t L) { return ((L + TB_ - 1) / TB_) * TB_; }

int64_t trsm_dinv_doubles(int64_t r) { return ((r + TB_ - 1) / TB_) * TB_ * TB_; }

void trsm_prepare(cudaStream_t s, const double *R, int64_t ldr, int64_t r, double *DinvF,
                  double *DinvB) {
    if (r <= 0) return;
    diag_inv_kernel<<<(unsigned)((r + TB_ - 1) / TB_), 32, 0, s>>>(R, ldr, r, DinvF, DinvB);
    ELM_CHECK_LAUNCH();
}

void trsm_fwd(cudaStream_t s, const double *R, int64_t ldr, const double *DinvF, int64_t r,
              double *B, int64_t ldb, int64_t q, int *tflag) {
    trsm_any<false>(s, R, ldr, DinvF, r, B, ldb, q, tflag);
}

void trsm_bwd(cudaStream_t s, const double *Rt, int64_t ldr, const double *DinvB, int64_t r,
              double *B, int64_t ldb, int64_t q, int *tflag, bool df) {
    if (df) trsm_any<true, true>(s, Rt, ldr, DinvB, r, B, ldb, q, tflag);
    else trsm_any<true>(s, Rt, ldr, DinvB, r, B, ldb, q, tflag);
}

}  // namespace elm
