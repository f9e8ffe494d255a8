// Internal declarations of libelm.so (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "elm.h"
#include "mixed_limits.h"

#define ELM_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            throw ElmError(ELM_ERR_CUDA, std::string(#call) + ": " +           \
                                             cudaGetErrorString(e_));          \
        }                                                                      \
    } while (0)

// Every kernel launch site ends with ELM_CHECK_LAUNCH(), which also counts it.
namespace elm {
void count_launch();
void count_launches(int64_t n);   // kernels of a replayed graph
}
#define ELM_CHECK_LAUNCH()              \
    do {                                \
        elm::count_launch();            \
        ELM_CUDA(cudaGetLastError());   \
    } while (0)

struct ElmError {
    int status;
    std::string msg;
    ElmError(int s, std::string m) : status(s), msg(std::move(m)) {}
};

// Device-side state of one pivoted factorisation (kept in workspace).
struct FactorState {
    int64_t k;        // pivots taken so far
    int64_t Lr;       // active (not yet pivoted) columns
    int64_t rank;     // final rank (valid once done)
    int32_t done;     // 1 once the stopping rule fired or all columns pivoted
    int32_t flags;    // bit 0: non-finite value met; bit 1: a bounded wait expired
    int64_t steps;    // pivots taken by the last panel
    double stop_val;  // largest rejected diagonal (unit-diagonal scale), 0 if none
};

// Bump allocator over the context's device workspace.  With base == nullptr
// it only measures.
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    template <class T>
    T *take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        if (base && used > cap) throw ElmError(ELM_ERR_NOMEM, "workspace overflow");
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

// Launch choices the autotuner times (0: the built-in default).
struct Tune {
    int panel_cs = 0;      // CTAs of a pivot-panel cluster: 8 or 16
    int panel_nb = 0;      // pivots per panel (double-float form up to 64, FP64 up to 24)
    int hid_stages = 0;    // pipeline stages of the mixed hidden-layer tensor kernel: 2 or 3
    int gram_stages = 0;   // pipeline stages of the mixed Gram tensor kernel: 2 or 3
    int lanes = 0;         // batched mixed calls: lanes of the back halves
};

struct elm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    char *ws = nullptr;      // main workspace (planned before launch)
    size_t ws_size = 0;
    char *aux = nullptr;     // solve workspace (sized once the rank is known)
    size_t aux_size = 0;
    char *batch = nullptr;   // mixed form: hidden layers and Grams awaiting their solves
    size_t batch_size = 0;
    std::string last_error;
    // phase timing (ELM_FLAG_PHASE_TIMING)
    bool timing = false;
    cudaEvent_t ev[ELM_NUM_PHASES + 1] = {};
    double phase_ms[ELM_NUM_PHASES] = {};
    // upload of host X in chunks, overlapped with the hidden layer (mixed form)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t xstart = nullptr;
    cudaEvent_t xready[8] = {};
    // batched mixed trainings: sub-contexts (own stream and workspaces) that
    // run problems' factorisations, solves and refinements side by side
    std::vector<elm_ctx *> lanes;
    bool own_stream = false;   // a lane's stream, created and destroyed with it
    // autotuned launch choices by shape bucket (elm_autotune, elm_autotune_load)
    std::map<std::string, Tune> tune;
};

// ---------------------------------------------------------------- kernels
namespace elm {

// FP64 hidden layer: Ht[j, i] = a_j g(sum_k X[i,k] W[k,j] + b_j).
void hidden_f64(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n,
                int64_t ldx, const double *W, int64_t ldw, const double *b,
                const double *a, int64_t L, int act, double *Ht, int64_t ldh);

// Ht[j, i] = a_j g(Ht[j, i] + b_j) in place for j < L, i < N (FP64): the
// activation of pre-activations formed elsewhere.
void act_rows_f64(cudaStream_t s, double *Ht, int64_t ldh, int64_t L, int64_t N, const double *b,
                  const double *a, int act);

// FP64 Gram of the augmented rows [Ht; T^T]: S = H^T H (full, both
// triangles), Z = H^T T.  part: workspace of gram_f64_parts(...) doubles.
int gram_f64_nsplit(int64_t L, int64_t m, int64_t N, int sms);
size_t gram_f64_ws(int64_t L, int64_t m, int nsplit);
void gram_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
              int64_t N, const double *T, int64_t ldt, int64_t m, double *S,
              int64_t lds, double *Z, int64_t ldz, double *part, int nsplit);

// Generic FP64 GEMM: C = alpha * A * B + beta * C with arbitrary element
// strides (so transposes are free).  A is M x K, B is K x N.
void gemm_f64(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t sAm, int64_t sAk, const double *B,
              int64_t sBk, int64_t sBn, double beta, double *C, int64_t ldc);

// Residual R = T - H beta with H given as Ht (L x N); R is N x m (ld m).
void resid_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
               int64_t N, const double *beta, int64_t m, const double *T,
               int64_t ldt, double *R);
// G = H^T R  (L x m) from Ht (L x N) and R (N x m); deterministic split.
size_t htr_f64_ws(int64_t L, int64_t m, int nsplit);
int htr_f64_nsplit(int64_t L, int64_t N, int sms);
void htr_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
             int64_t N, const double *R, int64_t m, double *G, double *part,
             int nsplit);

// The refinement products of the mixed form with H (N x L, sample-major)
// held as double-float pairs: Rd = T - H beta (N x m pairs; betaT scratch of
// L x min(m, 32) pairs) and G = H^T Rd (L x m) through
// htr_df_nsplit(L, N, sms) x L x m doubles of partial sums; double-float
// arithmetic, targets in passes of up to 32.
void resid_df(cudaStream_t s, const void *H, int64_t L, int64_t N, const double *beta,
              int64_t m, const double *T, int64_t ldt, void *Rd, void *betaT);
int htr_df_nsplit(int64_t L, int64_t N, int sms);
void htr_df(cudaStream_t s, const void *H, int64_t L, int64_t N, const void *Rd, int64_t m,
            double *G, double *part, int nsplit);

// Fused prediction Y = g(X W + b) beta (FP64).
void predict_f64(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n,
                 int64_t ldx, const double *W, int64_t ldw, const double *b,
                 const double *a, int64_t L, int act, const double *beta,
                 int64_t ldb, int64_t m, double *Y, int64_t ldy);

// ------------------------------------------------ factorisation and solves
struct FactorWs {
    double *A0, *A1;       // L x L ping-pong active matrices
    double *Rrow;          // L x L pivot rows in original column order
    double *P;             // nb x L panel rows (active index space)
    double *dS;            // L diagonal of S
    double *sc;            // L equilibration scales 1/sqrt(S_jj)
    int32_t *act0, *act1;  // active -> original index maps
    int32_t *rem;          // compaction map of the last panel
    int32_t *perm;         // pivot order
    FactorState *st;
    __nv_bfloat16 *G;      // digit planes of the panel rows (tensor-core trailing update)
    float *gs;             // their per-column power-of-two scales
};
size_t factor_ws_bytes(int64_t L);
FactorWs factor_ws_carve(Arena &ar, int64_t L);
// Row stride of the triangular factors: L rounded up to a multiple of 32,
// so every 32-column row segment of a 32 x 32 block is 16-byte aligned and
// inside the row (the solves fetch them with bulk copies).
int64_t tri_ld(int64_t L);
// Pivoted Cholesky of the L x L matrix S (lds).  Writes R (L rows, stride
// ldr >= tri_ld(L), pivot order, unscaled, zero below the diagonal, in rows
// >= rank and in the padding columns) and Rt = R^T (same shape), perm.
// The rank lives in w.st->rank (device).  df: keep the active matrix as
// double-float pairs, run the panels on the FP32 pipes and the trailing
// updates on the tensor cores from exact digit slices (about 2^-44 relative
// per update; for the mixed form, whose Gram matrix is itself accurate to
// about 2^-34), else FP64 throughout.
// cs, nb: cluster size (8 or 16) and panel width of the pivot panels
// (0: the built-in choice; nb is capped at the form's largest width).
// tc64 (FP64 panels only): the trailing updates on the tensor cores from
// exact seven-digit slices (FP64-level accuracy; the FP64 form with
// tensor-core products).
void factor_pivoted(cudaStream_t s, const double *S, int64_t lds, int64_t L,
                    double tau, const FactorWs &w, double *R, double *Rt, int64_t ldr,
                    int sms, bool df = false, int cs = 0, int nb = 0, bool tc64 = false);

// Trailing update on the tensor cores: after a panel (st->steps pivots,
// st->Lr columns left, compaction map rem) An[x, y] = A[rem x, rem y] -
// sum_t P[t, rem x] P[t, rem y], from exact 8-bit digit slices of the panel
// rows: double-float pairs in six digits (the mixed form), or FP64 values in
// seven digits with an exact integer fold (f64; FP64-level accuracy).  G:
// trail_tc_planes() planes of trail_tc_rows(L) rows x 32, gs:
// trail_tc_rows(L) scales.  Lup: an upper bound of st->Lr.  Panels of up to
// TRAIL_TC_K pivots (one K block of the digit planes).
constexpr int TRAIL_TC_K = 32;
int64_t trail_tc_rows(int64_t L);
int trail_tc_planes();
void trailing_tc(cudaStream_t s, const double *A, double *An, int64_t lda, const double *P,
                 int64_t ldp, const int32_t *rem, FactorState *st, __nv_bfloat16 *G, float *gs,
                 int64_t Lcap, int64_t Lup, bool f64);

// K = R11^{-1} B in place for the mixed form (B: r x q FP64, row stride ldb;
// R: upper-triangular factor, row stride ldr; DinvF: the inverses of its
// 32 x 32 diagonal blocks from trsm_prepare), by 32-row blocks whose updates
// of the rows above run on the tensor cores from exact 8-bit digit slices
// (double-float accurate).  ws: ksolve_tc_bytes(r, q) bytes; *flag |= 1 when
// a bounded device-side wait gives up.
size_t ksolve_tc_bytes(int64_t r, int64_t q);
void ksolve_tc(cudaStream_t s, const double *R, int64_t ldr, const double *DinvF, int64_t r,
               double *B, int64_t ldb, int64_t q, void *ws, int *flag);

// Solves with the leading r x r block R11 of such a factor.  trsm_prepare
// inverts its 32 x 32 diagonal blocks (DinvF, DinvB: trsm_dinv_doubles(r)
// each); trsm_fwd then overwrites B (r x q, ldb) with R11^{-T} B reading R,
// trsm_bwd with R11^{-1} B reading Rt.  *tflag |= 1 when a bounded
// device-side wait gives up.
int64_t trsm_dinv_doubles(int64_t r);
void trsm_prepare(cudaStream_t s, const double *R, int64_t ldr, int64_t r, double *DinvF,
                  double *DinvB);
void trsm_fwd(cudaStream_t s, const double *R, int64_t ldr, const double *DinvF, int64_t r,
              double *B, int64_t ldb, int64_t q, int *tflag);
// df: double-float arithmetic on the FP32 pipes (about 2^-44 per operation;
// for the mixed form, whose factor is itself double-float accurate).
void trsm_bwd(cudaStream_t s, const double *Rt, int64_t ldr, const double *DinvB, int64_t r,
              double *B, int64_t ldb, int64_t q, int *tflag, bool df = false);

// Gather rows: dst[i, :] = src[perm[i], :] for i < r_dev.
void gather_rows(cudaStream_t s, const double *src, int64_t lds, const int32_t *perm,
                 const int64_t *r_dev, int64_t rmax, int64_t m, double *dst, int64_t ldd);
// Scatter: beta[perm[i], :] = src[i, :] for i < L (ld of src m).
void scatter_rows(cudaStream_t s, const double *src, int64_t m, const int32_t *perm,
                  int64_t L, double *beta, int64_t ldb, double alpha, int accumulate);

// Norm helpers: out[0] = ||x||_F^2 over rows x cols.
void sumsq(cudaStream_t s, const double *x, int64_t rows, int64_t cols, int64_t ld,
           double *out);
// beta += dB; out[0] = ||dB||^2, out[1] = ||beta||^2.
void axpy_norms(cudaStream_t s, double *beta, const double *dB, int64_t count, double *out);
// A (n x n) = I.
void set_identity(cudaStream_t s, double *A, int64_t n);
// A[i, i] += 1, i < n
void add_identity(cudaStream_t s, double *A, int64_t n, int64_t lda);
// B (cols x rows, ldb) = A^T for A (rows x cols, lda).
void transpose_f64(cudaStream_t s, const double *A, int64_t rows, int64_t cols, int64_t lda,
                   double *B, int64_t ldb);
// C (q x q, both triangles) = I + A^T A for A (k x q, row-major, lda) in
// FP64; part: syrk_f64_ws(q, S) doubles, S = syrk_f64_splits(k, q, sms)
// pieces of the k range summed in a fixed order.
// Skinny FP64 products with a tall A (k x q, row-major, lda) and m columns
// (memory-bound on A, read once): out (q x m, contiguous) = A^T Y with Y
// (k x m, contiguous), split over the rows into S = atv_splits(k, q, sms)
// pieces summed in order (part: S q m doubles); Y (k x m) -= A V.
int atv_splits(int64_t k, int64_t q, int sms);
void atv_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda, const double *Y,
             int64_t m, double *out, double *part, int S);
void av_sub_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda,
                const double *V, int64_t m, double *Y);
int syrk_f64_splits(int64_t k, int64_t q, int sms);
size_t syrk_f64_ws(int64_t q, int S);
void syrk_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda, double *C,
              int64_t ldc, double *part, int S);
// Scan for non-finite entries; sets *flag = 1 if any.
void check_finite(cudaStream_t s, const void *x, int xdt, int64_t rows, int64_t cols,
                  int64_t ld, int32_t *flag);

// 2-D TMA map over a row-major FP64 matrix of `rows` x `cols` (row pitch
// ld elements, 16-byte aligned base and pitch), box bx x by elements, no
// swizzle; out-of-range rows and columns read as zero.
CUtensorMap make_map_f64(const double *base, int64_t rows, int64_t cols, int64_t ld, int bx,
                         int by);
// 3-D bf16 map over digit planes [planes][rows][32] (64-byte swizzle), box
// 32 x box_rows x box_planes.
CUtensorMap make_map_planes(const __nv_bfloat16 *base, int64_t rows, int planes, int box_rows,
                            int box_planes);

// ------------------------------------------- tensor-core digit products
int64_t oz_pad(int64_t v, int64_t q);
struct OzHidWs {
    __nv_bfloat16 *xp, *wp;  // digit planes of X and W
    double *xs, *ws;         // their power-of-two row / column scales
    float *xsf;              // the row scales of X as floats
    float4 *tab;             // sigmoid table
    float4 *rowc;            // per hidden row: epilogue constants (two float4)
};
// Sample rows of X arriving in chunks (copies in flight on another stream):
// chunk c covers rows row[c] .. row[c+1]-1 (the last one up to the padded
// row count), multiples of 64, ready once `ready[c]` has fired.
constexpr int OZ_MAX_CHUNKS = 8;
static_assert(OZ_MAX_CHUNKS == sizeof(elm_ctx::xready) / sizeof(cudaEvent_t), "chunk events");
struct OzRowChunks {
    int count = 0;
    int64_t row[OZ_MAX_CHUNKS] = {};
    cudaEvent_t ready[OZ_MAX_CHUNKS] = {};
};
// Scratch of oz_hidden for an N x n input and L (+ m target) rows.
OzHidWs oz_hid_carve(Arena &ar, int64_t N, int64_t n, int64_t L, int64_t m);
// Bytes of the Gram digit planes (5 planes of Lp x Np bf16,
// Lp = pad(L + m, 128), Np = pad(N, 64)).
size_t oz_gram_planes_bytes(int64_t N, int64_t L, int64_t m);
// H = a g(X W + b): pre-activation from exact digit slices on the tensor
// cores, activation in double-float in the epilogue, written straight into
// the Gram digit planes (rows < L, zero padding) with row scales hs, as
// FP64 H^T (row stride ldh) when Ht != NULL, and as double-float H (N x L,
// sample-major, eight bytes per element, about 2^-43 relative) when
// Hdf != NULL.  *err set on a device-side timeout; *nonfinite (if given)
// |= 1 when X holds a NaN or an infinity.  wait_ns bounds each pipeline
// wait of the tensor kernel (0: 2 s).
void oz_hidden(cudaStream_t s, const OzHidWs &w, const void *X, int xdt, int64_t N, int64_t n,
               int64_t ldx, const double *W, int64_t ldw, const double *b, const double *a,
               int act, int64_t L, int64_t m, __nv_bfloat16 *planes, double *hs, double *Ht,
               int64_t ldh, int *err, void *Hdf = nullptr,
               int32_t *nonfinite = nullptr, const OzRowChunks *chunks = nullptr,
               uint64_t wait_ns = 0, int stages = 3);
// T -> digit plane rows L .. L+m-1.
void oz_t_digits(cudaStream_t s, const double *T, int64_t ldt, int64_t N, int64_t L, int64_t m,
                 __nv_bfloat16 *planes, double *hs);
// G (Lt x Lt, both triangles, Lt = L + m): Gram of [H^T; T^T] from the planes.
// part (oz_gram_part_bytes()): int64 partial sums of the tiles of a last,
// partial wave of at most half the SM count, which are split over every SM
// by K chunks (NULL: no split).
size_t oz_gram_part_bytes();
void oz_gram(cudaStream_t s, const __nv_bfloat16 *planes, const double *hs, int64_t N,
             int64_t L, int64_t m, double *G, int64_t ldg, int *err, long long *part,
             uint64_t wait_ns = 0, int stages = 3);
// [H^T H, H^T T] (Lt x Lt, ldg, both triangles, Lt = L + m) of the FP64
// matrix A = [H^T; T^T] (Lt x N, lda) on the tensor cores, accurate to FP64
// level (eight 7-bit digits per element, every digit pair of weight above
// 2^-68 summed exactly).  planes: oz_exact_planes_bytes(N, L, m) bytes; hs,
// hsf: pad(Lt, 128) row scales; *err set on a device-side timeout,
// *nonfinite (if given) |= 1 when A holds a NaN or an infinity.
size_t oz_exact_planes_bytes(int64_t N, int64_t L, int64_t m);
void oz_gram_exact(cudaStream_t s, const double *A, int64_t lda, int64_t N, int64_t L, int64_t m,
                   __nv_bfloat16 *planes, double *hs, float *hsf, double *G, int64_t ldg, int *err,
                   int32_t *nonfinite, uint64_t wait_ns = 0);
// Pre-activations Ht[j, i] = sum_k X[i, k] W[k, j] (L x N, ldh) on the
// tensor cores, accurate to FP64 level: both operands split into eight 7-bit
// digits on a 2^-55 grid of their row's (X) or column's (W) power-of-two
// scale, every digit pair of weight above 2^-68 summed exactly, in two
// launches.  ws: oz_hidden_exact_bytes(N, n, L) bytes of device scratch;
// *err set on a device-side timeout, *nonfinite (if given) |= 1 when X or W
// holds a NaN or an infinity.
size_t oz_hidden_exact_bytes(int64_t N, int64_t n, int64_t L);
void oz_hidden_exact(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n, int64_t ldx,
                     const double *W, int64_t ldw, int64_t L, char *ws, double *Ht, int64_t ldh,
                     int *err, int32_t *nonfinite, uint64_t wait_ns = 0);
// Several problems' hidden layers (mixed form, H as double-float pairs and
// the Gram digit planes) and Grams [H^T H, H^T T] as one tensor-core launch
// each.  Every item carries its own inputs (device pointers), scratch (hw,
// planes, hs) and outputs (Hdf, G); dev: oz_batch_bytes(count) bytes of
// device memory for the launch descriptors; after_hidden (may be NULL) is
// recorded between the two launches.
struct OzBatchItem {
    const void *X;
    int xdt;
    int64_t N, n, ldx;
    const double *W;
    int64_t ldw;
    const double *b, *a;
    int act;
    int64_t L, m;
    const double *T;
    int64_t ldt;
    __nv_bfloat16 *planes;
    double *hs, *G;
    int64_t ldg;
    OzHidWs hw;
    void *Hdf;
    int32_t *nonfinite;
};
size_t oz_batch_bytes(int64_t count);
void oz_hidden_gram_batch(cudaStream_t s, const OzBatchItem *items, int64_t count, void *dev,
                          int *err, uint64_t wait_ns, cudaEvent_t after_hidden);
// out[i, c] = A[i * lda + c] - B[i * m + c]  (rows x m)
void sub_rows(cudaStream_t s, const double *A, int64_t lda, const double *B, int64_t rows,
              int64_t m, double *out);

}  // namespace elm
