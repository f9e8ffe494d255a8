/*
 * elm.h -- C ABI of the GB300 rank-based pseudoinverse ELM library (libelm.so).
 *
 * Paper: R. Ragala, G. Bharadwaja Kumar, "Rank Based Pseudoinverse
 * Computation in Extreme Learning Machine for large Datasets",
 * arXiv 2011.02436.  The library trains a single-hidden-layer network:
 *   H = g(X W + b)            (Eq. 1, Eq. 3; Algorithm 1 step 2)
 *   rank r, permutation P, H P = [H1 H2]   (Eq. 6; Algorithm 1 steps 3-4)
 *   beta = H^+ T              (Eq. 5, Eq. 7; Algorithm 1 step 9)
 *
 * Conventions for every entry point
 *   - Matrices are row-major.  "ld" arguments are row strides in elements.
 *   - Pointers may be device memory (cudaMalloc, PyTorch CUDA tensors) or
 *     host memory; the library asks the CUDA runtime which, per pointer,
 *     and stages host buffers through its own device workspace (the copies
 *     are enqueued on the context's stream).  The caller keeps ownership of
 *     every buffer it passes; nothing is retained after the call returns.
 *   - Work is enqueued on the context's stream.  Calls that return values
 *     on the host (ranks, results, host outputs) synchronise that stream
 *     before returning; elm_hidden and elm_predict with device outputs do
 *     not.
 *   - Errors are returned as an elm_status code, never thrown.  Arguments
 *     are validated before anything is launched (ELM_ERR_ARG).
 *     elm_last_error() gives a one-line description of the last failure.
 *   - One context per host thread.  The context owns a growable device
 *     workspace, freed by elm_destroy.
 */
#ifndef ELM_H
#define ELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elm_ctx elm_ctx;

typedef enum elm_status {
    ELM_OK = 0,
    ELM_ERR_ARG = 1,            /* invalid argument (detected before launch) */
    ELM_ERR_CUDA = 2,           /* a CUDA runtime call failed               */
    ELM_ERR_NOMEM = 3,          /* device workspace allocation failed       */
    ELM_ERR_NUMERIC = 4,        /* non-finite input or Gram matrix          */
    ELM_ERR_NOT_CONVERGED = 5,  /* refinement did not reach refine_tol; beta
                                   is still written (see elm_train)          */
    ELM_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up       */
    ELM_ERR_UNSUPPORTED = 7     /* size or mode outside the supported range */
} elm_status;

enum { ELM_ACT_SIGMOID = 0, ELM_ACT_TANH = 1 };   /* g: logistic (Section 4) or tanh */
enum { ELM_F32 = 0, ELM_F64 = 1 };               /* element type of X              */
/* Arithmetic of the dense products.  ELM_PREC_FP64: FP64 FMAs throughout.
 * ELM_PREC_MIXED: hidden layer and Gram from exact integer-digit slices on
 * the tensor cores (H to about 2^-44, the Gram to about 2^-34), rank
 * decision and factorisation in double-float, FP64 solves, refinement
 * against the double-float H.  ELM_PREC_FP64_TC: the FP64 form with its
 * hidden-layer products and Gram on the tensor cores, every operand element
 * rounded once at 2^-56 of its row's power-of-two scale, split into eight
 * 7-bit digits, and every digit pair above 2^-68 summed exactly (FP64-level
 * products; activation, factorisation, solves and refinement in FP64); the
 * mixed form hands the problems its Gram cannot settle to this form.
 * Size limits: the tensor-core products sum exact integers into int64 per
 * output element, which holds any data up to ELM_MIXED_MAX_ROWS samples (N
 * rounded up to 64) and ELM_MIXED_MAX_INPUTS inputs (n rounded up to 32)
 * in ELM_PREC_MIXED, and up to ELM_EXACT_MAX_K of either in
 * ELM_PREC_FP64_TC.  Beyond its limits a request takes the next form:
 * elm_train trains a mixed problem in the ELM_PREC_FP64_TC form and an
 * ELM_PREC_FP64_TC problem in the ELM_PREC_FP64 form (elm_result.form says
 * which), elm_hidden computes the pre-activation the same way, and
 * elm_rows_create builds an FP64 row block. */
enum { ELM_PREC_FP64 = 0, ELM_PREC_MIXED = 1, ELM_PREC_FP64_TC = 2 };
#define ELM_MIXED_MAX_ROWS 8257536   /* 8064 chunks of 1024 samples */
#define ELM_MIXED_MAX_INPUTS 64512   /* 63 chunks of 1024 inputs    */
#define ELM_EXACT_MAX_K 212735488    /* 415499 chunks of 512        */

/* Largest hidden-layer width L the factorisation kernels accept. */
#define ELM_MAX_L 16384

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t (may
 * be NULL for the legacy default stream).  *out receives the context. */
int elm_create(elm_ctx **out, int device, void *stream);
/* Free the context and its workspace.  NULL is accepted. */
int elm_destroy(elm_ctx *ctx);
/* Change the stream later calls enqueue on. */
int elm_set_stream(elm_ctx *ctx, void *stream);
/* Static description of a status code. */
const char *elm_status_string(int status);
/* Description of the last failure on this context ("" if none). */
const char *elm_last_error(elm_ctx *ctx);

/*
 * Hidden layer (Eq. 1, Eq. 3; Algorithm 1 step 2), stored transposed:
 *   Ht[j*ldh + i] = a_j * g( sum_k X[i*ldx + k] * W[k*ldw + j] + b_j )
 * X: N x n, element type x_dtype (ELM_F32 / ELM_F64).  W: n x L FP64.
 * b: L FP64.  a: L FP64 output scales, or NULL for all ones.  act: ELM_ACT_*.
 * Ht: L x N FP64 output (ldh >= N).  precision: ELM_PREC_FP64 computes the
 * products with FP64 FMAs; ELM_PREC_MIXED with exact integer-digit slices on
 * the tensor cores (the result is FP64 to about 2^-40 absolute);
 * ELM_PREC_FP64_TC with eight-digit slices on the tensor cores (X rows and W
 * columns rounded at 2^-56 of their largest magnitude, the rest exact) and
 * the activation in FP64.
 */
int elm_hidden(elm_ctx *ctx, const void *X, int x_dtype, int64_t N, int64_t n,
               int64_t ldx, const double *W, int64_t ldw, const double *b,
               const double *a, int64_t L, int act, int precision, double *Ht,
               int64_t ldh);

/*
 * Rank and pseudoinverse of H given as Ht (L x N, ldh >= N, FP64)
 * (Eq. 5, Eq. 6; Algorithm 1 steps 3-4).
 * The Gram matrix H^T H is equilibrated to unit diagonal and factorised by
 * diagonal-pivoted Cholesky; pivoting stops when the largest remaining
 * diagonal is <= tol_rank (tol_rank <= 0 selects L * 2^-52).
 *   rank_out: host int64, receives r.
 *   perm_out: int32[L] (host or device) or NULL: perm_out[0..r-1] are the
 *             columns of H1, perm_out[r..L-1] the dependent columns in
 *             ascending order.
 *   pinv_out: L x N (ldp >= N) FP64 receiving H^+, or NULL.  Forming H^+
 *             costs O(L N r); meant for small problems and tests.
 */
int elm_pinv_rank(elm_ctx *ctx, const double *Ht, int64_t L, int64_t N,
                  int64_t ldh, double tol_rank, int64_t *rank_out,
                  int32_t *perm_out, double *pinv_out, int64_t ldp);

/* One training problem for elm_train. */
typedef struct elm_problem {
    const void *X;      /* N x n, row stride ldx, type x_dtype              */
    int32_t x_dtype;    /* ELM_F32 or ELM_F64                                */
    int32_t act;        /* ELM_ACT_SIGMOID or ELM_ACT_TANH                   */
    int64_t N, n, ldx;
    const double *W;    /* n x L, row stride ldw                             */
    int64_t ldw;
    const double *b;    /* L                                                 */
    const double *a;    /* L output scales, or NULL                          */
    int64_t L;
    const double *T;    /* N x m targets, row stride ldt                     */
    int64_t m, ldt;
    double *beta;       /* output: L x m, row stride ldb                     */
    int64_t ldb;
} elm_problem;

typedef struct elm_train_opts {
    int32_t precision;  /* ELM_PREC_FP64, ELM_PREC_MIXED or ELM_PREC_FP64_TC */
    int32_t max_refine; /* refinement steps (< 0: default 2 FP64, 12 mixed;
                           mixed steps stop early once they stop contracting) */
    double tol_rank;    /* rank threshold on the unit-diagonal scale (<=0: L*2^-52
                           for FP64, max(L*2^-52, 2^-32) for MIXED, whose Gram
                           is exact up to dropped digit pairs below 2^-34)   */
    double refine_tol;  /* stop when ||dbeta||_F <= refine_tol ||beta||_F (<=0: 1e-12
                           for FP64, 1e-9 for MIXED)                          */
    int32_t flags;      /* ELM_FLAG_* bits                                   */
    int32_t wait_limit_ns; /* bound, in ns, of each pipeline wait inside the
                           tensor-core kernels of ELM_PREC_MIXED (<= 0: 2 s).
                           When a bound expires the kernel stops issuing
                           work, lets its own copies and MMAs finish, frees
                           its tensor memory and returns; the problem's
                           status is ELM_ERR_TIMEOUT and the context stays
                           usable.  Small values exist to exercise that path */
    int32_t block_split; /* > 0: instead of the rank-based route, the paper's
                           block formulae for the split H = [H1 H2] with H1
                           the first block_split columns (Eqs. 19-23: A =
                           H2^T H2, B = A^{-1} H2^T T, D = H1^T C H1 as the
                           Schur complement S11 - S12 A^{-1} S21, beta1 =
                           D^{-1} H1^T (T - H2 B), beta2 = B - A^{-1} H2^T H1
                           beta1), in FP64, followed by the refinement steps.
                           Needs 0 < block_split < L and H of full column
                           rank (A or D singular: ELM_ERR_NUMERIC); wide
                           problems (N < L) are rejected (ELM_ERR_ARG)     */
    int32_t lanes;      /* several ELM_PREC_MIXED problems in one call: how
                           many problems' factorisations, solves and
                           refinements run at the same time, each on its own
                           stream, workspaces and host thread, once the
                           call's batched hidden layers and Grams are done
                           (0: 4; at most ELM_MAX_LANES; 1: one after
                           another on the context's stream).  Every
                           problem's arithmetic is the same whatever lane
                           runs it, so beta does not depend on this value */
} elm_train_opts;

#define ELM_MAX_LANES 32

/* elm_train_opts.flags: record CUDA events around each training phase on
 * the context's stream (read them with elm_phase_times). */
#define ELM_FLAG_PHASE_TIMING 1

/* elm_result.form: the route that produced beta */
#define ELM_FORM_FP64 0          /* FP64 form (ELM_PREC_FP64)                   */
#define ELM_FORM_MIXED 1         /* mixed form                                  */
#define ELM_FORM_MIXED_TO_FP64 2 /* mixed form handed over to the FP64 form     */
#define ELM_FORM_WIDE 3          /* N < L: H^+ = H^T (H H^T)^+ in FP64 (the
                                    branch stated with Eq. 8), either precision */
#define ELM_FORM_BLOCK 4         /* the paper's block formulae (Eqs. 19-23),
                                    elm_train_opts.block_split, FP64          */
#define ELM_FORM_FP64_TC 5       /* FP64 form, Gram on the tensor cores       */

typedef struct elm_result {
    int64_t rank;         /* r                                              */
    int32_t refine_iters; /* refinement steps taken                         */
    int32_t status;       /* elm_status of this problem                     */
    double rel_update;    /* ||dbeta||_F / ||beta||_F of the last step      */
    int32_t form;         /* ELM_FORM_*                                     */
    int32_t reserved;     /* 0                                              */
} elm_result;

/*
 * Train `count` independent problems (Algorithm 1): hidden layer, Gram
 * H^T H and H^T T, pivoted rank decision, beta = H^+ T through the
 * full-rank factorisation H P = H1 [I K] (beta = P [I; K^T] (I + K K^T)^{-1}
 * (H1^T H1)^{-1} H1^T T), then refinement steps with the residual
 * H^T (T - H beta).  opts may be NULL (FP64 defaults).  results: host array
 * of `count` entries, or NULL.  Returns ELM_OK or the first failing status.
 * ELM_PREC_MIXED trains a problem in the FP64 form (ELM_PREC_FP64_TC)
 * instead when its tensor-core Gram cannot settle it: a rejected pivot above
 * the FP64 rank threshold, or refinement that does not reach refine_tol
 * (results[i].form tells which route produced beta).  With more than one
 * problem, the mixed form runs the hidden layers and Grams of the whole
 * call as one tensor-core launch each before the problems' solves.
 * A problem with fewer samples than hidden neurons (N < L) takes the wide
 * branch in either precision: the N x N Gram H H^T of the rows of H is
 * factorised by the same pivoted Cholesky (rank r over the rows, tol_rank
 * default N 2^-52), and beta = H^T (H H^T)^+ T is formed through the
 * full-rank factorisation of the rows, with refinement steps as above.
 * A problem whose FP64 refinement ends (after max_refine steps) with an
 * update above refine_tol gets ELM_ERR_NOT_CONVERGED: beta is written, and
 * results[i].rel_update tells how far the last step still moved it.  That
 * happens when H is so ill-conditioned that FP64 arithmetic cannot fix beta
 * to refine_tol (the residual equations contract by about kappa(H)^2 u per
 * step).  Every other non-OK status leaves beta unwritten.
 */
int elm_train(elm_ctx *ctx, const elm_problem *probs, int64_t count,
              const elm_train_opts *opts, elm_result *results);

/*
 * Prediction (Section 2, step 3): Y = g(X W + b) beta without storing H.
 * X, W, b, a, act as for elm_hidden; beta: L x m (ldb); Y: N x m FP64 (ldy).
 */
int elm_predict(elm_ctx *ctx, const void *X, int x_dtype, int64_t N,
                int64_t n, int64_t ldx, const double *W, int64_t ldw,
                const double *b, const double *a, int64_t L, int act,
                const double *beta, int64_t m, int64_t ldb, double *Y,
                int64_t ldy);

/*
 * Row-sharded training: the rows of H split into blocks (one per process or
 * GPU), each block contributing H_p^T H_p and H_p^T T_p, which a caller sums
 * over the blocks (one all-reduce) before a single factorisation; the
 * refinement residual H^T (T - H beta) is summed the same way.  This is the
 * distributed setting the paper names as future work (Section 5); the
 * arithmetic is that of elm_train (Eqs. 5-13, Algorithm 1) with the sums
 * over samples split.  The caller owns the exchange (for example
 * torch.distributed); the library never communicates.
 *
 * elm_rows_create: hidden layer of one row block (X: N x n, T: N x m) in the
 * given precision, kept on the device by the handle (FP64 H^T, or the
 * double-float H of the mixed form), and the block's Gram blocks.  Inputs
 * are staged as for elm_train; nothing is retained from them afterwards.
 * elm_rows_gram: S (L x L, lds >= L) = H_p^T H_p and Z (L x m, ldz >= m) =
 * H_p^T T_p of the block (host or device outputs; the call synchronises).
 * elm_rows_residual: Gres (L x m, ldr >= m) = H_p^T (T_p - H_p beta) for
 * beta (L x m, ldb >= m).  elm_rows_destroy frees the handle (NULL is
 * accepted).  A handle uses its context's stream and workspace: use it from
 * the context's thread, and destroy it before the context.
 *
 * elm_factor_gram: the pivoted rank decision and factorisation of a summed
 * Gram matrix S (L x L, lds) (Eq. 6; Algorithm 1 steps 3-4) with the rules
 * of elm_train for `precision` (tol_rank <= 0: the default threshold), kept
 * by the handle with everything the solves need for up to m right-hand
 * sides; *rank_out (host) receives r.  A mixed-precision decision that the
 * mixed Gram cannot settle (a rejected pivot above L 2^-52) returns
 * ELM_ERR_NUMERIC; factor the FP64 Gram instead.
 * elm_factor_solve: out (L x mc, ldo) = P [I; K^T] (I + K K^T)^{-1}
 * R11^{-1} R11^{-T} Z[perm[0..r-1]] for Z (L x mc, ldz), mc <= m: beta for
 * Z = H^T T, the correction for Z = Gres (Eq. 5, Eq. 7).
 */
typedef struct elm_rows elm_rows;
typedef struct elm_factor elm_factor;
int elm_rows_create(elm_ctx *ctx, const void *X, int x_dtype, int64_t N, int64_t n,
                    int64_t ldx, const double *W, int64_t ldw, const double *b,
                    const double *a, int64_t L, int act, const double *T, int64_t m,
                    int64_t ldt, int precision, elm_rows **out);
int elm_rows_gram(elm_rows *rows, double *S, int64_t lds, double *Z, int64_t ldz);
int elm_rows_residual(elm_rows *rows, const double *beta, int64_t ldb, double *Gres,
                      int64_t ldr);
int elm_rows_destroy(elm_rows *rows);
int elm_factor_gram(elm_ctx *ctx, const double *S, int64_t lds, int64_t L, int64_t m,
                    int precision, double tol_rank, elm_factor **out, int64_t *rank_out);
int elm_factor_solve(elm_factor *f, const double *Z, int64_t ldz, int64_t mc, double *out,
                     int64_t ldo);
int elm_factor_destroy(elm_factor *f);

/*
 * Instrumentation (the paper has no counterpart; it reports wall-clock
 * training time only, Section 4).
 *
 * elm_phase_times: milliseconds spent in each training phase, summed over
 * the elm_train calls made with ELM_FLAG_PHASE_TIMING since the previous
 * elm_phase_times call (which resets the sums).  Phases, in order:
 *   0 hidden layer (mixed form: with the digit rows of T)
 *   1 Gram H^T H, H^T T   2 pivoted factorisation
 *   3 first solve    4 refinement
 * Writes min(max_phases, ELM_NUM_PHASES) values to ms_out (host) and
 * returns ELM_NUM_PHASES, or a negative elm_status on error.
 *
 * elm_launch_counter: number of kernels this library has launched in the
 * process so far (all contexts).
 */
#define ELM_NUM_PHASES 5
int elm_phase_times(elm_ctx *ctx, double *ms_out, int max_phases);
const char *elm_phase_name(int phase);
int64_t elm_launch_counter(void);

/*
 * Autotuner (no counterpart in the paper: it picks launch shapes, not
 * arithmetic).  elm_autotune trains the given problems several times with
 * different launch choices and keeps the fastest for their shape bucket
 * (floor(log2) of L, N and n for one problem; of the problem count for a
 * batched call; per precision) in the context, where elm_train then uses
 * it for every problem of that bucket:
 *   one problem: the cluster size (8 or 16 CTAs) and width (16, 24 or 32
 *     pivots; FP64 forms up to 24) of the factorisation's pivot panels, by
 *     the factor phase's time, and for ELM_PREC_MIXED the pipeline depth
 *     (2 or 3 stages) of the hidden-layer and Gram tensor kernels, by their
 *     phases' times (CUDA events on the context's stream);
 *   several problems: elm_train_opts.lanes (1, 2, 4 or 8), by the call's time.
 * The runs write beta into the problems' outputs like elm_train (launch
 * choices can move beta only within the form's rounding).  opts: as for
 * elm_train (flags and lanes are set by the tuner).  cache_path (may be
 * NULL): a text file, one line per bucket ("<bucket> cs=.. nb=.. hs=.. gs=..
 * lanes=.."), rewritten with this bucket's choice.  out (may be NULL)
 * receives the choice.  elm_autotune_load reads such a file into the
 * context (lines that do not parse, or hold values outside the ranges
 * above, are skipped; ELM_ERR_ARG if the file cannot be opened).  Choices
 * hold until the context is destroyed; 0 in a field means the built-in
 * default.
 */
typedef struct elm_tune_choice {
    int32_t panel_cluster;  /* CTAs of a pivot-panel cluster                      */
    int32_t panel_width;    /* pivots per factorisation panel                     */
    int32_t hidden_stages;  /* pipeline stages of the mixed hidden-layer kernel   */
    int32_t gram_stages;    /* pipeline stages of the mixed Gram kernel           */
    int32_t lanes;          /* lanes of a batched mixed call                      */
    int32_t reserved;
    double best_ms;         /* one problem: chosen factor + hidden + Gram phase
                               times; several: the call's time (ms)            */
} elm_tune_choice;
int elm_autotune(elm_ctx *ctx, const elm_problem *probs, int64_t count,
                 const elm_train_opts *opts, const char *cache_path, elm_tune_choice *out);
int elm_autotune_load(elm_ctx *ctx, const char *cache_path);

/*
 * elm_hidden_noalloc -- the mixed-precision hidden layer of elm_hidden
 * (ELM_PREC_MIXED) for callers that may not allocate device memory, neither
 * themselves nor through the library: for example a plugin inside a host
 * framework that owns all device memory through its own pool, or a service
 * that forbids allocator calls once it has started.  The paper has no
 * counterpart; this is an interface variant, the arithmetic is that of
 * elm_hidden.
 *
 * No context is needed and nothing is allocated: all scratch (the digit
 * slices of X, W and H, their scales, the activation table and an error
 * flag) lives in one fixed device array compiled into the library, of
 * ELM_NOALLOC_SCRATCH_BYTES per device, held by every device that loads the
 * library until the process exits.  elm_hidden_noalloc_bytes() reports how
 * much of it a problem needs; larger problems get ELM_ERR_UNSUPPORTED.
 * X, W, b, a and Ht must be device memory of the current device, and
 * `stream` (a cudaStream_t, NULL for the legacy default stream) a stream of
 * that device; anything else is ELM_ERR_ARG.  The layouts are those of
 * elm_hidden.  The call synchronises `stream` before returning.
 *
 * The first call on a device looks up the array's device address with that
 * device current (once per device and CUDA context: a call after
 * cudaDeviceReset looks it up again); make that first call outside any
 * latency-critical section.  Every call on a device shares the same
 * array and leaves its contents behind, so calls that overlap on the GPU
 * (other threads or other streams) race and must be serialised by the
 * caller.
 */
#define ELM_NOALLOC_SCRATCH_BYTES (32u << 20)
int elm_hidden_noalloc(const void *X, int x_dtype, int64_t N, int64_t n, int64_t ldx,
                       const double *W, int64_t ldw, const double *b, const double *a,
                       int64_t L, int act, double *Ht, int64_t ldh, void *stream);
int elm_hidden_noalloc_bytes(int64_t N, int64_t n, int64_t L, int64_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* ELM_H */
