// C ABI of libelm.so (declared in include/elm.h): argument validation,
// host/device staging, workspace planning and the order of the training
// steps of Algorithm 1.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "elm_internal.cuh"

using namespace elm;

namespace elm {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace elm

namespace {

const char *kPhaseName[ELM_NUM_PHASES] = {"hidden", "gram", "factor", "solve", "refine"};

void mark(elm_ctx *ctx, int i) {
    if (ctx->timing) ELM_CUDA(cudaEventRecord(ctx->ev[i], ctx->stream));
}

// Adds the phases first .. last-1 (events first .. last) to the sums.
void collect_phases(elm_ctx *ctx, int first = 0, int last = ELM_NUM_PHASES) {
    if (!ctx->timing) return;
    ELM_CUDA(cudaEventSynchronize(ctx->ev[last]));
    for (int i = first; i < last; i++) {
        float ms = 0.f;
        ELM_CUDA(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        ctx->phase_ms[i] += ms;
    }
}

const char *kStatusText[] = {
    "ok",
    "invalid argument",
    "CUDA runtime error",
    "device workspace allocation failed",
    "non-finite input or Gram matrix",
    "refinement did not converge",
    "bounded device-side wait gave up",
    "unsupported size or mode",
};

template <class F>
int guarded(elm_ctx *ctx, F &&f) {
    try {
        f();
        if (ctx) ctx->last_error.clear();
        return ELM_OK;
    } catch (const ElmError &e) {
        if (ctx) ctx->last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->last_error = "host allocation failed";
        return ELM_ERR_NOMEM;
    } catch (...) {
        if (ctx) ctx->last_error = "unexpected exception";
        return ELM_ERR_CUDA;
    }
}

void require(bool ok, const char *what) {
    if (!ok) throw ElmError(ELM_ERR_ARG, what);
}

// Strided copy of `rows` rows of `width` bytes; one linear copy when both
// sides are contiguous (the 2-D copy path moves pinned host memory at well
// under half the rate of a linear copy on GB300).
void copy2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t rows,
            cudaMemcpyKind kind, cudaStream_t s) {
    if (rows == 0 || width == 0) return;
    if ((dpitch == width && spitch == width) || rows == 1)
        ELM_CUDA(cudaMemcpyAsync(dst, src, width * rows, kind, s));
    else
        ELM_CUDA(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s));
}

bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void grow(char **buf, size_t *size, size_t need, cudaStream_t s) {
    if (need <= *size) return;
    ELM_CUDA(cudaStreamSynchronize(s));
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *size = 0;
    size_t want = need + need / 8 + (1 << 20);
    if (cudaMalloc(buf, want) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        throw ElmError(ELM_ERR_NOMEM, "cudaMalloc of the workspace failed");
    }
    *size = want;
}

// Run `plan` once to measure, grow the buffer, run it again for real.
void with_arena(char **buf, size_t *size, cudaStream_t s,
                const std::function<void(Arena &)> &plan) {
    Arena m;
    plan(m);
    grow(buf, size, m.used, s);
    Arena a;
    a.base = *buf;
    a.cap = *size;
    plan(a);
}

// A read-only input matrix: the caller's pointer if it is device memory,
// else a staged device copy (row stride becomes `cols`).
struct In {
    const void *p = nullptr;
    int64_t ld = 0;
    bool host = false;
};

In stage(Arena &ar, cudaStream_t s, const void *p, int64_t rows, int64_t cols, int64_t ld,
         size_t esz) {
    In r;
    if (!p) return r;
    if (on_device(p)) {
        r.p = p;
        r.ld = ld;
        return r;
    }
    char *d = ar.take<char>((size_t)(rows * cols) * esz);
    r.p = d;
    r.ld = cols;
    r.host = true;
    if (d)
        copy2d(d, cols * esz, p, ld * esz, cols * esz, rows,
                                   cudaMemcpyHostToDevice, s);
    return r;
}

// ----------------------------------------------------------------- solves
// beta = H^+ Z through the full-rank factorisation H P = H1 [I K]
// (Eq. 5, Eq. 7): out[perm[i], :] = ([y; K^T y])[i, :] with
// y = (I + K K^T)^{-1} R11^{-1} R11^{-T} Z[perm[0..r-1], :] and
// K = R11^{-1} R12.  The r x r system I + K K^T is solved through the
// (L-r) x (L-r) system I + K^T K (Woodbury identity).  Everything that
// depends only on the factor (inverse diagonal blocks, K, the factor of
// I + K^T K) is prepared once and reused by every refinement step.
struct Solver {
    const double *R = nullptr, *Rt = nullptr;
    int64_t ld = 0;
    const int32_t *perm = nullptr;
    int64_t r = 0, L = 0, m = 0;
    double *DinvF = nullptr, *DinvB = nullptr;
    // r < L
    double *K = nullptr, *G2 = nullptr, *R2 = nullptr, *Rt2 = nullptr, *syrk_part = nullptr;
    double *atv_part = nullptr;
    int atv_split = 1;
    double *DinvF2 = nullptr, *DinvB2 = nullptr;
    int64_t ld2 = 0;
    FactorWs f2{};
    // per-solve scratch
    double *yb = nullptr, *v = nullptr, *w = nullptr;
    int *tflag = nullptr;
    char *kws = nullptr;   // the tensor-core K solve's digit planes
    // I + K^T K on the tensor cores (mixed form): K^T, its digit planes, scales
    double *Kt = nullptr, *khs = nullptr;
    __nv_bfloat16 *kplanes = nullptr;
    float *khsf = nullptr;
};

// The mixed form forms K = R11^{-1} R12 on the tensor cores (32-row blocks,
// exact digit updates) from this size on; smaller ones take the cluster solve.
static bool ksolve_on_tensor_cores(int64_t r, int64_t q) { return r >= 256 && q >= 64; }

// df_k: form K = R11^{-1} R12 in double-float (the mixed form, whose factor
// is double-float accurate): on the tensor cores by 32-row blocks from
// ksolve_on_tensor_cores' size on, else by the double-float cluster solve;
// the per-step solves stay FP64.
Solver solver_prepare(elm_ctx *ctx, cudaStream_t s, const double *R, const double *Rt,
                      int64_t ld, const int32_t *perm, int64_t r, int64_t L, int64_t m,
                      char **buf = nullptr, size_t *bufsize = nullptr, bool df_k = false) {
    Solver sv;
    sv.R = R;
    sv.Rt = Rt;
    sv.ld = ld;
    sv.perm = perm;
    sv.r = r;
    sv.L = L;
    sv.m = m;
    const int64_t q = L - r;
    sv.ld2 = q > 0 ? tri_ld(q) : 0;
    const int syrk_split = syrk_f64_splits(r, q, ctx->sm_count);
    const int atv_split = atv_splits(r, q, ctx->sm_count);
    sv.atv_split = atv_split;
    with_arena(buf ? buf : &ctx->aux, buf ? bufsize : &ctx->aux_size, s, [&](Arena &a) {
        sv.yb = a.take<double>(L * m);
        sv.DinvF = a.take<double>(trsm_dinv_doubles(r));
        sv.DinvB = a.take<double>(trsm_dinv_doubles(r));
        sv.tflag = a.take<int>(1);
        if (q > 0 && r > 0) {
            sv.K = a.take<double>(r * q);
            sv.G2 = a.take<double>(q * q);
            sv.syrk_part = a.take<double>(syrk_f64_ws(q, syrk_split));
            sv.atv_part = a.take<double>((int64_t)atv_split * q * m);
            sv.v = a.take<double>(q * m);
            sv.w = a.take<double>(q * m);
            sv.R2 = a.take<double>(q * sv.ld2);
            sv.Rt2 = a.take<double>(q * sv.ld2);
            sv.DinvF2 = a.take<double>(trsm_dinv_doubles(q));
            sv.DinvB2 = a.take<double>(trsm_dinv_doubles(q));
            sv.f2 = factor_ws_carve(a, q);
            if (df_k && ksolve_on_tensor_cores(r, q)) {
                sv.kws = a.take<char>(ksolve_tc_bytes(r, q));
                sv.Kt = a.take<double>(q * r);
                sv.kplanes = a.take<__nv_bfloat16>(oz_exact_planes_bytes(r, q, 0) / 2);
                sv.khs = a.take<double>(oz_pad(q, 128));
                sv.khsf = a.take<float>(oz_pad(q, 128));
            }
        }
    });
    ELM_CUDA(cudaMemsetAsync(sv.tflag, 0, sizeof(int), s));
    trsm_prepare(s, R, ld, r, sv.DinvF, sv.DinvB);
    if (q > 0 && r > 0) {
        copy2d(sv.K, q * sizeof(double), R + r, ld * sizeof(double),
                                   q * sizeof(double), r, cudaMemcpyDeviceToDevice, s);
        if (sv.kws) ksolve_tc(s, R, ld, sv.DinvF, r, sv.K, q, q, sv.kws, sv.tflag);
        else trsm_bwd(s, Rt, ld, sv.DinvB, r, sv.K, q, q, sv.tflag, df_k);
        if (sv.Kt) {
            // I + K^T K to FP64 accuracy on the tensor cores (the Gram of K's
            // columns, exact digit pairs)
            transpose_f64(s, sv.K, r, q, q, sv.Kt, r);
            oz_gram_exact(s, sv.Kt, r, r, q, 0, sv.kplanes, sv.khs, sv.khsf, sv.G2, q, sv.tflag,
                          nullptr);
            add_identity(s, sv.G2, q, q);
        } else {
            syrk_f64(s, sv.K, r, q, q, sv.G2, q, sv.syrk_part, syrk_split);   // I + K^T K
        }
        // I + K^T K is SPD with eigenvalues >= 1: full rank q (double-float
        // factor for the mixed form, like the Gram's)
        factor_pivoted(s, sv.G2, q, q, 0.0, sv.f2, sv.R2, sv.Rt2, sv.ld2, ctx->sm_count, df_k);
        trsm_prepare(s, sv.R2, sv.ld2, q, sv.DinvF2, sv.DinvB2);
    }
    return sv;
}

void solver_apply(cudaStream_t s, const Solver &sv, const double *Z, int64_t ldz, double *out,
                  int64_t ldo, int64_t mcols = -1) {
    const int64_t r = sv.r, L = sv.L, m = mcols > 0 ? mcols : sv.m, q = L - r;
    double *yb = sv.yb;
    gather_rows(s, Z, ldz, sv.perm, nullptr, r, m, yb, m);
    trsm_fwd(s, sv.R, sv.ld, sv.DinvF, r, yb, m, m, sv.tflag);
    trsm_bwd(s, sv.Rt, sv.ld, sv.DinvB, r, yb, m, m, sv.tflag);
    if (q > 0) {
        if (r > 0) {
            atv_f64(s, sv.K, r, q, q, yb, m, sv.v, sv.atv_part, sv.atv_split);   // K^T y
            ELM_CUDA(cudaMemsetAsync(sv.w, 0, sizeof(double) * q * m, s));
            gather_rows(s, sv.v, m, sv.f2.perm, &sv.f2.st->rank, q, m, sv.w, m);
            trsm_fwd(s, sv.R2, sv.ld2, sv.DinvF2, q, sv.w, m, m, sv.tflag);
            trsm_bwd(s, sv.Rt2, sv.ld2, sv.DinvB2, q, sv.w, m, m, sv.tflag);
            scatter_rows(s, sv.w, m, sv.f2.perm, q, sv.v, m, 1.0, 0);
            av_sub_f64(s, sv.K, r, q, q, sv.v, m, yb);                           // y -= K v
            atv_f64(s, sv.K, r, q, q, yb, m, yb + r * m, sv.atv_part, sv.atv_split);
        } else {
            ELM_CUDA(cudaMemsetAsync(yb, 0, sizeof(double) * L * m, s));
        }
    }
    scatter_rows(s, yb, m, sv.perm, L, out, ldo, 1.0, 0);
}

// Status of the solves so far (reads the device flag; synchronises s).
bool solver_timed_out(cudaStream_t s, const Solver &sv) {
    int f = 0;
    ELM_CUDA(cudaMemcpyAsync(&f, sv.tflag, sizeof f, cudaMemcpyDeviceToHost, s));
    ELM_CUDA(cudaStreamSynchronize(s));
    return f != 0;
}

int64_t read_rank(cudaStream_t s, const FactorWs &f, int32_t *flags, double *stop_val = nullptr) {
    FactorState st;
    ELM_CUDA(cudaMemcpyAsync(&st, f.st, sizeof st, cudaMemcpyDeviceToHost, s));
    ELM_CUDA(cudaStreamSynchronize(s));
    if (flags) *flags = st.flags;
    if (stop_val) *stop_val = st.stop_val;
    return st.rank;
}

void check_dims(int64_t N, int64_t n, int64_t ldx, int64_t L, int64_t ldw) {
    require(N >= 1 && n >= 1 && L >= 1, "N, n and L must be >= 1");
    require(ldx >= n, "ldx < n");
    require(ldw >= L, "ldw < L");
    require(L <= ELM_MAX_L, "L above ELM_MAX_L");
}

// ------------------------------------------------------------ one problem
struct Problem {
    const elm_problem *p;
    int prec;
    int max_refine;
    double tau;
    double tau64;      // the FP64 form's rank threshold L 2^-52 (unit-diagonal scale)
    double refine_tol;
    uint64_t wait_ns;  // bound of the tensor kernels' pipeline waits (0: default)
    bool wide;         // N < L: the branch H^+ = H^T (H H^T)^+
    int64_t block;     // > 0: the paper's block formulae, H1 = first `block` columns
    int lanes;         // batched mixed trainings: back halves run side by side
    Tune tune;         // autotuned launch choices of the problem's shape bucket
};

// Frees a context's device buffers, events, owned stream and lanes (not the
// object itself).
void release_ctx(elm_ctx *ctx) {
    cudaSetDevice(ctx->device);
    for (elm_ctx *l : ctx->lanes) {
        release_ctx(l);
        delete l;
    }
    ctx->lanes.clear();
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->batch) cudaFree(ctx->batch);
    ctx->ws = ctx->aux = ctx->batch = nullptr;
    ctx->ws_size = ctx->aux_size = ctx->batch_size = 0;
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
        ctx->copy_stream = nullptr;
    }
    if (ctx->xstart) cudaEventDestroy(ctx->xstart), ctx->xstart = nullptr;
    for (auto &e : ctx->xready)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    ctx->stream = nullptr;
}

// Lane i of a context: its own non-blocking stream, workspaces and events.
elm_ctx *lane_of(elm_ctx *ctx, size_t i) {
    while (ctx->lanes.size() <= i) {
        elm_ctx *l = new elm_ctx;
        l->device = ctx->device;
        l->sm_count = ctx->sm_count;
        try {
            ELM_CUDA(cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking));
            l->own_stream = true;
            for (auto &e : l->ev) ELM_CUDA(cudaEventCreate(&e));
        } catch (...) {
            release_ctx(l);
            delete l;
            throw;
        }
        ctx->lanes.push_back(l);
    }
    return ctx->lanes[i];
}

// Shape buckets of the autotune cache: floor(log2) of L, N and n per
// precision for one problem; of the problem count for a batched call.
int ilog2(int64_t v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        r++;
    }
    return r;
}
std::string tune_key(int prec, const elm_problem &p) {
    return "p" + std::to_string(prec) + "_L" + std::to_string(ilog2(p.L)) + "_N" +
           std::to_string(ilog2(p.N)) + "_n" + std::to_string(ilog2(p.n));
}
std::string tune_batch_key(int prec, int64_t count) {
    return "p" + std::to_string(prec) + "_batch" + std::to_string(ilog2(count));
}

void train_mixed(elm_ctx *ctx, const Problem &P, elm_result *res);
void train_wide(elm_ctx *ctx, const Problem &P, elm_result *res);
void train_block(elm_ctx *ctx, const Problem &P, elm_result *res);

void train_one(elm_ctx *ctx, const Problem &P, elm_result *res) {
    if (P.block > 0) return train_block(ctx, P, res);
    if (P.wide) return train_wide(ctx, P, res);
    if (P.prec == ELM_PREC_MIXED) return train_mixed(ctx, P, res);
    // FP64 form; ELM_PREC_FP64_TC forms its Gram on the tensor cores
    const bool tc = P.prec == ELM_PREC_FP64_TC;
    res->form = tc ? ELM_FORM_FP64_TC : ELM_FORM_FP64;
    res->reserved = 0;
    const elm_problem &pb = *P.p;
    cudaStream_t s = ctx->stream;
    const int64_t N = pb.N, n = pb.n, L = pb.L, m = pb.m, Lt = L + m;
    const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
    const int ns = gram_f64_nsplit(L, m, N, ctx->sm_count);
    const int hs = htr_f64_nsplit(L, N, ctx->sm_count);
    In X, W, b, a, T;
    double *Ht, *S, *Z, *gpart = nullptr, *R, *Rt, *beta, *dB, *Rres, *G, *hpart, *norms;
    double *rs = nullptr;
    float *rsf = nullptr;
    __nv_bfloat16 *planes = nullptr;
    int *err = nullptr;
    int64_t lds = L, ldz = m;
    int32_t *flag;
    FactorWs f;
    with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
        X = stage(ar, s, pb.X, N, n, pb.ldx, xsz);
        W = stage(ar, s, pb.W, n, L, pb.ldw, 8);
        b = stage(ar, s, pb.b, 1, L, L, 8);
        a = stage(ar, s, pb.a, 1, L, L, 8);
        T = stage(ar, s, pb.T, N, m, pb.ldt, 8);
        if (tc) {
            // [H^T; T^T] in one buffer, the Gram [H^T H, H^T T] beside it
            Ht = ar.take<double>(Lt * N);
            S = ar.take<double>(Lt * Lt);
            Z = S + L;
            lds = ldz = Lt;
            // the hidden product's digit planes, then the Gram's, in one buffer
            const size_t hb = oz_hidden_exact_bytes(N, n, L), gb = oz_exact_planes_bytes(N, L, m);
            planes = (__nv_bfloat16 *)ar.take<char>(hb > gb ? hb : gb);
            rs = ar.take<double>(oz_pad(Lt, 128));
            rsf = ar.take<float>(oz_pad(Lt, 128));
            err = ar.take<int>(1);
        } else {
            Ht = ar.take<double>(L * N);
            S = ar.take<double>(L * L);
            Z = ar.take<double>(L * m);
            gpart = ar.take<double>(gram_f64_ws(L, m, ns));
        }
        R = ar.take<double>(L * tri_ld(L));
        Rt = ar.take<double>(L * tri_ld(L));
        beta = ar.take<double>(L * m);
        dB = ar.take<double>(L * m);
        Rres = ar.take<double>(N * m);
        G = ar.take<double>(L * m);
        hpart = ar.take<double>(htr_f64_ws(L, m, hs));
        norms = ar.take<double>(2);
        flag = ar.take<int32_t>(1);
        f = factor_ws_carve(ar, L);
    });
    ELM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    if (tc) ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    check_finite(s, X.p, pb.x_dtype, N, n, X.ld, flag);
    const double *Wd = (const double *)W.p, *bd = (const double *)b.p,
                 *ad = (const double *)a.p, *Td = (const double *)T.p;
    mark(ctx, 0);
    // Algorithm 1 step 2: H (stored transposed); ELM_PREC_FP64_TC forms the
    // pre-activations on the tensor cores to FP64 accuracy
    if (tc) {
        oz_hidden_exact(s, X.p, pb.x_dtype, N, n, X.ld, Wd, W.ld, L, (char *)planes, Ht, N, err,
                        nullptr, P.wait_ns);
        act_rows_f64(s, Ht, N, L, N, bd, ad, pb.act);
        transpose_f64(s, Td, N, m, T.ld, Ht + L * N, N);           // T^T below H^T
    } else {
        hidden_f64(s, X.p, pb.x_dtype, N, n, X.ld, Wd, W.ld, bd, ad, L, pb.act, Ht, N);
    }
    mark(ctx, 1);
    // Eqs. 9-13: Gram blocks H^T H and H^T T
    if (tc) oz_gram_exact(s, Ht, N, N, L, m, planes, rs, rsf, S, Lt, err, nullptr, P.wait_ns);
    else gram_f64(s, Ht, N, L, N, Td, T.ld, m, S, L, Z, m, gpart, ns);
    mark(ctx, 2);
    // Eq. 6, Algorithm 1 steps 3-4: permutation, rank, split
    factor_pivoted(s, S, lds, L, P.tau, f, R, Rt, tri_ld(L), ctx->sm_count, /*df=*/false,
                   P.tune.panel_cs, P.tune.panel_nb, /*tc64=*/tc);
    mark(ctx, 3);
    int32_t fl = 0, xfl = 0;
    int terr = 0;
    const int64_t r = read_rank(s, f, &fl);
    ELM_CUDA(cudaMemcpy(&xfl, flag, sizeof xfl, cudaMemcpyDeviceToHost));
    if (tc) ELM_CUDA(cudaMemcpy(&terr, err, sizeof terr, cudaMemcpyDeviceToHost));
    res->rank = r;
    res->refine_iters = 0;
    res->rel_update = 0.0;
    res->status = ELM_OK;
    if ((fl & 2) || terr) {             // a bounded device-side wait expired
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if ((fl & 1) || xfl) {
        res->status = ELM_ERR_NUMERIC;
        return;
    }
    // Eq. 5, Eq. 7: beta = H^+ T
    const Solver sv = solver_prepare(ctx, s, R, Rt, tri_ld(L), f.perm, r, L, m);
    solver_apply(s, sv, Z, ldz, beta, m);
    mark(ctx, 4);
    // refinement with the residual T - H beta
    double nrm[2] = {0.0, 0.0};
    bool converged = P.max_refine == 0;
    for (int it = 0; it < P.max_refine; it++) {
        resid_f64(s, Ht, N, L, N, beta, m, Td, T.ld, Rres);
        htr_f64(s, Ht, N, L, N, Rres, m, G, hpart, hs);
        solver_apply(s, sv, G, m, dB, m);
        axpy_norms(s, beta, dB, L * m, norms);
        ELM_CUDA(cudaMemcpyAsync(nrm, norms, sizeof nrm, cudaMemcpyDeviceToHost, s));
        ELM_CUDA(cudaStreamSynchronize(s));
        res->refine_iters = it + 1;
        res->rel_update = nrm[1] > 0.0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (res->rel_update <= P.refine_tol) {
            converged = true;
            break;
        }
    }
    mark(ctx, 5);
    // the last step still moved beta by more than refine_tol: beta is
    // returned, flagged as not converged
    if (!converged) res->status = ELM_ERR_NOT_CONVERGED;
    if (!isfinite(res->rel_update)) res->status = ELM_ERR_NUMERIC;
    if (solver_timed_out(s, sv)) res->status = ELM_ERR_TIMEOUT;
    const cudaMemcpyKind kind = on_device(pb.beta) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost;
    copy2d(pb.beta, pb.ldb * sizeof(double), beta, m * sizeof(double),
                               m * sizeof(double), L, kind, s);
    ELM_CUDA(cudaStreamSynchronize(s));
    collect_phases(ctx);
}

// ----------------------------------------------------------- wide branch
// N < L (the branch stated with Eq. 8): H^+ = H^T (H H^T)^+.  The N x N Gram
// of the rows of H is factorised by the pivoted Cholesky of the tall case,
// which now pivots over samples: P H = [I; K^T] H1 with H1 the r
// independent rows and K = R11^{-1} R12 (H2 = K^T H1 follows from
// H2 H1^T = R12^T R11).  Both factors have full rank, so
//   H^+ = H1^+ [I; K^T]^+ P = H1^T (R11^T R11)^{-1} (I + K K^T)^{-1} [I K] P,
// the Moore-Penrose inverse for every rank (Eq. 5).  (I + K K^T)^{-1} is
// applied through I + K^T K (Woodbury), whose factor the solver prepares.
struct WideScratch {
    double *PT, *ym, *zf, *hpart;
    int hs;
};

void wide_apply(cudaStream_t s, const Solver &sv, const double *Ht, int64_t L, int64_t N,
                const double *Tin, int64_t ldt, double *out, const WideScratch &ws) {
    const int64_t r = sv.r, q = N - r, m = sv.m;
    if (r == 0) {
        ELM_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * L * m, s));
        return;
    }
    double *w = sv.yb;                                              // r x m
    gather_rows(s, Tin, ldt, sv.perm, nullptr, N, m, ws.PT, m);     // P T
    ELM_CUDA(cudaMemcpyAsync(w, ws.PT, sizeof(double) * r * m, cudaMemcpyDeviceToDevice, s));
    if (q > 0) {
        // w = [I K] P T
        ELM_CUDA(cudaMemsetAsync(ws.ym, 0, sizeof(double) * r * m, s));
        av_sub_f64(s, sv.K, r, q, q, ws.PT + r * m, m, ws.ym);      // ym = -K (P T)[r:]
        sub_rows(s, w, m, ws.ym, r, m, w);
        // w = (I + K K^T)^{-1} w = w - K (I + K^T K)^{-1} K^T w
        atv_f64(s, sv.K, r, q, q, w, m, sv.v, sv.atv_part, sv.atv_split);
        ELM_CUDA(cudaMemsetAsync(sv.w, 0, sizeof(double) * q * m, s));
        gather_rows(s, sv.v, m, sv.f2.perm, &sv.f2.st->rank, q, m, sv.w, m);
        trsm_fwd(s, sv.R2, sv.ld2, sv.DinvF2, q, sv.w, m, m, sv.tflag);
        trsm_bwd(s, sv.Rt2, sv.ld2, sv.DinvB2, q, sv.w, m, m, sv.tflag);
        scatter_rows(s, sv.w, m, sv.f2.perm, q, sv.v, m, 1.0, 0);
        av_sub_f64(s, sv.K, r, q, q, sv.v, m, w);
    }
    // (R11^T R11)^{-1} w, then beta = H1^T z (z scattered to the rows of H)
    trsm_fwd(s, sv.R, sv.ld, sv.DinvF, r, w, m, m, sv.tflag);
    trsm_bwd(s, sv.Rt, sv.ld, sv.DinvB, r, w, m, m, sv.tflag);
    ELM_CUDA(cudaMemsetAsync(ws.zf, 0, sizeof(double) * N * m, s));
    scatter_rows(s, w, m, sv.perm, r, ws.zf, m, 1.0, 0);
    htr_f64(s, Ht, N, L, N, ws.zf, m, out, ws.hpart, ws.hs);
}

void train_wide(elm_ctx *ctx, const Problem &P, elm_result *res) {
    res->form = ELM_FORM_WIDE;
    res->reserved = 0;
    const elm_problem &pb = *P.p;
    cudaStream_t s = ctx->stream;
    const int64_t N = pb.N, n = pb.n, L = pb.L, m = pb.m;
    const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
    const int ns = gram_f64_nsplit(N, 0, L, ctx->sm_count);
    const int hs = htr_f64_nsplit(L, N, ctx->sm_count);
    In X, W, b, a, T;
    double *Ht, *H, *K, *gpart, *R, *Rt, *beta, *dB, *Rres, *norms;
    int32_t *flag;
    FactorWs f;
    WideScratch ws{};
    ws.hs = hs;
    with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
        X = stage(ar, s, pb.X, N, n, pb.ldx, xsz);
        W = stage(ar, s, pb.W, n, L, pb.ldw, 8);
        b = stage(ar, s, pb.b, 1, L, L, 8);
        a = stage(ar, s, pb.a, 1, L, L, 8);
        T = stage(ar, s, pb.T, N, m, pb.ldt, 8);
        Ht = ar.take<double>(L * N);
        H = ar.take<double>(N * L);
        K = ar.take<double>(N * N);
        gpart = ar.take<double>(gram_f64_ws(N, 0, ns));
        R = ar.take<double>(N * tri_ld(N));
        Rt = ar.take<double>(N * tri_ld(N));
        beta = ar.take<double>(L * m);
        dB = ar.take<double>(L * m);
        Rres = ar.take<double>(N * m);
        ws.PT = ar.take<double>(N * m);
        ws.ym = ar.take<double>(N * m);
        ws.zf = ar.take<double>(N * m);
        ws.hpart = ar.take<double>(htr_f64_ws(L, m, hs));
        norms = ar.take<double>(2);
        flag = ar.take<int32_t>(1);
        f = factor_ws_carve(ar, N);
    });
    ELM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    check_finite(s, X.p, pb.x_dtype, N, n, X.ld, flag);
    const double *Wd = (const double *)W.p, *bd = (const double *)b.p,
                 *ad = (const double *)a.p, *Td = (const double *)T.p;
    mark(ctx, 0);
    hidden_f64(s, X.p, pb.x_dtype, N, n, X.ld, Wd, W.ld, bd, ad, L, pb.act, Ht, N);
    transpose_f64(s, Ht, L, N, N, H, L);
    mark(ctx, 1);
    // H H^T: the Gram of the rows of H
    gram_f64(s, H, L, N, L, nullptr, 0, 0, K, N, nullptr, 0, gpart, ns);
    mark(ctx, 2);
    factor_pivoted(s, K, N, N, P.tau, f, R, Rt, tri_ld(N), ctx->sm_count);
    mark(ctx, 3);
    int32_t fl = 0, xfl = 0;
    const int64_t r = read_rank(s, f, &fl);
    ELM_CUDA(cudaMemcpy(&xfl, flag, sizeof xfl, cudaMemcpyDeviceToHost));
    res->rank = r;
    res->refine_iters = 0;
    res->rel_update = 0.0;
    res->status = ELM_OK;
    if (fl & 2) {
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if ((fl & 1) || xfl) {
        res->status = ELM_ERR_NUMERIC;
        return;
    }
    const Solver sv = solver_prepare(ctx, s, R, Rt, tri_ld(N), f.perm, r, N, m);
    wide_apply(s, sv, Ht, L, N, Td, T.ld, beta, ws);
    mark(ctx, 4);
    double nrm[2] = {0.0, 0.0};
    bool converged = P.max_refine == 0;
    for (int it = 0; it < P.max_refine; it++) {
        resid_f64(s, Ht, N, L, N, beta, m, Td, T.ld, Rres);          // T - H beta
        wide_apply(s, sv, Ht, L, N, Rres, m, dB, ws);                 // H^+ (T - H beta)
        axpy_norms(s, beta, dB, L * m, norms);
        ELM_CUDA(cudaMemcpyAsync(nrm, norms, sizeof nrm, cudaMemcpyDeviceToHost, s));
        ELM_CUDA(cudaStreamSynchronize(s));
        res->refine_iters = it + 1;
        res->rel_update = nrm[1] > 0.0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (res->rel_update <= P.refine_tol) {
            converged = true;
            break;
        }
    }
    mark(ctx, 5);
    if (!converged) res->status = ELM_ERR_NOT_CONVERGED;
    if (!isfinite(res->rel_update)) res->status = ELM_ERR_NUMERIC;
    if (solver_timed_out(s, sv)) res->status = ELM_ERR_TIMEOUT;
    const cudaMemcpyKind kind = on_device(pb.beta) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost;
    copy2d(pb.beta, pb.ldb * sizeof(double), beta, m * sizeof(double), m * sizeof(double), L,
           kind, s);
    ELM_CUDA(cudaStreamSynchronize(s));
    collect_phases(ctx);
}

// ------------------------------------------------ the paper's block route
// Eqs. 19-23 (transposition of Eq. 19 fixed) for a full-rank split
// H = [H1 H2], H1 the first r1 columns:
//   A = H2^T H2 = S22,  B = A^{-1} H2^T Y = A^{-1} Z2,
//   D = H1^T C H1 = S11 - S12 A^{-1} S21  (C = I - H2 A^{-1} H2^T, Eq. 22),
//   beta1 = D^{-1} H1^T (Y - H2 B) = D^{-1} (Z1 - S12 B),
//   beta2 = B - A^{-1} H2^T H1 beta1 = B - (A^{-1} S21) beta1,
// everything from the Gram blocks S = H^T H and Z = H^T Y, so the N x N
// matrix C is never formed.  A and D are SPD when H has full column rank;
// they are factorised by the pivoted Cholesky and a rank below their size
// means the split is singular.
struct SpdFactor {
    const double *R, *Rt;
    int64_t ld, n;
    const int32_t *perm;
    double *DinvF, *DinvB;
    int *tflag;
};

// out (n x mc, ldo) = M^{-1} Z for the factorised SPD matrix M (n x n)
void spd_apply(cudaStream_t s, const SpdFactor &F, const double *Z, int64_t ldz, double *out,
               int64_t ldo, int64_t mc, double *yb) {
    gather_rows(s, Z, ldz, F.perm, nullptr, F.n, mc, yb, mc);
    trsm_fwd(s, F.R, F.ld, F.DinvF, F.n, yb, mc, mc, F.tflag);
    trsm_bwd(s, F.Rt, F.ld, F.DinvB, F.n, yb, mc, mc, F.tflag);
    scatter_rows(s, yb, mc, F.perm, F.n, out, ldo, 1.0, 0);
}

struct BlockRoute {
    SpdFactor A, D;
    const double *S;    // L x L Gram (ld L)
    int64_t L, r1, q, m;
    double *M;          // A^{-1} S21 (q x r1)
    double *Bv, *rhs, *yb;
};

// out (L x m) = the block formulae applied to Zin (L x m, ldz)
void block_apply(cudaStream_t s, const BlockRoute &b, const double *Zin, int64_t ldz,
                 double *out) {
    const int64_t L = b.L, r1 = b.r1, q = b.q, m = b.m;
    spd_apply(s, b.A, Zin + r1 * ldz, ldz, b.Bv, m, m, b.yb);                 // B
    copy2d(b.rhs, m * 8, Zin, ldz * 8, m * 8, r1, cudaMemcpyDeviceToDevice, s);
    gemm_f64(s, r1, m, q, -1.0, b.S + r1, L, 1, b.Bv, m, 1, 1.0, b.rhs, m);  // Z1 - S12 B
    spd_apply(s, b.D, b.rhs, m, out, m, m, b.yb);                              // beta1
    ELM_CUDA(cudaMemcpyAsync(out + r1 * m, b.Bv, sizeof(double) * q * m,
                             cudaMemcpyDeviceToDevice, s));
    gemm_f64(s, q, m, r1, -1.0, b.M, r1, 1, out, m, 1, 1.0, out + r1 * m, m);  // beta2
}

void train_block(elm_ctx *ctx, const Problem &P, elm_result *res) {
    res->form = ELM_FORM_BLOCK;
    res->reserved = 0;
    const elm_problem &pb = *P.p;
    cudaStream_t s = ctx->stream;
    const int64_t N = pb.N, n = pb.n, L = pb.L, m = pb.m, r1 = P.block, q = L - r1;
    const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
    const int ns = gram_f64_nsplit(L, m, N, ctx->sm_count);
    const int hs = htr_f64_nsplit(L, N, ctx->sm_count);
    const int64_t nm = r1 > q ? r1 : q, mm = m > r1 ? m : r1;
    In X, W, b, a, T;
    double *Ht, *S, *Z, *gpart, *RA, *RtA, *RD, *RtD, *Dm, *beta, *dB, *Rres, *G, *hpart, *norms;
    int32_t *flag;
    int *tflag;
    FactorWs fA, fD;
    BlockRoute br{};
    with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
        X = stage(ar, s, pb.X, N, n, pb.ldx, xsz);
        W = stage(ar, s, pb.W, n, L, pb.ldw, 8);
        b = stage(ar, s, pb.b, 1, L, L, 8);
        a = stage(ar, s, pb.a, 1, L, L, 8);
        T = stage(ar, s, pb.T, N, m, pb.ldt, 8);
        Ht = ar.take<double>(L * N);
        S = ar.take<double>(L * L);
        Z = ar.take<double>(L * m);
        gpart = ar.take<double>(gram_f64_ws(L, m, ns));
        RA = ar.take<double>(q * tri_ld(q));
        RtA = ar.take<double>(q * tri_ld(q));
        RD = ar.take<double>(r1 * tri_ld(r1));
        RtD = ar.take<double>(r1 * tri_ld(r1));
        Dm = ar.take<double>(r1 * r1);
        br.A.DinvF = ar.take<double>(trsm_dinv_doubles(q));
        br.A.DinvB = ar.take<double>(trsm_dinv_doubles(q));
        br.D.DinvF = ar.take<double>(trsm_dinv_doubles(r1));
        br.D.DinvB = ar.take<double>(trsm_dinv_doubles(r1));
        br.M = ar.take<double>(q * r1);
        br.Bv = ar.take<double>(q * m);
        br.rhs = ar.take<double>(r1 * m);
        br.yb = ar.take<double>(nm * mm);
        beta = ar.take<double>(L * m);
        dB = ar.take<double>(L * m);
        Rres = ar.take<double>(N * m);
        G = ar.take<double>(L * m);
        hpart = ar.take<double>(htr_f64_ws(L, m, hs));
        norms = ar.take<double>(2);
        flag = ar.take<int32_t>(1);
        tflag = ar.take<int>(1);
        fA = factor_ws_carve(ar, q);
        fD = factor_ws_carve(ar, r1);
    });
    ELM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    ELM_CUDA(cudaMemsetAsync(tflag, 0, sizeof(int), s));
    check_finite(s, X.p, pb.x_dtype, N, n, X.ld, flag);
    const double *Wd = (const double *)W.p, *bd = (const double *)b.p,
                 *ad = (const double *)a.p, *Td = (const double *)T.p;
    mark(ctx, 0);
    hidden_f64(s, X.p, pb.x_dtype, N, n, X.ld, Wd, W.ld, bd, ad, L, pb.act, Ht, N);
    mark(ctx, 1);
    gram_f64(s, Ht, N, L, N, Td, T.ld, m, S, L, Z, m, gpart, ns);       // Eqs. 9-13
    mark(ctx, 2);
    res->rank = 0;
    res->refine_iters = 0;
    res->rel_update = 0.0;
    res->status = ELM_OK;
    // A = S22 (Eq. 20), then M = A^{-1} S21 and D = S11 - S12 M (Eq. 23)
    factor_pivoted(s, S + r1 * L + r1, L, q, (double)q * ldexp(1.0, -52), fA, RA, RtA,
                   tri_ld(q), ctx->sm_count);
    int32_t fl = 0, xfl = 0;
    const int64_t rA = read_rank(s, fA, &fl);
    ELM_CUDA(cudaMemcpy(&xfl, flag, sizeof xfl, cudaMemcpyDeviceToHost));
    if (fl & 2) {
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if ((fl & 1) || xfl || rA < q) {     // non-finite, or A singular
        res->status = ELM_ERR_NUMERIC;
        res->rank = rA;
        return;
    }
    br.A = SpdFactor{RA, RtA, tri_ld(q), q, fA.perm, br.A.DinvF, br.A.DinvB, tflag};
    trsm_prepare(s, RA, tri_ld(q), q, br.A.DinvF, br.A.DinvB);
    spd_apply(s, br.A, S + r1 * L, L, br.M, r1, r1, br.yb);
    copy2d(Dm, r1 * 8, S, L * 8, r1 * 8, r1, cudaMemcpyDeviceToDevice, s);
    gemm_f64(s, r1, r1, q, -1.0, S + r1, L, 1, br.M, r1, 1, 1.0, Dm, r1);
    factor_pivoted(s, Dm, r1, r1, (double)r1 * ldexp(1.0, -52), fD, RD, RtD, tri_ld(r1),
                   ctx->sm_count);
    const int64_t rD = read_rank(s, fD, &fl);
    if (fl & 2) {
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if ((fl & 1) || rD < r1) {           // D singular: H is rank deficient
        res->status = ELM_ERR_NUMERIC;
        res->rank = rA + rD;
        return;
    }
    res->rank = L;
    mark(ctx, 3);
    br.D = SpdFactor{RD, RtD, tri_ld(r1), r1, fD.perm, br.D.DinvF, br.D.DinvB, tflag};
    trsm_prepare(s, RD, tri_ld(r1), r1, br.D.DinvF, br.D.DinvB);
    br.S = S;
    br.L = L;
    br.r1 = r1;
    br.q = q;
    br.m = m;
    block_apply(s, br, Z, m, beta);                                      // Eqs. 19, 21
    mark(ctx, 4);
    double nrm[2] = {0.0, 0.0};
    bool converged = P.max_refine == 0;
    for (int it = 0; it < P.max_refine; it++) {
        resid_f64(s, Ht, N, L, N, beta, m, Td, T.ld, Rres);
        htr_f64(s, Ht, N, L, N, Rres, m, G, hpart, hs);
        block_apply(s, br, G, m, dB);
        axpy_norms(s, beta, dB, L * m, norms);
        ELM_CUDA(cudaMemcpyAsync(nrm, norms, sizeof nrm, cudaMemcpyDeviceToHost, s));
        ELM_CUDA(cudaStreamSynchronize(s));
        res->refine_iters = it + 1;
        res->rel_update = nrm[1] > 0.0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (res->rel_update <= P.refine_tol) {
            converged = true;
            break;
        }
    }
    mark(ctx, 5);
    if (!converged) res->status = ELM_ERR_NOT_CONVERGED;
    if (!isfinite(res->rel_update)) res->status = ELM_ERR_NUMERIC;
    int tf = 0;
    ELM_CUDA(cudaMemcpyAsync(&tf, tflag, sizeof tf, cudaMemcpyDeviceToHost, s));
    ELM_CUDA(cudaStreamSynchronize(s));
    if (tf) res->status = ELM_ERR_TIMEOUT;
    const cudaMemcpyKind kind = on_device(pb.beta) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost;
    copy2d(pb.beta, pb.ldb * sizeof(double), beta, m * sizeof(double), m * sizeof(double), L,
           kind, s);
    ELM_CUDA(cudaStreamSynchronize(s));
    collect_phases(ctx);
}

// Mixed form: H, H^T H and H^T T from exact digit slices on the tensor
// cores (the Gram is that of H on a 2^-34 grid), rank decision and
// factorisation in double-float, FP64 solves, then refinement steps whose
// residual G = H^T (T - H beta) reads H itself, kept in double-float
// (about 2^-43), so the steps converge to the least-squares solution of
// the accurate H, not of the grid H.  Two cases the grid Gram cannot
// settle fall back to the FP64 form for that problem: a rejected pivot
// above the FP64 threshold L 2^-52 (the FP64 rank rule might keep it), and
// refinement that does not reach refine_tol (H too ill-conditioned for a
// Gram accurate to 2^-34 to precondition the steps).
// The front half (hidden layer and Gram) keeps its results in the
// context's batch buffer; the back half below takes its scratch from the main
// workspace, which the FP64 hand-over reuses.
struct MixedData {
    const double *T;     // staged targets (N x m, ldt)
    int64_t ldt;
    double *G;           // [H^T H, H^T T] (Lt x Lt)
    void *Hdf;           // H as double-float pairs, sample-major
    int32_t *flag;       // non-finite X
    int *err;            // a tensor-kernel wait expired
};

// Factorisation, solves, refinement and the FP64 hand-over of one mixed
// training whose Gram is ready.
void mixed_back(elm_ctx *ctx, const Problem &P, elm_result *res, const MixedData &D,
                int first_phase) {
    const elm_problem &pb = *P.p;
    cudaStream_t s = ctx->stream;
    const int64_t N = pb.N, L = pb.L, m = pb.m;
    const int64_t Lt = L + m;
    const int hs_split = htr_df_nsplit(L, N, ctx->sm_count);
    double *R, *Rt, *beta, *dB, *Rres, *Gres, *hpart, *norms, *betaT;
    FactorWs f;
    with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
        R = ar.take<double>(L * tri_ld(L));
        Rt = ar.take<double>(L * tri_ld(L));
        beta = ar.take<double>(L * m);
        dB = ar.take<double>(L * m);
        Rres = ar.take<double>(N * m);
        Gres = ar.take<double>(L * m);
        hpart = ar.take<double>((int64_t)hs_split * L * m);
        betaT = ar.take<double>(L * (m < 32 ? m : 32));
        norms = ar.take<double>(2);
        f = factor_ws_carve(ar, L);
    });
    auto fallback = [&]() {
        Problem P64 = P;
        P64.prec = ELM_PREC_FP64_TC;
        P64.max_refine = 2;
        P64.tau = P.tau64;
        P64.refine_tol = 1e-12;
        train_one(ctx, P64, res);
        res->form = ELM_FORM_MIXED_TO_FP64;
    };
    // Eq. 6, Algorithm 1 steps 3-4 (double-float)
    factor_pivoted(s, D.G, Lt, L, P.tau, f, R, Rt, tri_ld(L), ctx->sm_count, /*df=*/true,
                   P.tune.panel_cs, P.tune.panel_nb);
    mark(ctx, 3);
    int32_t fl = 0, xfl = 0;
    int terr = 0;
    double stop_val = 0.0;
    const int64_t r = read_rank(s, f, &fl, &stop_val);
    ELM_CUDA(cudaMemcpy(&xfl, D.flag, sizeof xfl, cudaMemcpyDeviceToHost));
    ELM_CUDA(cudaMemcpy(&terr, D.err, sizeof terr, cudaMemcpyDeviceToHost));
    res->rank = r;
    res->refine_iters = 0;
    res->rel_update = 0.0;
    res->status = ELM_OK;
    res->form = ELM_FORM_MIXED;
    res->reserved = 0;
    if (terr || (fl & 2)) {
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if ((fl & 1) || xfl) {
        res->status = ELM_ERR_NUMERIC;
        return;
    }
    // a rank decision the mixed Gram cannot settle goes to the FP64 form
    if (r < L && stop_val > P.tau64) return fallback();
    const double *Z = D.G + L;   // Z[l, c] = G[l, L + c]
    // Eq. 5, Eq. 7 (FP64)
    const Solver sv = solver_prepare(ctx, s, R, Rt, tri_ld(L), f.perm, r, L, m, nullptr, nullptr,
                                     /*df_k=*/true);
    solver_apply(s, sv, Z, Lt, beta, m);
    mark(ctx, 4);
    double nrm[2] = {0.0, 0.0};
    bool converged = P.max_refine == 0;
    double prev = INFINITY;
    for (int it = 0; it < P.max_refine; it++) {
        resid_df(s, D.Hdf, L, N, beta, m, D.T, D.ldt, Rres, betaT);     // T - H beta (pairs)
        htr_df(s, D.Hdf, L, N, Rres, m, Gres, hpart, hs_split);        // H^T (T - H beta)
        solver_apply(s, sv, Gres, m, dB, m);
        axpy_norms(s, beta, dB, L * m, norms);
        ELM_CUDA(cudaMemcpyAsync(nrm, norms, sizeof nrm, cudaMemcpyDeviceToHost, s));
        ELM_CUDA(cudaStreamSynchronize(s));
        res->refine_iters = it + 1;
        res->rel_update = nrm[1] > 0.0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (res->rel_update <= P.refine_tol) {
            converged = true;
            break;
        }
        // the steps must contract; once they stop doing so the grid Gram
        // is too coarse a preconditioner for this H
        if (it >= 1 && !(res->rel_update < 0.5 * prev)) break;
        prev = res->rel_update;
    }
    mark(ctx, 5);
    if (solver_timed_out(s, sv)) {
        res->status = ELM_ERR_TIMEOUT;
        return;
    }
    if (!converged) return fallback();
    if (!isfinite(res->rel_update)) res->status = ELM_ERR_NUMERIC;
    const cudaMemcpyKind kind = on_device(pb.beta) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost;
    copy2d(pb.beta, pb.ldb * sizeof(double), beta, m * sizeof(double), m * sizeof(double), L,
           kind, s);
    ELM_CUDA(cudaStreamSynchronize(s));
    collect_phases(ctx, first_phase, ELM_NUM_PHASES);
}

void train_mixed(elm_ctx *ctx, const Problem &P, elm_result *res) {
    const elm_problem &pb = *P.p;
    cudaStream_t s = ctx->stream;
    const int64_t N = pb.N, n = pb.n, L = pb.L, m = pb.m;
    const int64_t Lt = L + m, Lp = oz_pad(Lt, 128);
    const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
    In X, W, b, a, T;
    double *hs, *G, *Hdf;
    long long *gpart;
    __nv_bfloat16 *planes;
    int32_t *flag;
    int *err;
    OzHidWs hw;
    // host X is uploaded in row chunks on a second stream; the hidden layer
    // takes each chunk as it lands (below)
    const bool x_host = !on_device(pb.X);
    char *xdev = nullptr;
    with_arena(&ctx->batch, &ctx->batch_size, s, [&](Arena &ar) {
        if (x_host) {
            xdev = ar.take<char>((size_t)(N * n) * xsz);
            X.p = xdev;
            X.ld = n;
            X.host = true;
        } else {
            X = stage(ar, s, pb.X, N, n, pb.ldx, xsz);
        }
        W = stage(ar, s, pb.W, n, L, pb.ldw, 8);
        b = stage(ar, s, pb.b, 1, L, L, 8);
        a = stage(ar, s, pb.a, 1, L, L, 8);
        T = stage(ar, s, pb.T, N, m, pb.ldt, 8);
        planes = (__nv_bfloat16 *)ar.take<char>(oz_gram_planes_bytes(N, L, m));
        hs = ar.take<double>(Lp);
        G = ar.take<double>(Lt * Lt);
        hw = oz_hid_carve(ar, N, n, L, m);
        Hdf = ar.take<double>(N * L);    // H as double-float pairs, eight bytes each
        gpart = (long long *)ar.take<char>(oz_gram_part_bytes());
        flag = ar.take<int32_t>(1);
        err = ar.take<int>(1);
    });
    ELM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const double *Wd = (const double *)W.p, *bd = (const double *)b.p,
                 *ad = (const double *)a.p, *Td = (const double *)T.p;
    OzRowChunks xc;
    if (x_host) {
        if (!ctx->copy_stream) {
            ELM_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
            ELM_CUDA(cudaEventCreateWithFlags(&ctx->xstart, cudaEventDisableTiming));
            for (auto &e : ctx->xready)
                ELM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        // the buffer is free once the work already queued on s is done
        ELM_CUDA(cudaEventRecord(ctx->xstart, s));
        ELM_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->xstart, 0));
        const int64_t Np = oz_pad(N, 64);
        const int64_t nch = Np / 64 < 4 ? Np / 64 : 4;
        xc.count = (int)nch;
        for (int c = 0; c < xc.count; c++) {
            xc.row[c] = c * Np / nch / 64 * 64;
            xc.ready[c] = ctx->xready[c];
        }
        for (int c = 0; c < xc.count; c++) {
            const int64_t r0 = xc.row[c];
            const int64_t r1 = c + 1 < xc.count ? xc.row[c + 1] : N;
            if (r1 > r0 && r0 < N)
                copy2d(xdev + (size_t)r0 * n * xsz, n * xsz,
                       (const char *)pb.X + (size_t)r0 * pb.ldx * xsz, pb.ldx * xsz, n * xsz,
                       (r1 < N ? r1 : N) - r0, cudaMemcpyHostToDevice, ctx->copy_stream);
            ELM_CUDA(cudaEventRecord(xc.ready[c], ctx->copy_stream));
        }
    }
    mark(ctx, 0);
    // Algorithm 1 step 2 (Eq. 1, 3): pre-activation on the tensor cores,
    // activation in the epilogue, digit planes of H and H itself
    oz_hidden(s, hw, X.p, pb.x_dtype, N, n, X.ld, Wd, W.ld, bd, ad, pb.act, L, m, planes, hs,
              nullptr, 0, err, Hdf, /*nonfinite=*/flag, x_host ? &xc : nullptr, P.wait_ns,
              P.tune.hid_stages ? P.tune.hid_stages : 3);
    // digit rows of the targets beside those of H (part of the hidden phase,
    // so the Gram phase times the Gram kernel alone)
    oz_t_digits(s, Td, T.ld, N, L, m, planes, hs);
    mark(ctx, 1);
    // Eqs. 9-13: [H^T H, H^T T] on the tensor cores
    oz_gram(s, planes, hs, N, L, m, G, Lt, err, gpart, P.wait_ns,
            P.tune.gram_stages ? P.tune.gram_stages : 3);
    mark(ctx, 2);
    mixed_back(ctx, P, res, MixedData{Td, T.ld, G, Hdf, flag, err}, 0);
}

// The back halves (factorisation, solves, refinement, and the FP64 form for
// a problem handed over) of problems i0 .. i0+gn-1 of a batched call, on nl
// lanes at once: one host thread per lane (this thread drives lane 0) takes
// the next problem and runs it on the lane's own stream and workspaces, so
// one problem's host waits and small launches overlap another's kernels.
// Each problem's arithmetic is the serial route's, whatever lane runs it.
// The first error stops the hand-out; the call reports it after the lanes
// are done.  Phase times are summed over the lanes.
void back_halves_on_lanes(elm_ctx *ctx, const std::vector<Problem> &Ps, int64_t i0, int64_t gn,
                          const std::vector<MixedData> &data, elm_result *res, int nl) {
    std::vector<elm_ctx *> ls((size_t)nl);
    for (int l = 0; l < nl; l++) ls[(size_t)l] = lane_of(ctx, (size_t)l);
    // the lanes start once the batch's hidden layers and Grams are done
    cudaEvent_t ready = nullptr;
    ELM_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    struct EvGuard {
        cudaEvent_t e;
        ~EvGuard() { cudaEventDestroy(e); }
    } guard{ready};
    ELM_CUDA(cudaEventRecord(ready, ctx->stream));
    for (elm_ctx *l : ls) {
        l->timing = ctx->timing;
        ELM_CUDA(cudaStreamWaitEvent(l->stream, ready, 0));
    }
    // the lanes take the problems in descending order of their estimated
    // back-half work (factorisation L^3/3, refinement 2 N L m), so that no
    // large problem starts last and leaves one lane running alone
    std::vector<int64_t> order((size_t)gn);
    for (int64_t j = 0; j < gn; j++) order[(size_t)j] = j;
    auto cost = [&](int64_t j) {
        const elm_problem *q = Ps[(size_t)(i0 + j)].p;
        const double L = (double)q->L;
        return L * L * L / 3.0 + 2.0 * (double)q->N * L * (double)q->m;
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return cost(a) > cost(b); });
    std::atomic<int64_t> next{0};
    std::atomic<bool> stop{false};
    std::mutex mu;
    int err_status = ELM_OK;
    std::string err_msg;
    auto work = [&](elm_ctx *lc) {
        if (cudaSetDevice(lc->device) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            if (err_status == ELM_OK) err_status = ELM_ERR_CUDA, err_msg = "cudaSetDevice failed";
            stop = true;
            return;
        }
        for (;;) {
            if (stop.load()) return;
            const int64_t n = next.fetch_add(1);
            if (n >= gn) return;
            const int64_t j = order[(size_t)n];
            elm_result r{};
            try {
                mark(lc, 2);
                mixed_back(lc, Ps[i0 + j], &r, data[(size_t)j], 2);
            } catch (const ElmError &e) {
                r.status = e.status;
                std::lock_guard<std::mutex> lk(mu);
                if (err_status == ELM_OK) err_status = e.status, err_msg = e.msg;
                stop = true;
            } catch (...) {
                r.status = ELM_ERR_CUDA;
                std::lock_guard<std::mutex> lk(mu);
                if (err_status == ELM_OK) err_status = ELM_ERR_CUDA, err_msg = "lane failed";
                stop = true;
            }
            if (res) res[i0 + j] = r;
        }
    };
    std::vector<std::thread> th;
    try {
        for (int l = 1; l < nl; l++) th.emplace_back(work, ls[(size_t)l]);
    } catch (...) {
        stop = true;   // no thread for this lane: the running ones finish
    }
    work(ls[0]);
    for (auto &t : th) t.join();
    for (elm_ctx *l : ls) {
        ELM_CUDA(cudaStreamSynchronize(l->stream));
        for (int i = 0; i < ELM_NUM_PHASES; i++) {
            ctx->phase_ms[i] += l->phase_ms[i];
            l->phase_ms[i] = 0.0;
        }
    }
    if (err_status != ELM_OK) throw ElmError(err_status, err_msg);
}

// Several mixed-form problems: their hidden layers and Grams as one
// tensor-core launch each (the problems' data side by side in the batch
// buffer, in groups that fit half of the free device memory), then each
// problem's factorisation, solves and refinement.
void train_batch_mixed(elm_ctx *ctx, const std::vector<Problem> &Ps, elm_result *res) {
    cudaStream_t s = ctx->stream;
    const int64_t count = (int64_t)Ps.size();
    auto need = [&](const elm_problem &pb) {
        Arena m;
        const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
        const int64_t Lt = pb.L + pb.m;
        if (!on_device(pb.X)) m.take<char>((size_t)(pb.N * pb.n) * xsz);
        if (!on_device(pb.W)) m.take<double>(pb.n * pb.L);
        if (!on_device(pb.b)) m.take<double>(pb.L);
        if (pb.a && !on_device(pb.a)) m.take<double>(pb.L);
        if (!on_device(pb.T)) m.take<double>(pb.N * pb.m);
        m.take<char>(oz_gram_planes_bytes(pb.N, pb.L, pb.m));
        m.take<double>(oz_pad(Lt, 128));
        m.take<double>(Lt * Lt);
        oz_hid_carve(m, pb.N, pb.n, pb.L, pb.m);
        m.take<double>(pb.N * pb.L);
        m.take<int32_t>(1);
        return m.used + 256;
    };
    size_t free_b = 0, total_b = 0;
    ELM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = (free_b + ctx->batch_size) / 2;
    int64_t i0 = 0;
    while (i0 < count) {
        // the next group: as many problems as the budget holds (at least one)
        size_t used = oz_batch_bytes(1);
        int64_t i1 = i0;
        while (i1 < count) {
            const size_t add = need(*Ps[i1].p) + oz_batch_bytes(i1 - i0 + 1) - oz_batch_bytes(i1 - i0);
            if (i1 > i0 && used + add > budget) break;
            used += add;
            i1++;
        }
        const int64_t gn = i1 - i0;
        std::vector<OzBatchItem> items(gn);
        std::vector<MixedData> data(gn);
        char *dev = nullptr;
        int *err = nullptr;
        with_arena(&ctx->batch, &ctx->batch_size, s, [&](Arena &ar) {
            dev = ar.take<char>(oz_batch_bytes(gn));
            err = ar.take<int>(1);
            for (int64_t j = 0; j < gn; j++) {
                const elm_problem &pb = *Ps[i0 + j].p;
                const size_t xsz = pb.x_dtype == ELM_F64 ? 8 : 4;
                const int64_t N = pb.N, n = pb.n, L = pb.L, m = pb.m, Lt = L + m;
                const In X = stage(ar, s, pb.X, N, n, pb.ldx, xsz);
                const In W = stage(ar, s, pb.W, n, L, pb.ldw, 8);
                const In b = stage(ar, s, pb.b, 1, L, L, 8);
                const In a = stage(ar, s, pb.a, 1, L, L, 8);
                const In T = stage(ar, s, pb.T, N, m, pb.ldt, 8);
                OzBatchItem &q = items[j];
                q.X = X.p;
                q.xdt = pb.x_dtype;
                q.N = N;
                q.n = n;
                q.ldx = X.ld;
                q.W = (const double *)W.p;
                q.ldw = W.ld;
                q.b = (const double *)b.p;
                q.a = (const double *)a.p;
                q.act = pb.act;
                q.L = L;
                q.m = m;
                q.T = (const double *)T.p;
                q.ldt = T.ld;
                q.planes = (__nv_bfloat16 *)ar.take<char>(oz_gram_planes_bytes(N, L, m));
                q.hs = ar.take<double>(oz_pad(Lt, 128));
                q.G = ar.take<double>(Lt * Lt);
                q.ldg = Lt;
                q.hw = oz_hid_carve(ar, N, n, L, m);
                q.Hdf = ar.take<double>(N * L);
                q.nonfinite = ar.take<int32_t>(1);
                data[j] = MixedData{q.T, q.ldt, q.G, q.Hdf, q.nonfinite, err};
            }
        });
        ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        for (int64_t j = 0; j < gn; j++)
            ELM_CUDA(cudaMemsetAsync(items[j].nonfinite, 0, sizeof(int32_t), s));
        mark(ctx, 0);
        oz_hidden_gram_batch(s, items.data(), gn, dev, err, Ps[i0].wait_ns,
                             ctx->timing ? ctx->ev[1] : nullptr);
        mark(ctx, 2);
        collect_phases(ctx, 0, 2);
        const int nl = (int)(Ps[i0].lanes < gn ? Ps[i0].lanes : gn);
        if (nl > 1) {
            back_halves_on_lanes(ctx, Ps, i0, gn, data, res, nl);
        } else {
            for (int64_t j = 0; j < gn; j++) {
                elm_result r{};
                mark(ctx, 2);
                try {
                    mixed_back(ctx, Ps[i0 + j], &r, data[j], 2);
                } catch (const ElmError &e) {
                    r.status = e.status;
                    if (res) res[i0 + j] = r;
                    throw;
                }
                if (res) res[i0 + j] = r;
            }
        }
        i0 = i1;
    }
}

// ------------------------------------------------------ row-sharded route
// Owned device memory of a handle (freed with it).
struct OwnedMem {
    char *p = nullptr;
    size_t size = 0;
    ~OwnedMem() {
        if (p) cudaFree(p);
    }
};

}  // namespace

// One row block of a problem: its hidden layer kept on the device.
struct elm_rows {
    elm_ctx *ctx = nullptr;
    int precision = ELM_PREC_FP64;
    int64_t N = 0, L = 0, m = 0;
    OwnedMem mem;                 // H, T, S, Z and the residual scratch
    double *Ht = nullptr;         // FP64 form: L x N
    void *Hdf = nullptr;          // mixed form: N x L double-float pairs
    double *T = nullptr, *S = nullptr, *Z = nullptr, *Rres = nullptr, *part = nullptr,
           *betaT = nullptr, *beta = nullptr;
    int nsplit = 1;
};

// A factorised Gram matrix and everything its solves need.
struct elm_factor {
    elm_ctx *ctx = nullptr;
    int64_t L = 0, m = 0, r = 0;
    OwnedMem mem;                 // R, R^T, permutation
    OwnedMem aux;                 // the solver's buffers
    Solver sv;
    double *stage = nullptr, *out = nullptr;   // staging of host right-hand sides
};

namespace {

void rows_build(elm_rows *h, const void *X, int xdt, int64_t n, int64_t ldx, const double *Wp,
                int64_t ldw, const double *bp, const double *ap, int act, const double *Tp,
                int64_t ldt) {
    elm_ctx *ctx = h->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = h->N, L = h->L, m = h->m;
    const bool mixed = h->precision == ELM_PREC_MIXED;
    const size_t xsz = xdt == ELM_F64 ? 8 : 4;
    h->nsplit = mixed ? htr_df_nsplit(L, N, ctx->sm_count) : htr_f64_nsplit(L, N, ctx->sm_count);
    // owned: H, T, S, Z, residual scratch
    Arena plan;
    auto carve = [&](Arena &ar) {
        if (mixed) h->Hdf = ar.take<double>(N * L);
        else h->Ht = ar.take<double>(L * N);
        h->T = ar.take<double>(N * m);
        h->S = ar.take<double>(L * L);
        h->Z = ar.take<double>(L * m);
        h->Rres = ar.take<double>(N * m);
        h->part = ar.take<double>((size_t)h->nsplit * L * m);
        h->betaT = ar.take<double>(L * (m < 32 ? m : 32));
        h->beta = ar.take<double>(L * m);
    };
    carve(plan);
    if (cudaMalloc(&h->mem.p, plan.used) != cudaSuccess) {
        cudaGetLastError();
        h->mem.p = nullptr;
        throw ElmError(ELM_ERR_NOMEM, "cudaMalloc of the row block failed");
    }
    h->mem.size = plan.used;
    Arena own;
    own.base = h->mem.p;
    own.cap = h->mem.size;
    carve(own);
    // transient scratch in the context's workspace
    In Xs, Ws, bs, as, Ts;
    double *G = nullptr, *hs = nullptr, *gpart = nullptr;
    __nv_bfloat16 *planes = nullptr;
    long long *ipart = nullptr;
    int *err = nullptr;
    int32_t *flag = nullptr;
    OzHidWs hw{};
    const int64_t Lt = L + m, Lp = oz_pad(Lt, 128);
    const int ns = gram_f64_nsplit(L, m, N, ctx->sm_count);
    with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
        Xs = stage(ar, s, X, N, n, ldx, xsz);
        Ws = stage(ar, s, Wp, n, L, ldw, 8);
        bs = stage(ar, s, bp, 1, L, L, 8);
        as = stage(ar, s, ap, 1, L, L, 8);
        Ts = stage(ar, s, Tp, N, m, ldt, 8);
        flag = ar.take<int32_t>(1);
        err = ar.take<int>(1);
        if (mixed) {
            planes = (__nv_bfloat16 *)ar.take<char>(oz_gram_planes_bytes(N, L, m));
            hs = ar.take<double>(Lp);
            G = ar.take<double>(Lt * Lt);
            hw = oz_hid_carve(ar, N, n, L, m);
            ipart = (long long *)ar.take<char>(oz_gram_part_bytes());
        } else {
            gpart = ar.take<double>(gram_f64_ws(L, m, ns));
        }
    });
    copy2d(h->T, m * 8, Ts.p, Ts.ld * 8, m * 8, N, cudaMemcpyDeviceToDevice, s);
    ELM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const double *Wd = (const double *)Ws.p, *bd = (const double *)bs.p, *ad = (const double *)as.p;
    if (mixed) {
        oz_hidden(s, hw, Xs.p, xdt, N, n, Xs.ld, Wd, Ws.ld, bd, ad, act, L, m, planes, hs, nullptr,
                  0, err, h->Hdf, flag);
        oz_t_digits(s, h->T, m, N, L, m, planes, hs);
        oz_gram(s, planes, hs, N, L, m, G, Lt, err, ipart);
        copy2d(h->S, L * 8, G, Lt * 8, L * 8, L, cudaMemcpyDeviceToDevice, s);
        copy2d(h->Z, m * 8, G + L, Lt * 8, m * 8, L, cudaMemcpyDeviceToDevice, s);
    } else {
        check_finite(s, Xs.p, xdt, N, n, Xs.ld, flag);
        hidden_f64(s, Xs.p, xdt, N, n, Xs.ld, Wd, Ws.ld, bd, ad, L, act, h->Ht, N);
        gram_f64(s, h->Ht, N, L, N, h->T, m, m, h->S, L, h->Z, m, gpart, ns);
    }
    int32_t xfl = 0;
    int terr = 0;
    ELM_CUDA(cudaMemcpyAsync(&xfl, flag, sizeof xfl, cudaMemcpyDeviceToHost, s));
    ELM_CUDA(cudaMemcpyAsync(&terr, err, sizeof terr, cudaMemcpyDeviceToHost, s));
    ELM_CUDA(cudaStreamSynchronize(s));
    if (terr) throw ElmError(ELM_ERR_TIMEOUT, "tensor-core kernel wait expired");
    if (xfl) throw ElmError(ELM_ERR_NUMERIC, "non-finite input");
}

}  // namespace

extern "C" {

const char *elm_status_string(int status) {
    if (status < 0 || status >= (int)(sizeof kStatusText / sizeof kStatusText[0]))
        return "unknown status";
    return kStatusText[status];
}

const char *elm_last_error(elm_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int elm_create(elm_ctx **out, int device, void *stream) {
    if (!out) return ELM_ERR_ARG;
    *out = nullptr;
    elm_ctx *ctx = new (std::nothrow) elm_ctx;
    if (!ctx) return ELM_ERR_NOMEM;
    int st = guarded(ctx, [&] {
        int count = 0;
        ELM_CUDA(cudaGetDeviceCount(&count));
        require(device >= 0 && device < count, "no such CUDA device");
        ELM_CUDA(cudaSetDevice(device));
        ctx->device = device;
        ctx->stream = (cudaStream_t)stream;
        ELM_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
        for (auto &e : ctx->ev) ELM_CUDA(cudaEventCreate(&e));
    });
    if (st != ELM_OK) {
        delete ctx;
        return st;
    }
    *out = ctx;
    return ELM_OK;
}

int elm_destroy(elm_ctx *ctx) {
    if (!ctx) return ELM_OK;
    release_ctx(ctx);
    delete ctx;
    return ELM_OK;
}

int elm_set_stream(elm_ctx *ctx, void *stream) {
    if (!ctx) return ELM_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return ELM_OK;
}

int elm_hidden(elm_ctx *ctx, const void *X, int x_dtype, int64_t N, int64_t n, int64_t ldx,
               const double *W, int64_t ldw, const double *b, const double *a, int64_t L,
               int act, int precision, double *Ht, int64_t ldh) {
    if (!ctx) return ELM_ERR_ARG;
    return guarded(ctx, [&] {
        check_dims(N, n, ldx, L, ldw);
        require(X && W && b && Ht, "X, W, b and Ht must be non-NULL");
        require(x_dtype == ELM_F32 || x_dtype == ELM_F64, "x_dtype");
        require(act == ELM_ACT_SIGMOID || act == ELM_ACT_TANH, "act");
        require(precision == ELM_PREC_FP64 || precision == ELM_PREC_MIXED ||
                    precision == ELM_PREC_FP64_TC, "precision");
        require(ldh >= N, "ldh < N");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const size_t xsz = x_dtype == ELM_F64 ? 8 : 4;
        In Xs, Ws, bs, as;
        double *out = nullptr, *hs = nullptr;
        __nv_bfloat16 *planes = nullptr;
        int *err = nullptr;
        OzHidWs hw{};
        char *xws = nullptr;
        // beyond the sizes a form's exact products hold: the next form (mixed,
        // then FP64-accurate tensor cores, then FP64)
        const int prec = route_precision(precision, N, n);
        const bool mixed = prec == ELM_PREC_MIXED, tc = prec == ELM_PREC_FP64_TC;
        const bool dev_out = on_device(Ht);
        with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
            Xs = stage(ar, s, X, N, n, ldx, xsz);
            Ws = stage(ar, s, W, n, L, ldw, 8);
            bs = stage(ar, s, b, 1, L, L, 8);
            as = stage(ar, s, a, 1, L, L, 8);
            out = dev_out ? Ht : ar.take<double>(L * N);
            if (mixed) {
                planes = (__nv_bfloat16 *)ar.take<char>(oz_gram_planes_bytes(N, L, 0));
                hs = ar.take<double>(oz_pad(L, 128));
                err = ar.take<int>(1);
                hw = oz_hid_carve(ar, N, n, L, 0);
            }
            if (tc) {
                xws = ar.take<char>(oz_hidden_exact_bytes(N, n, L));
                err = ar.take<int>(1);
            }
        });
        const int64_t ldo = dev_out ? ldh : N;
        if (mixed) {
            ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
            oz_hidden(s, hw, Xs.p, x_dtype, N, n, Xs.ld, (const double *)Ws.p, Ws.ld,
                      (const double *)bs.p, (const double *)as.p, act, L, 0, planes, hs, out, ldo,
                      err);
            int terr = 0;
            ELM_CUDA(cudaMemcpyAsync(&terr, err, sizeof terr, cudaMemcpyDeviceToHost, s));
            ELM_CUDA(cudaStreamSynchronize(s));
            if (terr) throw ElmError(ELM_ERR_TIMEOUT, "tensor-core kernel wait expired");
        } else if (tc) {
            ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
            oz_hidden_exact(s, Xs.p, x_dtype, N, n, Xs.ld, (const double *)Ws.p, Ws.ld, L, xws,
                            out, ldo, err, nullptr);
            act_rows_f64(s, out, ldo, L, N, (const double *)bs.p, (const double *)as.p, act);
            int terr = 0;
            ELM_CUDA(cudaMemcpyAsync(&terr, err, sizeof terr, cudaMemcpyDeviceToHost, s));
            ELM_CUDA(cudaStreamSynchronize(s));
            if (terr) throw ElmError(ELM_ERR_TIMEOUT, "tensor-core kernel wait expired");
        } else {
            hidden_f64(s, Xs.p, x_dtype, N, n, Xs.ld, (const double *)Ws.p, Ws.ld,
                       (const double *)bs.p, (const double *)as.p, L, act, out, ldo);
        }
        if (!dev_out) {
            copy2d(Ht, ldh * 8, out, N * 8, N * 8, L,
                                       cudaMemcpyDeviceToHost, s);
            ELM_CUDA(cudaStreamSynchronize(s));
        } else if (Xs.host || Ws.host || bs.host || as.host) {
            ELM_CUDA(cudaStreamSynchronize(s));
        }
    });
}

int elm_pinv_rank(elm_ctx *ctx, const double *Ht, int64_t L, int64_t N, int64_t ldh,
                  double tol_rank, int64_t *rank_out, int32_t *perm_out, double *pinv_out,
                  int64_t ldp) {
    if (!ctx) return ELM_ERR_ARG;
    return guarded(ctx, [&] {
        require(L >= 1 && N >= 1, "L and N must be >= 1");
        require(L <= ELM_MAX_L, "L above ELM_MAX_L");
        require(ldh >= N, "ldh < N");
        require(Ht && rank_out, "Ht and rank_out must be non-NULL");
        require(!pinv_out || ldp >= N, "ldp < N");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const int ns = gram_f64_nsplit(L, 0, N, ctx->sm_count);
        In H;
        double *S, *gpart, *R, *Rt, *pv = nullptr;
        FactorWs f;
        const bool dev_p = pinv_out && on_device(pinv_out);
        with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
            H = stage(ar, s, Ht, L, N, ldh, 8);
            S = ar.take<double>(L * L);
            gpart = ar.take<double>(gram_f64_ws(L, 0, ns));
            R = ar.take<double>(L * tri_ld(L));
            Rt = ar.take<double>(L * tri_ld(L));
            f = factor_ws_carve(ar, L);
            if (pinv_out && !dev_p) pv = ar.take<double>(L * N);
        });
        const double *Hd = (const double *)H.p;
        gram_f64(s, Hd, H.ld, L, N, nullptr, 0, 0, S, L, nullptr, 0, gpart, ns);
        const double tau = tol_rank > 0.0 ? tol_rank : (double)L * ldexp(1.0, -52);
        factor_pivoted(s, S, L, L, tau, f, R, Rt, tri_ld(L), ctx->sm_count);
        int32_t fl = 0;
        const int64_t r = read_rank(s, f, &fl);
        if (fl & 2) throw ElmError(ELM_ERR_TIMEOUT, "factorisation wait expired");
        if (fl & 1) throw ElmError(ELM_ERR_NUMERIC, "non-finite Gram matrix");
        *rank_out = r;
        if (perm_out) {
            cudaMemcpyKind k = on_device(perm_out) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost;
            ELM_CUDA(cudaMemcpyAsync(perm_out, f.perm, sizeof(int32_t) * L, k, s));
        }
        if (pinv_out) {
            double *dst = dev_p ? pinv_out : pv;
            const int64_t ldd = dev_p ? ldp : N;
            const Solver sv = solver_prepare(ctx, s, R, Rt, tri_ld(L), f.perm, r, L, N);
            solver_apply(s, sv, Hd, H.ld, dst, ldd);
            if (solver_timed_out(s, sv)) throw ElmError(ELM_ERR_TIMEOUT, "solve wait expired");
            if (!dev_p)
                copy2d(pinv_out, ldp * 8, pv, N * 8, N * 8, L,
                                           cudaMemcpyDeviceToHost, s);
        }
        ELM_CUDA(cudaStreamSynchronize(s));
    });
}

int elm_train(elm_ctx *ctx, const elm_problem *probs, int64_t count,
              const elm_train_opts *opts, elm_result *results) {
    if (!ctx) return ELM_ERR_ARG;
    elm_train_opts o{};
    o.precision = ELM_PREC_FP64;
    o.max_refine = -1;
    if (opts) o = *opts;
    int first = ELM_OK;
    int st = guarded(ctx, [&] {
        require(count >= 0, "count < 0");
        require(count == 0 || probs, "probs is NULL");
        require(o.precision == ELM_PREC_FP64 || o.precision == ELM_PREC_MIXED ||
                    o.precision == ELM_PREC_FP64_TC, "precision");
        require(o.block_split >= 0, "block_split < 0");
        require(o.lanes >= 0 && o.lanes <= ELM_MAX_LANES, "lanes");
        for (int64_t i = 0; i < count; i++) {
            const elm_problem &p = probs[i];
            check_dims(p.N, p.n, p.ldx, p.L, p.ldw);
            require(p.m >= 1 && p.ldt >= p.m && p.ldb >= p.m, "m, ldt or ldb");
            require(p.X && p.W && p.b && p.T && p.beta, "NULL problem pointer");
            require(p.x_dtype == ELM_F32 || p.x_dtype == ELM_F64, "x_dtype");
            require(p.act == ELM_ACT_SIGMOID || p.act == ELM_ACT_TANH, "act");
            require(o.block_split == 0 || (o.block_split < p.L && p.N >= p.L),
                    "block_split needs 0 < block_split < L <= N");
        }
        ELM_CUDA(cudaSetDevice(ctx->device));
        ctx->timing = (o.flags & ELM_FLAG_PHASE_TIMING) != 0;
        std::vector<Problem> plan(count);
        for (int64_t i = 0; i < count; i++) {
            Problem &P = plan[i];
            P.p = &probs[i];
            // a problem larger than its form's exact products hold (int64
            // running sums) trains in the next form
            P.prec = route_precision(o.precision, probs[i].N, probs[i].n);
            P.max_refine = o.max_refine >= 0 ? o.max_refine
                                             : (P.prec == ELM_PREC_MIXED ? 12 : 2);
            // default rank threshold on the unit-diagonal scale: L 2^-52 for
            // the FP64 Gram; the mixed Gram drops digit pairs below 2^-34 of
            // the leading term, so its threshold sits above that level
            const double tau64 = (double)probs[i].L * ldexp(1.0, -52);
            P.tau64 = o.tol_rank > 0.0 ? o.tol_rank : tau64;
            P.tau = o.tol_rank > 0.0 ? o.tol_rank
                                     : (P.prec == ELM_PREC_MIXED ? fmax(tau64, ldexp(1.0, -32))
                                                                 : tau64);
            // mixed form: stop three orders below its 1e-6 accuracy target
            // (its Gram matrix alone limits beta to about 1e-10); once an
            // update is that small the remaining error is smaller still
            P.refine_tol = o.refine_tol > 0.0 ? o.refine_tol
                                              : (P.prec == ELM_PREC_MIXED ? 1e-9 : 1e-12);
            P.wait_ns = o.wait_limit_ns > 0 ? (uint64_t)o.wait_limit_ns : 0;
            // fewer samples than neurons: the wide branch, FP64 rules on the
            // N x N Gram
            P.wide = probs[i].N < probs[i].L;
            P.block = o.block_split;
            P.lanes = o.lanes > 0 ? o.lanes : 4;
            if (P.block > 0) {                 // the paper's block route: FP64 rules
                P.tau = P.tau64 = o.tol_rank > 0.0 ? o.tol_rank : tau64;
                if (o.max_refine < 0) P.max_refine = 2;
                if (!(o.refine_tol > 0.0)) P.refine_tol = 1e-12;
            }
            if (P.wide) {
                P.tau = o.tol_rank > 0.0 ? o.tol_rank : (double)probs[i].N * ldexp(1.0, -52);
                P.tau64 = P.tau;
                if (o.max_refine < 0) P.max_refine = 2;
                if (!(o.refine_tol > 0.0)) P.refine_tol = 1e-12;
            }
        }
        // autotuned launch choices of each problem's shape bucket, and the
        // lanes of a batched call
        for (int64_t i = 0; i < count; i++) {
            const auto it = ctx->tune.find(tune_key(plan[i].prec, probs[i]));
            if (it != ctx->tune.end()) plan[i].tune = it->second;
            if (o.lanes == 0 && count > 1) {
                const auto bt = ctx->tune.find(tune_batch_key(o.precision, count));
                if (bt != ctx->tune.end() && bt->second.lanes > 0) plan[i].lanes = bt->second.lanes;
            }
        }
        // mixed-form problems of a multi-problem call: hidden layers and
        // Grams batched; the others one by one
        std::vector<Problem> batch;
        std::vector<int64_t> where;
        for (int64_t i = 0; i < count; i++) {
            const Problem &P = plan[i];
            if (count > 1 && P.prec == ELM_PREC_MIXED && !P.wide && P.block == 0) {
                batch.push_back(P);
                where.push_back(i);
            }
        }
        std::vector<elm_result> bres(batch.size());
        if (!batch.empty()) {
            try {
                train_batch_mixed(ctx, batch, bres.data());
            } catch (...) {
                for (size_t j = 0; j < batch.size(); j++)
                    if (results) results[where[j]] = bres[j];
                throw;
            }
        }
        size_t nb = 0;
        for (int64_t i = 0; i < count; i++) {
            elm_result r{};
            if (nb < where.size() && where[nb] == i) {
                r = bres[nb++];
            } else {
                try {
                    train_one(ctx, plan[i], &r);
                } catch (const ElmError &e) {
                    // the problem's own entry reports the failure too
                    r.status = e.status;
                    if (results) results[i] = r;
                    throw;
                }
            }
            if (results) results[i] = r;
            if (first == ELM_OK && r.status != ELM_OK) first = r.status;
        }
    });
    return st != ELM_OK ? st : first;
}

namespace {

// One line of the autotune cache file: "<bucket> cs=.. nb=.. hs=.. gs=.. lanes=..".
bool tune_parse(const char *line, std::string &key, Tune &t) {
    char k[128];
    int cs, nb, hs, gs, ln;
    if (sscanf(line, "%127s cs=%d nb=%d hs=%d gs=%d lanes=%d", k, &cs, &nb, &hs, &gs, &ln) != 6)
        return false;
    const bool ok = (cs == 0 || cs == 8 || cs == 16) && nb >= 0 && nb <= 64 &&
                    (hs == 0 || hs == 2 || hs == 3) && (gs == 0 || gs == 2 || gs == 3) &&
                    ln >= 0 && ln <= ELM_MAX_LANES;
    if (!ok) return false;
    key = k;
    t.panel_cs = cs;
    t.panel_nb = nb;
    t.hid_stages = hs;
    t.gram_stages = gs;
    t.lanes = ln;
    return true;
}
std::string tune_line(const std::string &key, const Tune &t) {
    char b[256];
    snprintf(b, sizeof b, "%s cs=%d nb=%d hs=%d gs=%d lanes=%d", key.c_str(), t.panel_cs,
             t.panel_nb, t.hid_stages, t.gram_stages, t.lanes);
    return b;
}
// Rewrites the cache file with `key` set to t (other buckets kept).
void tune_store(const char *path, const std::string &key, const Tune &t) {
    std::vector<std::string> lines;
    if (FILE *f = fopen(path, "r")) {
        char buf[512];
        while (fgets(buf, sizeof buf, f)) {
            std::string k;
            Tune u;
            if (tune_parse(buf, k, u) && k != key) lines.push_back(tune_line(k, u));
        }
        fclose(f);
    }
    lines.push_back(tune_line(key, t));
    FILE *g = fopen(path, "w");
    if (!g) throw ElmError(ELM_ERR_ARG, "cannot write the autotune cache file");
    for (const auto &l : lines) fprintf(g, "%s\n", l.c_str());
    fclose(g);
}

}  // namespace

int elm_autotune(elm_ctx *ctx, const elm_problem *probs, int64_t count, const elm_train_opts *opts,
                 const char *cache_path, elm_tune_choice *out) {
    if (!ctx) return ELM_ERR_ARG;
    elm_train_opts o{};
    o.precision = ELM_PREC_FP64;
    o.max_refine = -1;
    if (opts) o = *opts;
    return guarded(ctx, [&] {
        require(count >= 1 && probs, "no problems to tune on");
        std::vector<elm_result> res((size_t)count);
        auto run = [&](const elm_train_opts &oo) {
            const int st = elm_train(ctx, probs, count, &oo, res.data());
            if (st != ELM_OK && st != ELM_ERR_NOT_CONVERGED)
                throw ElmError(st, "training failed while tuning: " + ctx->last_error);
        };
        Tune best;
        double best_ms = 0.0;
        std::string key;
        if (count > 1) {
            // a batched call: the lanes of its back halves, by the call's time
            key = tune_batch_key(o.precision, count);
            ctx->tune.erase(key);
            elm_train_opts oo = o;
            oo.flags &= ~ELM_FLAG_PHASE_TIMING;
            run(oo);   // workspaces
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            ELM_CUDA(cudaEventCreate(&e0));
            ELM_CUDA(cudaEventCreate(&e1));
            best_ms = INFINITY;
            best.lanes = 4;
            for (int ln : {1, 2, 4, 8}) {
                oo.lanes = ln;
                ELM_CUDA(cudaEventRecord(e0, ctx->stream));
                run(oo);   // returns once every lane is done
                ELM_CUDA(cudaEventRecord(e1, ctx->stream));
                ELM_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                ELM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best.lanes = ln;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        } else {
            // one problem: the panels' cluster size and width by the factor
            // phase, the tensor kernels' pipeline depth by their own phases
            key = tune_key(o.precision, probs[0]);
            ctx->tune.erase(key);
            const bool mixed = o.precision == ELM_PREC_MIXED;
            elm_train_opts oo = o;
            oo.flags |= ELM_FLAG_PHASE_TIMING;
            run(oo);   // workspaces
            std::vector<std::pair<int, int>> combos;
            for (int cs : {8, 16})
                for (int nb : {16, 24, 32})
                    if (mixed || nb <= 24) combos.push_back({cs, nb});
            double fbest = INFINITY, hsum[4] = {0, 0, 0, 0}, gsum[4] = {0, 0, 0, 0};
            int cnt[4] = {0, 0, 0, 0};
            for (size_t i = 0; i < combos.size(); i++) {
                Tune t;
                t.panel_cs = combos[i].first;
                t.panel_nb = combos[i].second;
                const int stg = i % 2 == 0 ? 3 : 2;
                if (mixed) t.hid_stages = t.gram_stages = stg;
                ctx->tune[key] = t;
                for (double &x : ctx->phase_ms) x = 0.0;
                run(oo);
                if (ctx->phase_ms[2] < fbest) {
                    fbest = ctx->phase_ms[2];
                    best.panel_cs = t.panel_cs;
                    best.panel_nb = t.panel_nb;
                }
                hsum[stg] += ctx->phase_ms[0];
                gsum[stg] += ctx->phase_ms[1];
                cnt[stg]++;
            }
            best_ms = fbest;
            if (mixed && cnt[2] > 0 && cnt[3] > 0) {
                const double h2 = hsum[2] / cnt[2], h3 = hsum[3] / cnt[3];
                const double g2 = gsum[2] / cnt[2], g3 = gsum[3] / cnt[3];
                best.hid_stages = h2 < h3 ? 2 : 3;
                best.gram_stages = g2 < g3 ? 2 : 3;
                best_ms += (h2 < h3 ? h2 : h3) + (g2 < g3 ? g2 : g3);
            }
            for (double &x : ctx->phase_ms) x = 0.0;
        }
        ctx->tune[key] = best;
        if (cache_path) tune_store(cache_path, key, best);
        if (out) {
            out->panel_cluster = best.panel_cs;
            out->panel_width = best.panel_nb;
            out->hidden_stages = best.hid_stages;
            out->gram_stages = best.gram_stages;
            out->lanes = best.lanes;
            out->reserved = 0;
            out->best_ms = best_ms;
        }
    });
}

int elm_autotune_load(elm_ctx *ctx, const char *cache_path) {
    if (!ctx || !cache_path) return ELM_ERR_ARG;
    return guarded(ctx, [&] {
        FILE *f = fopen(cache_path, "r");
        require(f != nullptr, "cannot open the autotune cache file");
        char buf[512];
        while (fgets(buf, sizeof buf, f)) {
            std::string k;
            Tune t;
            if (tune_parse(buf, k, t)) ctx->tune[k] = t;
        }
        fclose(f);
    });
}

int elm_phase_times(elm_ctx *ctx, double *ms_out, int max_phases) {
    if (!ctx || (max_phases > 0 && !ms_out)) return -ELM_ERR_ARG;
    for (int i = 0; i < ELM_NUM_PHASES; i++) {
        if (i < max_phases) ms_out[i] = ctx->phase_ms[i];
        ctx->phase_ms[i] = 0.0;
    }
    return ELM_NUM_PHASES;
}

const char *elm_phase_name(int phase) {
    return (phase >= 0 && phase < ELM_NUM_PHASES) ? kPhaseName[phase] : "";
}

int64_t elm_launch_counter(void) { return g_launches.load(); }

int elm_predict(elm_ctx *ctx, const void *X, int x_dtype, int64_t N, int64_t n, int64_t ldx,
                const double *W, int64_t ldw, const double *b, const double *a, int64_t L,
                int act, const double *beta, int64_t m, int64_t ldb, double *Y, int64_t ldy) {
    if (!ctx) return ELM_ERR_ARG;
    return guarded(ctx, [&] {
        check_dims(N, n, ldx, L, ldw);
        require(X && W && b && beta && Y, "NULL pointer");
        require(m >= 1 && ldb >= m && ldy >= m, "m, ldb or ldy");
        require(x_dtype == ELM_F32 || x_dtype == ELM_F64, "x_dtype");
        require(act == ELM_ACT_SIGMOID || act == ELM_ACT_TANH, "act");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const size_t xsz = x_dtype == ELM_F64 ? 8 : 4;
        In Xs, Ws, bs, as, Bs;
        double *out = nullptr;
        const bool dev_out = on_device(Y);
        with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
            Xs = stage(ar, s, X, N, n, ldx, xsz);
            Ws = stage(ar, s, W, n, L, ldw, 8);
            bs = stage(ar, s, b, 1, L, L, 8);
            as = stage(ar, s, a, 1, L, L, 8);
            Bs = stage(ar, s, beta, L, m, ldb, 8);
            out = dev_out ? Y : ar.take<double>(N * m);
        });
        const int64_t ldo = dev_out ? ldy : m;
        predict_f64(s, Xs.p, x_dtype, N, n, Xs.ld, (const double *)Ws.p, Ws.ld,
                    (const double *)bs.p, (const double *)as.p, L, act,
                    (const double *)Bs.p, Bs.ld, m, out, ldo);
        if (!dev_out) {
            copy2d(Y, ldy * 8, out, m * 8, m * 8, N,
                                       cudaMemcpyDeviceToHost, s);
            ELM_CUDA(cudaStreamSynchronize(s));
        } else if (Xs.host || Ws.host || bs.host || as.host || Bs.host) {
            ELM_CUDA(cudaStreamSynchronize(s));
        }
    });
}

int elm_rows_create(elm_ctx *ctx, const void *X, int x_dtype, int64_t N, int64_t n,
                    int64_t ldx, const double *W, int64_t ldw, const double *b,
                    const double *a, int64_t L, int act, const double *T, int64_t m,
                    int64_t ldt, int precision, elm_rows **out) {
    if (!ctx || !out) return ELM_ERR_ARG;
    *out = nullptr;
    elm_rows *h = nullptr;
    int st = guarded(ctx, [&] {
        check_dims(N, n, ldx, L, ldw);
        require(X && W && b && T, "X, W, b and T must be non-NULL");
        require(m >= 1 && ldt >= m, "m or ldt");
        require(x_dtype == ELM_F32 || x_dtype == ELM_F64, "x_dtype");
        require(act == ELM_ACT_SIGMOID || act == ELM_ACT_TANH, "act");
        require(precision == ELM_PREC_FP64 || precision == ELM_PREC_MIXED, "precision");
        ELM_CUDA(cudaSetDevice(ctx->device));
        h = new elm_rows;
        h->ctx = ctx;
        // a mixed row block larger than the mixed products hold: FP64
        h->precision = precision == ELM_PREC_MIXED && !mixed_fits(N, n) ? ELM_PREC_FP64 : precision;
        h->N = N;
        h->L = L;
        h->m = m;
        rows_build(h, X, x_dtype, n, ldx, W, ldw, b, a, act, T, ldt);
    });
    if (st != ELM_OK) {
        delete h;
        return st;
    }
    *out = h;
    return ELM_OK;
}

int elm_rows_gram(elm_rows *h, double *S, int64_t lds, double *Z, int64_t ldz) {
    if (!h) return ELM_ERR_ARG;
    elm_ctx *ctx = h->ctx;
    return guarded(ctx, [&] {
        require(S && Z && lds >= h->L && ldz >= h->m, "S, Z, lds or ldz");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const int64_t L = h->L, m = h->m;
        copy2d(S, lds * 8, h->S, L * 8, L * 8, L,
               on_device(S) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        copy2d(Z, ldz * 8, h->Z, m * 8, m * 8, L,
               on_device(Z) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        ELM_CUDA(cudaStreamSynchronize(s));
    });
}

int elm_rows_residual(elm_rows *h, const double *beta, int64_t ldb, double *Gres, int64_t ldr) {
    if (!h) return ELM_ERR_ARG;
    elm_ctx *ctx = h->ctx;
    return guarded(ctx, [&] {
        require(beta && Gres && ldb >= h->m && ldr >= h->m, "beta, Gres, ldb or ldr");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const int64_t N = h->N, L = h->L, m = h->m;
        copy2d(h->beta, m * 8, beta, ldb * 8, m * 8, L,
               on_device(beta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        double *G = nullptr;
        const bool dev_out = on_device(Gres) && ldr == m;
        with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
            G = dev_out ? Gres : ar.take<double>(L * m);
        });
        if (h->precision == ELM_PREC_MIXED) {
            resid_df(s, h->Hdf, L, N, h->beta, m, h->T, m, h->Rres, h->betaT);
            htr_df(s, h->Hdf, L, N, h->Rres, m, G, h->part, h->nsplit);
        } else {
            resid_f64(s, h->Ht, N, L, N, h->beta, m, h->T, m, h->Rres);
            htr_f64(s, h->Ht, N, L, N, h->Rres, m, G, h->part, h->nsplit);
        }
        if (!dev_out)
            copy2d(Gres, ldr * 8, G, m * 8, m * 8, L,
                   on_device(Gres) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        ELM_CUDA(cudaStreamSynchronize(s));
    });
}

int elm_rows_destroy(elm_rows *h) {
    if (!h) return ELM_OK;
    cudaSetDevice(h->ctx->device);
    if (h->ctx->stream) cudaStreamSynchronize(h->ctx->stream);
    delete h;
    return ELM_OK;
}

int elm_factor_gram(elm_ctx *ctx, const double *S, int64_t lds, int64_t L, int64_t m,
                    int precision, double tol_rank, elm_factor **out, int64_t *rank_out) {
    if (!ctx || !out) return ELM_ERR_ARG;
    *out = nullptr;
    elm_factor *f = nullptr;
    int st = guarded(ctx, [&] {
        require(S && rank_out, "S and rank_out must be non-NULL");
        require(L >= 1 && L <= ELM_MAX_L && lds >= L && m >= 1, "L, lds or m");
        require(precision == ELM_PREC_FP64 || precision == ELM_PREC_MIXED, "precision");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const bool mixed = precision == ELM_PREC_MIXED;
        const double tau64 = (double)L * ldexp(1.0, -52);
        const double tau = tol_rank > 0.0 ? tol_rank : (mixed ? fmax(tau64, ldexp(1.0, -32)) : tau64);
        f = new elm_factor;
        f->ctx = ctx;
        f->L = L;
        f->m = m;
        double *R = nullptr, *Rt = nullptr;
        int32_t *perm = nullptr;
        auto carve = [&](Arena &ar) {
            R = ar.take<double>(L * tri_ld(L));
            Rt = ar.take<double>(L * tri_ld(L));
            perm = ar.take<int32_t>(L);
            f->stage = ar.take<double>(L * m);
            f->out = ar.take<double>(L * m);
        };
        Arena plan;
        carve(plan);
        if (cudaMalloc(&f->mem.p, plan.used) != cudaSuccess) {
            cudaGetLastError();
            f->mem.p = nullptr;
            throw ElmError(ELM_ERR_NOMEM, "cudaMalloc of the factor failed");
        }
        f->mem.size = plan.used;
        Arena own;
        own.base = f->mem.p;
        own.cap = f->mem.size;
        carve(own);
        In Sd;
        FactorWs fw;
        with_arena(&ctx->ws, &ctx->ws_size, s, [&](Arena &ar) {
            Sd = stage(ar, s, S, L, L, lds, 8);
            fw = factor_ws_carve(ar, L);
        });
        factor_pivoted(s, (const double *)Sd.p, Sd.ld, L, tau, fw, R, Rt, tri_ld(L),
                       ctx->sm_count, mixed);
        int32_t fl = 0;
        double stop_val = 0.0;
        const int64_t r = read_rank(s, fw, &fl, &stop_val);
        if (fl & 2) throw ElmError(ELM_ERR_TIMEOUT, "factorisation wait expired");
        if (fl & 1) throw ElmError(ELM_ERR_NUMERIC, "non-finite Gram matrix");
        if (mixed && tol_rank <= 0.0 && r < L && stop_val > tau64)
            throw ElmError(ELM_ERR_NUMERIC,
                           "mixed rank decision unsettled: a rejected pivot lies above L 2^-52; "
                           "factor the FP64 Gram");
        ELM_CUDA(cudaMemcpyAsync(perm, fw.perm, sizeof(int32_t) * L, cudaMemcpyDeviceToDevice, s));
        f->r = r;
        f->sv = solver_prepare(ctx, s, R, Rt, tri_ld(L), perm, r, L, m, &f->aux.p, &f->aux.size);
        ELM_CUDA(cudaStreamSynchronize(s));
        *rank_out = r;
    });
    if (st != ELM_OK) {
        delete f;
        return st;
    }
    *out = f;
    return ELM_OK;
}

int elm_factor_solve(elm_factor *f, const double *Z, int64_t ldz, int64_t mc, double *out,
                     int64_t ldo) {
    if (!f) return ELM_ERR_ARG;
    elm_ctx *ctx = f->ctx;
    return guarded(ctx, [&] {
        require(Z && out && mc >= 1 && mc <= f->m && ldz >= mc && ldo >= mc, "Z, out or mc");
        ELM_CUDA(cudaSetDevice(ctx->device));
        cudaStream_t s = ctx->stream;
        const int64_t L = f->L;
        copy2d(f->stage, mc * 8, Z, ldz * 8, mc * 8, L,
               on_device(Z) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        solver_apply(s, f->sv, f->stage, mc, f->out, mc, mc);
        if (solver_timed_out(s, f->sv)) throw ElmError(ELM_ERR_TIMEOUT, "solve wait expired");
        copy2d(out, ldo * 8, f->out, mc * 8, mc * 8, L,
               on_device(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        ELM_CUDA(cudaStreamSynchronize(s));
    });
}

int elm_factor_destroy(elm_factor *f) {
    if (!f) return ELM_OK;
    cudaSetDevice(f->ctx->device);
    if (f->ctx->stream) cudaStreamSynchronize(f->ctx->stream);
    delete f;
    return ELM_OK;
}

}  // extern "C"
