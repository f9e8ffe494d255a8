/*
 * Plain FP64 CPU oracle for rank-based pseudoinverse ELM training.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library calls, links or
 * includes this file; only the test-suite, the GPU smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, helper or
 * constant with the CUDA path.
 *
 * Every matrix is row-major FP64.  Loops are plain and in the order the
 * definitions state; the only parallelism is OpenMP over independent output
 * rows, so every result is independent of the thread count.  Build with
 * -ffp-contract=off so x86 and Arm round identically.
 *
 * Paper: Ragala & Bharadwaja Kumar, "Rank Based Pseudoinverse Computation in
 * Extreme Learning Machine for large Datasets" (arXiv 2011.02436).
 *
 * Functions and the passage each follows:
 *   orc_hidden      H_ij = a_j g(x_i . w_j + b_j)   Eq. 1, Eq. 3; Alg. 1 step 2
 *   orc_gram        S = H^T H, Z = H^T T            Eqs. 9-13 (the Gram blocks)
 *   orc_pivchol     permutation P, rank r, H P = [H1 H2]
 *                                                   Eq. 6; Alg. 1 steps 3-4
 *   orc_frsolve     beta = H^+ T through the full-rank factorisation
 *                   H P = H1 [I K]                  Eq. 5, Eq. 7 (reading below)
 *   orc_train       steps above + 2 refinement steps      Alg. 1
 *   orc_pinv        explicit H^+ (tiny inputs)      Eq. 5
 *   orc_predict     Y = H beta                      Section 2, step 3
 *   orc_block_rbp   the paper's block formulae for a full-rank split
 *                   (A, B, C, D; transposition fixed)     Eqs. 19-23
 *
 * Reading of the paper used here (the paper inverts H^T H, Eq. 8, which is
 * singular whenever r < L): the columns of H P split into H1 (N x r,
 * independent) and H2 = H1 K (dependent), K = (H1^T H1)^{-1} H1^T H2.  Then
 * H P = H1 [I K] is a full-rank factorisation and
 *     H^+ = P [I; K^T] (I + K K^T)^{-1} (H1^T H1)^{-1} H1^T,
 * which is exactly the Moore-Penrose inverse for every rank and reduces to
 * Eq. 8 when r = L.  H1^T H1 = R11^T R11 and H1^T H2 = R11^T R12 come from a
 * diagonal-pivoted Cholesky factorisation of the Gram matrix.
 *
 * Parity pins: see tests/test_oracle_pins.py (Penrose conditions, Eq. 8
 * closed form, SVD pseudoinverse, duplicate-neuron closed form, invariants,
 * a hand-worked pivoted Cholesky, the Eqs. 19-23 block identity).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ACT_SIGMOID 0
#define ORC_ACT_TANH 1

static double orc_g(double z, int act)
{
    if (act == ORC_ACT_TANH) return tanh(z);
    return 1.0 / (1.0 + exp(-z));          /* logistic sigmoid, Section 4 */
}

/* H (N x L) = a_j * g(sum_k X[i,k] W[k,j] + b_j); the sum runs k = 0..n-1
 * and b_j is added last.  a may be NULL (all ones).  Eq. 1, Eq. 3. */
void orc_hidden(const double *X, int64_t N, int64_t n, const double *W,
                int64_t L, const double *b, const double *a, int act,
                double *H)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        double *z = H + i * L;
        for (int64_t j = 0; j < L; j++) z[j] = 0.0;
        for (int64_t k = 0; k < n; k++) {
            double x = X[i * n + k];
            const double *w = W + k * L;
            for (int64_t j = 0; j < L; j++) z[j] += x * w[j];
        }
        for (int64_t j = 0; j < L; j++) {
            double s = a ? a[j] : 1.0;
            z[j] = s * orc_g(z[j] + b[j], act);
        }
    }
}

/* S (L x L, both triangles) = H^T H and Z (L x m) = H^T T; every entry sums
 * over samples i = 0..N-1 in ascending order.  Eqs. 9-13. */
void orc_gram(const double *H, int64_t N, int64_t L, const double *T,
              int64_t m, double *S, double *Z)
{
    const int64_t JB = 32;
#pragma omp parallel for schedule(dynamic)
    for (int64_t j0 = 0; j0 < L; j0 += JB) {
        int64_t j1 = j0 + JB < L ? j0 + JB : L;
        for (int64_t j = j0; j < j1; j++) {
            for (int64_t l = 0; l <= j; l++) S[j * L + l] = 0.0;
            for (int64_t c = 0; c < m; c++) Z[j * m + c] = 0.0;
        }
        for (int64_t i = 0; i < N; i++) {
            const double *h = H + i * L;
            const double *t = T ? T + i * m : NULL;
            for (int64_t j = j0; j < j1; j++) {
                double hj = h[j];
                double *s = S + j * L;
                for (int64_t l = 0; l <= j; l++) s[l] += hj * h[l];
                if (t)
                    for (int64_t c = 0; c < m; c++) Z[j * m + c] += hj * t[c];
            }
        }
    }
    for (int64_t j = 0; j < L; j++)
        for (int64_t l = j + 1; l < L; l++) S[j * L + l] = S[l * L + j];
}

/*
 * Rank-revealing diagonal-pivoted Cholesky of the Gram matrix S (L x L).
 * Eq. 6 and Alg. 1 steps 3-4: choose a permutation P that moves linearly
 * independent columns first, find the rank r, split H P = [H1 H2].
 *
 * 1. Equilibrate: d_j = S_jj, s_j = 1/sqrt(d_j) (0 if d_j <= 0),
 *    A = diag(s) S diag(s), computed as (S_jl * s_j) * s_l.
 * 2. Right-looking Cholesky with diagonal pivoting on A: at step k take the
 *    largest remaining diagonal (ties: lowest original column index); stop
 *    with r = k when it is <= tau.
 * 3. Unscale: R = Rtilde diag(sqrt(d_perm)).
 * Outputs perm[L] (first r = columns of H1, the rest in ascending original
 * index), R (L x L row-major; rows 0..r-1 hold [R11 R12] in pivot order,
 * the rest zero).  Returns r.
 */
int64_t orc_pivchol(const double *S, int64_t L, double tau, int64_t *perm,
                    double *R)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)(L * L));
    double *d = (double *)malloc(sizeof(double) * (size_t)L);
    double *s = (double *)malloc(sizeof(double) * (size_t)L);
    for (int64_t j = 0; j < L; j++) {
        d[j] = S[j * L + j];
        s[j] = d[j] > 0.0 ? 1.0 / sqrt(d[j]) : 0.0;
        perm[j] = j;
    }
    for (int64_t j = 0; j < L; j++)
        for (int64_t l = 0; l < L; l++) A[j * L + l] = (S[j * L + l] * s[j]) * s[l];
    memset(R, 0, sizeof(double) * (size_t)(L * L));

    int64_t r = L;
    for (int64_t k = 0; k < L; k++) {
        int64_t p = k;
        for (int64_t j = k + 1; j < L; j++) {
            double aj = A[j * L + j], ap = A[p * L + p];
            if (aj > ap || (aj == ap && perm[j] < perm[p])) p = j;
        }
        if (!(A[p * L + p] > tau)) { r = k; break; }
        if (p != k) {
            for (int64_t x = 0; x < L; x++) {          /* swap rows k, p */
                double t = A[k * L + x]; A[k * L + x] = A[p * L + x]; A[p * L + x] = t;
            }
            for (int64_t x = 0; x < L; x++) {          /* swap columns k, p */
                double t = A[x * L + k]; A[x * L + k] = A[x * L + p]; A[x * L + p] = t;
            }
            for (int64_t i = 0; i < k; i++) {          /* computed rows of R */
                double t = R[i * L + k]; R[i * L + k] = R[i * L + p]; R[i * L + p] = t;
            }
            int64_t t = perm[k]; perm[k] = perm[p]; perm[p] = t;
        }
        double rkk = sqrt(A[k * L + k]);
        R[k * L + k] = rkk;
        for (int64_t j = k + 1; j < L; j++) R[k * L + j] = A[k * L + j] / rkk;
        for (int64_t j = k + 1; j < L; j++)
            for (int64_t l = k + 1; l < L; l++)
                A[j * L + l] -= R[k * L + j] * R[k * L + l];
    }
    /* the columns left out of H1 in ascending original index */
    for (int64_t a = r; a < L; a++)
        for (int64_t c = a + 1; c < L; c++)
            if (perm[c] < perm[a]) {
                int64_t t = perm[a]; perm[a] = perm[c]; perm[c] = t;
                for (int64_t i = 0; i < r; i++) {
                    double u = R[i * L + a]; R[i * L + a] = R[i * L + c]; R[i * L + c] = u;
                }
            }
    for (int64_t i = 0; i < r; i++)
        for (int64_t j = i; j < L; j++) R[i * L + j] *= sqrt(d[perm[j]]);
    free(A); free(d); free(s);
    return r;
}

/* x = U^{-1} b for upper-triangular U (r x r, leading dim ldu); b, x are
 * r x q (ld q); in place on b. */
static void orc_solve_upper(const double *U, int64_t ldu, int64_t r,
                            double *B, int64_t q)
{
    for (int64_t i = r - 1; i >= 0; i--)
        for (int64_t c = 0; c < q; c++) {
            double v = B[i * q + c];
            for (int64_t j = i + 1; j < r; j++) v -= U[i * ldu + j] * B[j * q + c];
            B[i * q + c] = v / U[i * ldu + i];
        }
}

/* x = U^{-T} b (forward substitution with U^T lower-triangular). */
static void orc_solve_upper_t(const double *U, int64_t ldu, int64_t r,
                              double *B, int64_t q)
{
    for (int64_t i = 0; i < r; i++)
        for (int64_t c = 0; c < q; c++) {
            double v = B[i * q + c];
            for (int64_t j = 0; j < i; j++) v -= U[j * ldu + i] * B[j * q + c];
            B[i * q + c] = v / U[i * ldu + i];
        }
}

/* Unpivoted Cholesky M = U^T U (M r x r SPD); U written to Uout (r x r). */
static int orc_chol(const double *M, int64_t r, double *U)
{
    memset(U, 0, sizeof(double) * (size_t)(r * r));
    for (int64_t k = 0; k < r; k++) {
        double v = M[k * r + k];
        for (int64_t i = 0; i < k; i++) v -= U[i * r + k] * U[i * r + k];
        if (!(v > 0.0)) return -1;
        double ukk = sqrt(v);
        U[k * r + k] = ukk;
        for (int64_t j = k + 1; j < r; j++) {
            double w = M[k * r + j];
            for (int64_t i = 0; i < k; i++) w -= U[i * r + k] * U[i * r + j];
            U[k * r + j] = w / ukk;
        }
    }
    return 0;
}

/*
 * beta (L x m) = H^+ Z-side solve through the full-rank factorisation:
 *   Zp = Z[perm[0..r-1], :]                         (H1^T T)
 *   K  = R11^{-1} R12                               (H2 = H1 K)
 *   c  = R11^{-1} R11^{-T} Zp                       ((H1^T H1)^{-1} H1^T T)
 *   y  = (I + K K^T)^{-1} c      (y = c when r = L)
 *   beta[perm[i]] = [y; K^T y][i]                   (Eq. 7: beta = [beta1; beta2])
 * R is the output of orc_pivchol.  Returns 0, or -1 if I + K K^T fails to
 * factor (it cannot in exact arithmetic: it is >= I).
 */
int orc_frsolve(const double *R, int64_t L, int64_t r, const int64_t *perm,
                const double *Z, int64_t m, double *beta)
{
    int64_t q = L - r;
    double *c = (double *)malloc(sizeof(double) * (size_t)(r * m + 1));
    for (int64_t i = 0; i < r; i++)
        for (int64_t t = 0; t < m; t++) c[i * m + t] = Z[perm[i] * m + t];
    orc_solve_upper_t(R, L, r, c, m);
    orc_solve_upper(R, L, r, c, m);
    double *K = NULL, *y = c;
    int rc = 0;
    if (q > 0) {
        K = (double *)malloc(sizeof(double) * (size_t)(r * q + 1));
        for (int64_t i = 0; i < r; i++)
            for (int64_t j = 0; j < q; j++) K[i * q + j] = R[i * L + r + j];
        orc_solve_upper(R, L, r, K, q);
        double *M = (double *)malloc(sizeof(double) * (size_t)(r * r));
        double *U = (double *)malloc(sizeof(double) * (size_t)(r * r));
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < r; i++)
            for (int64_t j = 0; j < r; j++) {
                double v = (i == j) ? 1.0 : 0.0;
                for (int64_t t = 0; t < q; t++) v += K[i * q + t] * K[j * q + t];
                M[i * r + j] = v;
            }
        rc = orc_chol(M, r, U);
        if (rc == 0) {
            orc_solve_upper_t(U, r, r, c, m);
            orc_solve_upper(U, r, r, c, m);
        }
        free(M); free(U);
    }
    for (int64_t i = 0; i < r; i++)
        for (int64_t t = 0; t < m; t++) beta[perm[i] * m + t] = y[i * m + t];
    for (int64_t j = 0; j < q; j++)
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t i = 0; i < r; i++) v += K[i * q + j] * y[i * m + t];
            beta[perm[r + j] * m + t] = v;
        }
    free(c);
    if (K) free(K);
    return rc;
}

/* Y (N x m) = H beta, sum over j ascending.  Section 2, step 3. */
void orc_matmul_hb(const double *H, int64_t N, int64_t L, const double *beta,
                   int64_t m, double *Y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++)
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t j = 0; j < L; j++) v += H[i * L + j] * beta[j * m + t];
            Y[i * m + t] = v;
        }
}

/* Default rank threshold on the unit-diagonal scale: L * 2^-52. */
double orc_default_tau(int64_t L) { return (double)L * ldexp(1.0, -52); }

/*
 * Full training (Alg. 1): hidden layer, Gram, pivoted rank decision,
 * full-rank solve, then `nrefine` correction steps
 *   Rres = T - H beta, G = H^T Rres, beta += frsolve(G)
 * (each correction lies in the row space of H, so beta stays the
 * minimum-norm solution).  tau <= 0 selects orc_default_tau(L).
 * H_out (N x L), perm (L), may be NULL.  Returns the rank, or -1 on failure.
 */
int64_t orc_train(const double *X, int64_t N, int64_t n, const double *W,
                  int64_t L, const double *b, const double *a, int act,
                  const double *T, int64_t m, double tau, int nrefine,
                  double *beta, int64_t *perm_out, double *H_out)
{
    double *H = H_out ? H_out : (double *)malloc(sizeof(double) * (size_t)(N * L));
    double *S = (double *)malloc(sizeof(double) * (size_t)(L * L));
    double *Z = (double *)malloc(sizeof(double) * (size_t)(L * m));
    double *R = (double *)malloc(sizeof(double) * (size_t)(L * L));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    if (tau <= 0.0) tau = orc_default_tau(L);
    orc_hidden(X, N, n, W, L, b, a, act, H);
    orc_gram(H, N, L, T, m, S, Z);
    int64_t r = orc_pivchol(S, L, tau, perm, R);
    int rc = orc_frsolve(R, L, r, perm, Z, m, beta);
    if (rc == 0 && nrefine > 0) {
        double *Y = (double *)malloc(sizeof(double) * (size_t)(N * m));
        double *dB = (double *)malloc(sizeof(double) * (size_t)(L * m));
        for (int it = 0; it < nrefine && rc == 0; it++) {
            orc_matmul_hb(H, N, L, beta, m, Y);
            for (int64_t i = 0; i < N * m; i++) Y[i] = T[i] - Y[i];
            orc_gram(H, N, L, Y, m, S, Z);   /* Z = H^T (T - H beta) */
            rc = orc_frsolve(R, L, r, perm, Z, m, dB);
            for (int64_t i = 0; i < L * m; i++) beta[i] += dB[i];
        }
        free(Y); free(dB);
    }
    if (perm_out) memcpy(perm_out, perm, sizeof(int64_t) * (size_t)L);
    if (!H_out) free(H);
    free(S); free(Z); free(R); free(perm);
    return rc == 0 ? r : -1;
}

/* Explicit H^+ (L x N) for an N x L matrix H: the full-rank solve with
 * Z = H^T, i.e. beta for T = I_N.  Returns the rank. */
int64_t orc_pinv(const double *H, int64_t N, int64_t L, double tau,
                 double *Hp)
{
    double *S = (double *)malloc(sizeof(double) * (size_t)(L * L));
    double *Z = (double *)malloc(sizeof(double) * (size_t)(L * N));
    double *R = (double *)malloc(sizeof(double) * (size_t)(L * L));
    double *I = (double *)calloc((size_t)(N * N), sizeof(double));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    for (int64_t i = 0; i < N; i++) I[i * N + i] = 1.0;
    if (tau <= 0.0) tau = orc_default_tau(L);
    orc_gram(H, N, L, I, N, S, Z);
    int64_t r = orc_pivchol(S, L, tau, perm, R);
    int rc = orc_frsolve(R, L, r, perm, Z, N, Hp);
    free(S); free(Z); free(R); free(I); free(perm);
    return rc == 0 ? r : -1;
}

/* Y (N x m) = g(X W + b) beta.  Section 2, step 3. */
void orc_predict(const double *X, int64_t N, int64_t n, const double *W,
                 int64_t L, const double *b, const double *a, int act,
                 const double *beta, int64_t m, double *Y)
{
    double *H = (double *)malloc(sizeof(double) * (size_t)(N * L));
    orc_hidden(X, N, n, W, L, b, a, act, H);
    orc_matmul_hb(H, N, L, beta, m, Y);
    free(H);
}

/* Inverse of an SPD matrix via unpivoted Cholesky (helper for the block
 * formulae below).  Returns -1 if not positive definite. */
static int orc_spd_inverse(const double *M, int64_t k, double *Minv)
{
    double *U = (double *)malloc(sizeof(double) * (size_t)(k * k));
    int rc = orc_chol(M, k, U);
    if (rc == 0) {
        memset(Minv, 0, sizeof(double) * (size_t)(k * k));
        for (int64_t i = 0; i < k; i++) Minv[i * k + i] = 1.0;
        orc_solve_upper_t(U, k, k, Minv, k);
        orc_solve_upper(U, k, k, Minv, k);
    }
    free(U);
    return rc;
}

/*
 * The paper's block route for a column split of a FULL-RANK H into
 * H1 = H[:, 0..r1-1] and H2 = H[:, r1..L-1] (Eqs. 19-23, with Eq. 19's
 * H1 read as H1^T and Eq. 21's B as (L-r1) x m):
 *   A = H2^T H2                       Eq. 20
 *   B = A^{-1} H2^T Y                 Eq. 21
 *   C = I_N - H2 A^{-1} H2^T          Eq. 22 (N x N)
 *   D = H1^T C H1                     Eq. 23
 *   beta1 = D^{-1} H1^T (Y - H2 B),  beta2 = B - A^{-1} H2^T H1 beta1  Eq. 19
 * Small inputs only (C is N x N).  Returns 0, or -1 when A or D is singular.
 */
int orc_block_rbp(const double *H, int64_t N, int64_t L, int64_t r1,
                  const double *Y, int64_t m, double *beta)
{
    int64_t q = L - r1;
    if (r1 <= 0 || q <= 0) return -1;
    double *A = (double *)malloc(sizeof(double) * (size_t)(q * q));
    double *Ai = (double *)malloc(sizeof(double) * (size_t)(q * q));
    double *B = (double *)malloc(sizeof(double) * (size_t)(q * m));
    double *C = (double *)malloc(sizeof(double) * (size_t)(N * N));
    double *D = (double *)malloc(sizeof(double) * (size_t)(r1 * r1));
    double *Di = (double *)malloc(sizeof(double) * (size_t)(r1 * r1));
    double *t1 = (double *)malloc(sizeof(double) * (size_t)(q * (N > m ? N : m)));
    double *t2 = (double *)malloc(sizeof(double) * (size_t)(N * (r1 > m ? r1 : m)));
    int rc = -1;
#define H1(i, j) H[(i) * L + (j)]
#define H2(i, j) H[(i) * L + r1 + (j)]
    for (int64_t a = 0; a < q; a++)                        /* Eq. 20 */
        for (int64_t c = 0; c < q; c++) {
            double v = 0.0;
            for (int64_t i = 0; i < N; i++) v += H2(i, a) * H2(i, c);
            A[a * q + c] = v;
        }
    if (orc_spd_inverse(A, q, Ai) != 0) goto done;
    for (int64_t a = 0; a < q; a++)                        /* H2^T Y */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t i = 0; i < N; i++) v += H2(i, a) * Y[i * m + t];
            t1[a * m + t] = v;
        }
    for (int64_t a = 0; a < q; a++)                        /* Eq. 21 */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t c = 0; c < q; c++) v += Ai[a * q + c] * t1[c * m + t];
            B[a * m + t] = v;
        }
    for (int64_t a = 0; a < q; a++)                        /* A^{-1} H2^T */
        for (int64_t i = 0; i < N; i++) {
            double v = 0.0;
            for (int64_t c = 0; c < q; c++) v += Ai[a * q + c] * H2(i, c);
            t1[a * N + i] = v;
        }
    for (int64_t i = 0; i < N; i++)                        /* Eq. 22 */
        for (int64_t k = 0; k < N; k++) {
            double v = 0.0;
            for (int64_t a = 0; a < q; a++) v += H2(i, a) * t1[a * N + k];
            C[i * N + k] = (i == k ? 1.0 : 0.0) - v;
        }
    for (int64_t i = 0; i < N; i++)                        /* C H1 */
        for (int64_t j = 0; j < r1; j++) {
            double v = 0.0;
            for (int64_t k = 0; k < N; k++) v += C[i * N + k] * H1(k, j);
            t2[i * r1 + j] = v;
        }
    for (int64_t a = 0; a < r1; a++)                       /* Eq. 23 */
        for (int64_t j = 0; j < r1; j++) {
            double v = 0.0;
            for (int64_t i = 0; i < N; i++) v += H1(i, a) * t2[i * r1 + j];
            D[a * r1 + j] = v;
        }
    if (orc_spd_inverse(D, r1, Di) != 0) goto done;
    for (int64_t i = 0; i < N; i++)                        /* Y - H2 B */
        for (int64_t t = 0; t < m; t++) {
            double v = Y[i * m + t];
            for (int64_t a = 0; a < q; a++) v -= H2(i, a) * B[a * m + t];
            t2[i * m + t] = v;
        }
    for (int64_t a = 0; a < r1; a++)                       /* H1^T (Y - H2 B) */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t i = 0; i < N; i++) v += H1(i, a) * t2[i * m + t];
            t1[a * m + t] = v;
        }
    for (int64_t a = 0; a < r1; a++)                       /* beta1, Eq. 19 */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t c = 0; c < r1; c++) v += Di[a * r1 + c] * t1[c * m + t];
            beta[a * m + t] = v;
        }
    for (int64_t i = 0; i < N; i++)                        /* H1 beta1 */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t a = 0; a < r1; a++) v += H1(i, a) * beta[a * m + t];
            t2[i * m + t] = v;
        }
    for (int64_t a = 0; a < q; a++)                        /* H2^T H1 beta1 */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t i = 0; i < N; i++) v += H2(i, a) * t2[i * m + t];
            t1[a * m + t] = v;
        }
    for (int64_t a = 0; a < q; a++)                        /* beta2, Eq. 19 */
        for (int64_t t = 0; t < m; t++) {
            double v = 0.0;
            for (int64_t c = 0; c < q; c++) v += Ai[a * q + c] * t1[c * m + t];
            beta[(r1 + a) * m + t] = B[a * m + t] - v;
        }
    rc = 0;
#undef H1
#undef H2
done:
    free(A); free(Ai); free(B); free(C); free(D); free(Di); free(t1); free(t2);
    return rc;
}
