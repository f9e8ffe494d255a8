// FP64 dense kernels of the plain path: hidden layer (Eq. 1, 3), Gram
// blocks (Eqs. 9-13), refinement residuals, fused prediction (Section 2,
// step 3) and a generic strided GEMM used by the solves.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM, so these
// kernels are bound by DFMA issue, not by HBM: each keeps a 4x4 register
// tile per thread fed from shared memory, and every output element is
// accumulated by one thread in a fixed order (no atomics), so results are
// deterministic and two bitwise-equal input columns give bitwise-equal
// outputs.
#include <math.h>

#include <type_traits>

#include "df_arith.cuh"
#include "elm_internal.cuh"

namespace elm {

namespace {

constexpr int TB = 64;   // output tile edge
constexpr int TK = 16;   // k-slab depth
constexpr int NT = 256;  // threads per block (16 x 16, 4 x 4 outputs each)

__device__ __forceinline__ double act_f64(double z, int act) {
    return act == ELM_ACT_TANH ? tanh(z) : 1.0 / (1.0 + exp(-z));
}

template <typename XT>
__device__ __forceinline__ double ld_x(const XT *p) { return (double)(*p); }

// ---------------------------------------------------------------- hidden
// Ht[j, i] = a_j g(sum_k X[i,k] W[k,j] + b_j); block = 64 neurons x 64
// samples; k runs in ascending slabs of 16.
template <typename XT>
__global__ void __launch_bounds__(NT)
hidden_f64_kernel(const XT *__restrict__ X, int64_t N, int64_t n, int64_t ldx,
                  const double *__restrict__ W, int64_t ldw,
                  const double *__restrict__ b, const double *__restrict__ a,
                  int64_t L, int act, double *__restrict__ Ht, int64_t ldh) {
    __shared__ double Ws[TK][TB];
    __shared__ double Xs[TK][TB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * TB, j0 = (int64_t)blockIdx.y * TB;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < n; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TB; e += NT) {
            int kk = e / TB, jj = e % TB;
            int64_t k = k0 + kk, j = j0 + jj;
            Ws[kk][jj] = (k < n && j < L) ? W[k * ldw + j] : 0.0;
            int ii = e / TK, kx = e % TK;
            int64_t i = i0 + ii, k2 = k0 + kx;
            Xs[kx][ii] = (i < N && k2 < n) ? ld_x(X + i * ldx + k2) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double w[4], x[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                w[q] = Ws[kk][ty + 16 * q];
                x[q] = Xs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[p][q] = fma(w[p], x[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; p++) {
        int64_t j = j0 + ty + 16 * p;
        if (j >= L) continue;
        double bj = b[j], aj = a ? a[j] : 1.0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int64_t i = i0 + tx + 16 * q;
            if (i < N) Ht[j * ldh + i] = aj * act_f64(acc[p][q] + bj, act);
        }
    }
}

// ---------------------------------------------------------------- Gram
// Lower tiles of the Gram of the augmented rows [Ht ; T^T] over one k-range
// (split p of nsplit), written to part[p].  Row j < L is Ht[j, :], row
// L + c is T[:, c].
__device__ __forceinline__ double aug(const double *Ht, int64_t ldh, int64_t L,
                                      const double *T, int64_t ldt, int64_t j,
                                      int64_t i) {
    return j < L ? Ht[j * ldh + i] : T[i * ldt + (j - L)];
}

__global__ void __launch_bounds__(NT)
gram_f64_kernel(const double *__restrict__ Ht, int64_t ldh, int64_t L,
                int64_t N, const double *__restrict__ T, int64_t ldt, int64_t m,
                double *__restrict__ part, int64_t chunk) {
    __shared__ double As[TK][TB + 1];
    __shared__ double Bs[TK][TB + 1];
    const int64_t Lt = L + m;
    // triangular tile index -> (J >= I)
    int64_t t = blockIdx.x;
    int64_t J = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (J * (J + 1) / 2 > t) J--;
    while ((J + 1) * (J + 2) / 2 <= t) J++;
    int64_t I = t - J * (J + 1) / 2;
    const int64_t r0 = J * TB, c0 = I * TB;
    const int64_t kb = (int64_t)blockIdx.y * chunk;
    const int64_t ke = min(N, kb + chunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TB; e += NT) {
            int rr = e / TK, kk = e % TK;
            int64_t k = k0 + kk;
            int64_t jr = r0 + rr, jc = c0 + rr;
            As[kk][rr] = (k < ke && jr < Lt) ? aug(Ht, ldh, L, T, ldt, jr, k) : 0.0;
            Bs[kk][rr] = (k < ke && jc < Lt) ? aug(Ht, ldh, L, T, ldt, jc, k) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double u[4], v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                u[q] = As[kk][ty + 16 * q];
                v[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[p][q] = fma(u[p], v[q], acc[p][q]);
        }
        __syncthreads();
    }
    double *out = part + (int64_t)blockIdx.y * Lt * Lt;
#pragma unroll
    for (int p = 0; p < 4; p++) {
        int64_t j = r0 + ty + 16 * p;
        if (j >= Lt) continue;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int64_t l = c0 + tx + 16 * q;
            if (l < Lt && l <= j) out[j * Lt + l] = acc[p][q];
        }
    }
}

// Sum the splits in ascending order and scatter into S (both triangles) and Z.
__global__ void gram_reduce_kernel(const double *__restrict__ part, int nsplit,
                                   int64_t L, int64_t m, double *__restrict__ S,
                                   int64_t lds, double *__restrict__ Z,
                                   int64_t ldz) {
    const int64_t Lt = L + m;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = Lt * Lt;
    for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e / Lt, l = e % Lt;
        if (l > j || l >= L) continue;
        double v = 0.0;
        for (int p = 0; p < nsplit; p++) v += part[(int64_t)p * total + e];
        if (j < L) {
            S[j * lds + l] = v;
            S[l * lds + j] = v;
        } else {
            Z[l * ldz + (j - L)] = v;
        }
    }
}

// ---------------------------------------------------------------- GEMM
__global__ void __launch_bounds__(NT)
gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                const double *__restrict__ A, int64_t sAm, int64_t sAk,
                const double *__restrict__ B, int64_t sBk, int64_t sBn,
                double beta, double *__restrict__ C, int64_t ldc) {
    __shared__ double As[TK][TB + 1];
    __shared__ double Bs[TK][TB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * TB, n0 = (int64_t)blockIdx.x * TB;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < K; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TB; e += NT) {
            int rr = e / TK, kk = e % TK;
            int64_t k = k0 + kk, i = m0 + rr;
            As[kk][rr] = (k < K && i < M) ? A[i * sAm + k * sAk] : 0.0;
            int kk2 = e / TB, cc = e % TB;
            int64_t k2 = k0 + kk2, j = n0 + cc;
            Bs[kk2][cc] = (k2 < K && j < N) ? B[k2 * sBk + j * sBn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double u[4], v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                u[q] = As[kk][ty + 16 * q];
                v[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[p][q] = fma(u[p], v[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; p++) {
        int64_t i = m0 + ty + 16 * p;
        if (i >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int64_t j = n0 + tx + 16 * q;
            if (j >= N) continue;
            double v = alpha * acc[p][q];
            C[i * ldc + j] = beta == 0.0 ? v : v + beta * C[i * ldc + j];
        }
    }
}

// ---------------------------------------------------------------- residual
// R[i, c] = T[i, c] - sum_j Ht[j, i] beta[j, c]; one thread per sample, 8
// target columns per grid.y slice, j ascending.
constexpr int RC = 8;
__global__ void __launch_bounds__(128)
resid_f64_kernel(const double *__restrict__ Ht, int64_t ldh, int64_t L,
                 int64_t N, const double *__restrict__ beta, int64_t m,
                 const double *__restrict__ T, int64_t ldt,
                 double *__restrict__ R) {
    __shared__ double Bs[64][RC];
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int c0 = blockIdx.y * RC;
    double acc[RC] = {};
    for (int64_t j0 = 0; j0 < L; j0 += 64) {
        for (int e = threadIdx.x; e < 64 * RC; e += 128) {
            int jj = e / RC, cc = e % RC;
            int64_t j = j0 + jj;
            Bs[jj][cc] = (j < L && c0 + cc < m) ? beta[j * m + c0 + cc] : 0.0;
        }
        __syncthreads();
        if (i < N) {
            int64_t jn = min((int64_t)64, L - j0);
            for (int jj = 0; jj < jn; jj++) {
                double h = Ht[(j0 + jj) * ldh + i];
#pragma unroll
                for (int c = 0; c < RC; c++) acc[c] = fma(h, Bs[jj][c], acc[c]);
            }
        }
        __syncthreads();
    }
    if (i < N)
#pragma unroll
        for (int c = 0; c < RC; c++)
            if (c0 + c < m) R[i * m + c0 + c] = T[i * ldt + c0 + c] - acc[c];
}

// G[j, c] (split p) = sum_{i in split p} Ht[j, i] R[i, c]: one warp per
// neuron j, lane l takes i = l, l+32, ... then a fixed shuffle tree.
__global__ void __launch_bounds__(256)
htr_f64_kernel(const double *__restrict__ Ht, int64_t ldh, int64_t L,
               int64_t N, const double *__restrict__ R, int64_t m,
               double *__restrict__ part, int64_t chunk) {
    __shared__ double Rs[256][RC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + warp;
    const int c0 = blockIdx.z * RC;
    const int64_t ib = (int64_t)blockIdx.y * chunk, ie = min(N, ib + chunk);
    double acc[RC] = {};
    for (int64_t i0 = ib; i0 < ie; i0 += 256) {
        for (int e = threadIdx.x; e < 256 * RC; e += 256) {
            int ii = e / RC, cc = e % RC;
            int64_t i = i0 + ii;
            Rs[ii][cc] = (i < ie && c0 + cc < m) ? R[i * m + c0 + cc] : 0.0;
        }
        __syncthreads();
        if (j < L) {
            for (int ii = lane; ii < 256; ii += 32) {
                int64_t i = i0 + ii;
                double h = i < ie ? Ht[j * ldh + i] : 0.0;
#pragma unroll
                for (int c = 0; c < RC; c++) acc[c] = fma(h, Rs[ii][c], acc[c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < RC; c++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0 && j < L)
#pragma unroll
        for (int c = 0; c < RC; c++)
            if (c0 + c < m) part[((int64_t)blockIdx.y * L + j) * m + c0 + c] = acc[c];
}

// The refinement products of the mixed form with H (N x L, sample-major)
// held as double-float pairs: Rd = T - H beta (pairs) and G = H^T Rd, every
// product a TwoProduct and every sum a TwoSum on the FP32 pipes (about
// 2^-44 relative), so the residual is as accurate as the H it reads.  RC
// (a compile-time count >= the targets) keeps the accumulators in
// registers.

// betaT[c, j] = beta[j, c0 + c] as pairs (c < mc)
__global__ void beta_pairs_kernel(const double *__restrict__ beta, int64_t L, int64_t m,
                                  int64_t c0, int64_t mc, df::F2 *__restrict__ betaT) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L * mc) return;
    const int64_t c = e / L, j = e % L;
    betaT[e] = df::d2df(beta[j * m + c0 + c]);
}

// Rd[i, :] = T[i, :] - H[i, :] beta: one warp per SPW samples, lanes over
// the neurons (coalesced rows of H), warp reductions.  The CTA stages betaT
// in tiles of JT neurons in shared memory, so each value is fetched from L2
// once per CTA and reused by its 8 SPW samples; at most 128 registers keep
// two CTAs per SM.
template <int RC>
constexpr int spw_for() { return RC <= 10 ? 4 : (RC <= 20 ? 2 : 1); }   // register budget
template <int RC>
__host__ __device__ constexpr int rjt_for() { return RC <= 16 ? 256 : 128; }                // <= 32 KB of tile
template <int RC, int SPW = spw_for<RC>()>
__global__ void __launch_bounds__(256, 2)
resid_df_kernel(const df::F2 *__restrict__ H, int64_t L, int64_t N,
                const df::F2 *__restrict__ betaT, int64_t m, int64_t c0, int mc,
                const double *__restrict__ T, int64_t ldt, df::F2 *__restrict__ Rd) {
    constexpr int JT = rjt_for<RC>();
    __shared__ df::F2 bs[RC][JT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * 8 + warp) * SPW;
    float ah[SPW][RC], al[SPW][RC];
#pragma unroll
    for (int q = 0; q < SPW; q++)
#pragma unroll
        for (int c = 0; c < RC; c++) ah[q][c] = al[q][c] = 0.f;
    for (int64_t j0 = 0; j0 < L; j0 += JT) {
        __syncthreads();
        for (int e = threadIdx.x; e < RC * JT; e += 256) {
            const int c = e / JT, jj = e % JT;
            const int64_t j = j0 + jj;
            bs[c][jj] = (c < mc && j < L) ? betaT[c * L + j] : df::F2{0.f, 0.f};
        }
        __syncthreads();
        if (i0 >= N) continue;   // warp-uniform; the barriers above stay collective
#pragma unroll 1
        for (int st = 0; st < JT / 32; st++) {
            if (j0 + st * 32 >= L) break;   // warp-uniform
            const int64_t j = j0 + st * 32 + lane;
            df::F2 h[SPW];
#pragma unroll
            for (int q = 0; q < SPW; q++)
                h[q] = (i0 + q < N && j < L) ? H[(i0 + q) * L + j] : df::F2{0.f, 0.f};
#pragma unroll
            for (int c = 0; c < RC; c++) {
                const df::F2 bv = bs[c][st * 32 + lane];
#pragma unroll
                for (int q = 0; q < SPW; q++) df::df_acc_prod(ah[q][c], al[q][c], h[q], bv);
            }
        }
    }
    if (i0 >= N) return;
#pragma unroll
    for (int q = 0; q < SPW; q++) {
        const int64_t i = i0 + q;
#pragma unroll
        for (int c = 0; c < RC; c++) {
            if (c >= mc) break;
            df::F2 v = df::df_renorm(ah[q][c], al[q][c]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const df::F2 w{__shfl_xor_sync(0xffffffffu, v.h, o),
                               __shfl_xor_sync(0xffffffffu, v.l, o)};
                v = df::df_add(v, w);
            }
            if (lane == 0 && i < N)
                Rd[i * m + c0 + c] = df::df_add(df::d2df(T[i * ldt + c0 + c]), df::df_neg(v));
        }
    }
}

// part[p, j, :] = sum over the samples of split p of H[i, j] Rd[i, :]: one
// thread per neuron (coalesced rows of H), the split's Rd rows staged in
// shared memory (broadcast reads)
constexpr int HT_ROWS = 64;
template <int RC>
__global__ void __launch_bounds__(256)
htr_df_kernel(const df::F2 *__restrict__ H, int64_t L, int64_t N, const df::F2 *__restrict__ Rd,
              int64_t m, int64_t c0, int mc, double *__restrict__ part, int64_t chunk) {
    __shared__ df::F2 Rs[HT_ROWS][RC];
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t ib = (int64_t)blockIdx.y * chunk, ie = min(N, ib + chunk);
    float ah[RC], al[RC];
#pragma unroll
    for (int c = 0; c < RC; c++) ah[c] = al[c] = 0.f;
    for (int64_t i0 = ib; i0 < ie; i0 += HT_ROWS) {
        __syncthreads();
        for (int e = threadIdx.x; e < HT_ROWS * RC; e += 256) {
            const int ii = e / RC, cc = e % RC;
            const int64_t i = i0 + ii;
            Rs[ii][cc] = (i < ie && cc < mc) ? Rd[i * m + c0 + cc] : df::F2{0.f, 0.f};
        }
        __syncthreads();
        if (j < L) {
            const int in = (int)min((int64_t)HT_ROWS, ie - i0);
#pragma unroll 2
            for (int ii = 0; ii < in; ii++) {
                const df::F2 h = H[(i0 + ii) * L + j];
#pragma unroll
                for (int c = 0; c < RC; c++) df::df_acc_prod(ah[c], al[c], h, Rs[ii][c]);
            }
        }
    }
    if (j < L)
#pragma unroll
        for (int c = 0; c < RC; c++)
            if (c < mc)
                part[((int64_t)blockIdx.y * L + j) * m + c0 + c] = df::f2d(ah[c]) + df::f2d(al[c]);
}

__global__ void split_sum_kernel(const double *__restrict__ part, int nsplit,
                                 int64_t count, double *__restrict__ out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    double v = 0.0;
    for (int p = 0; p < nsplit; p++) v += part[(int64_t)p * count + e];
    out[e] = v;
}

// ---------------------------------------------------------------- predict
// Y[i, c] = sum_j g(x_i . w_j + b_j) a_j beta[j, c] for 16 target columns;
// 64 samples per block, neurons in ascending tiles of 64; the H tile never
// leaves shared memory (it overlays the X/W staging slabs).
constexpr int PC = 16;
template <typename XT>
__global__ void __launch_bounds__(NT)
predict_f64_kernel(const XT *__restrict__ X, int64_t N, int64_t n, int64_t ldx,
                   const double *__restrict__ W, int64_t ldw,
                   const double *__restrict__ b, const double *__restrict__ a,
                   int64_t L, int act, const double *__restrict__ beta,
                   int64_t ldb, int64_t m, double *__restrict__ Y, int64_t ldy) {
    __shared__ union {
        struct {
            double Ws[TK][TB];
            double Xs[TK][TB + 1];
        } st;
        double Hs[TB][TB + 1];
    } sm;
    __shared__ double Bs[TB][PC + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * TB;
    const int yi = threadIdx.x & 63, yg = threadIdx.x >> 6;  // sample, column group
    double yacc[PC / 4] = {};
    for (int64_t j0 = 0; j0 < L; j0 += TB) {
        double acc[4][4] = {};
        for (int64_t k0 = 0; k0 < n; k0 += TK) {
            for (int e = threadIdx.x; e < TK * TB; e += NT) {
                int kk = e / TB, jj = e % TB;
                int64_t k = k0 + kk, j = j0 + jj;
                sm.st.Ws[kk][jj] = (k < n && j < L) ? W[k * ldw + j] : 0.0;
                int ii = e / TK, kx = e % TK;
                int64_t i = i0 + ii, k2 = k0 + kx;
                sm.st.Xs[kx][ii] = (i < N && k2 < n) ? ld_x(X + i * ldx + k2) : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < TK; kk++) {
                double w[4], x[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    w[q] = sm.st.Ws[kk][ty + 16 * q];
                    x[q] = sm.st.Xs[kk][tx + 16 * q];
                }
#pragma unroll
                for (int p = 0; p < 4; p++)
#pragma unroll
                    for (int q = 0; q < 4; q++) acc[p][q] = fma(w[p], x[q], acc[p][q]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int p = 0; p < 4; p++) {
            int64_t j = j0 + ty + 16 * p;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double hv = 0.0;
                if (j < L) hv = (a ? a[j] : 1.0) * act_f64(acc[p][q] + b[j], act);
                sm.Hs[tx + 16 * q][ty + 16 * p] = hv;
            }
        }
        for (int e = threadIdx.x; e < TB * PC; e += NT) {
            int jj = e / PC, c = e % PC;
            int64_t j = j0 + jj;
            Bs[jj][c] = (j < L && c < m) ? beta[j * ldb + c] : 0.0;
        }
        __syncthreads();
        for (int jj = 0; jj < TB; jj++) {
            double h = sm.Hs[yi][jj];
#pragma unroll
            for (int q = 0; q < PC / 4; q++) yacc[q] = fma(h, Bs[jj][yg + 4 * q], yacc[q]);
        }
        __syncthreads();
    }
    int64_t i = i0 + yi;
    if (i < N)
#pragma unroll
        for (int q = 0; q < PC / 4; q++) {
            int c = yg + 4 * q;
            if (c < m) Y[i * ldy + c] = yacc[q];
        }
}

__global__ void sumsq_kernel(const double *__restrict__ x, int64_t rows,
                             int64_t cols, int64_t ld, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    int64_t total = rows * cols;
    for (int64_t e = threadIdx.x; e < total; e += 256) {
        double v = x[(e / cols) * ld + e % cols];
        s = fma(v, v, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// a warp per row (grid-strided), lanes over the columns
template <typename XT>
__global__ void check_finite_kernel(const XT *__restrict__ x, int64_t rows,
                                    int64_t cols, int64_t ld, int32_t *flag) {
    const int lane = threadIdx.x & 31;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows;
         i += (int64_t)gridDim.x * (blockDim.x >> 5))
        for (int64_t k = lane; k < cols; k += 32) bad |= !isfinite((double)x[i * ld + k]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void gather_rows_kernel(const double *__restrict__ src, int64_t lds,
                                   const int32_t *__restrict__ perm,
                                   const int64_t *__restrict__ r_dev, int64_t rmax,
                                   int64_t m, double *__restrict__ dst, int64_t ldd) {
    int64_t r = r_dev ? *r_dev : rmax;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < r * m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / m, c = e % m;
        dst[i * ldd + c] = src[(int64_t)perm[i] * lds + c];
    }
}

__global__ void scatter_rows_kernel(const double *__restrict__ src, int64_t m,
                                    const int32_t *__restrict__ perm, int64_t L,
                                    double *__restrict__ beta, int64_t ldb,
                                    double alpha, int accumulate) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < L * m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / m, c = e % m;
        double *d = beta + (int64_t)perm[i] * ldb + c;
        double v = alpha * src[i * m + c];
        *d = accumulate ? *d + v : v;
    }
}

// beta += dB; out[0] = ||dB||_F^2, out[1] = ||beta||_F^2 (one block, fixed
// reduction tree).
__global__ void axpy_norms_kernel(double *__restrict__ beta, const double *__restrict__ dB,
                                  int64_t count, double *__restrict__ out) {
    __shared__ double r0[256], r1[256];
    double a = 0.0, c = 0.0;
    for (int64_t e = threadIdx.x; e < count; e += 256) {
        double d = dB[e];
        double v = beta[e] + d;
        beta[e] = v;
        a = fma(d, d, a);
        c = fma(v, v, c);
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            r0[threadIdx.x] += r0[threadIdx.x + w];
            r1[threadIdx.x] += r1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = r0[0];
        out[1] = r1[0];
    }
}

__global__ void set_identity_kernel(double *__restrict__ A, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < n * n; e += (int64_t)gridDim.x * blockDim.x) A[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void add_identity_kernel(double *__restrict__ A, int64_t n, int64_t lda) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[i * lda + i] += 1.0;
}

__global__ void sub_rows_kernel(const double *__restrict__ A, int64_t lda,
                                const double *__restrict__ B, int64_t rows, int64_t m,
                                double *__restrict__ out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e < rows * m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / m, c = e % m;
        out[e] = A[i * lda + c] - B[e];
    }
}

// B (cols x rows, ldb) = A^T for A (rows x cols, lda): 32 x 32 tiles through
// shared memory, both sides coalesced.
// Ht[j, i] = a_j g(Ht[j, i] + b_j): row j = blockIdx.y (the same
// expression as the FP64 hidden layer's epilogue)
__global__ void act_rows_f64_kernel(double *__restrict__ Ht, int64_t ldh, int64_t N,
                                    const double *__restrict__ b, const double *__restrict__ a,
                                    int act) {
    const int64_t j = blockIdx.y, i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double aj = a ? a[j] : 1.0;
    Ht[j * ldh + i] = aj * act_f64(Ht[j * ldh + i] + b[j], act);
}

__global__ void transpose_f64_kernel(const double *__restrict__ A, int64_t rows, int64_t cols,
                                     int64_t lda, double *__restrict__ B, int64_t ldb) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t r = r0 + yy, c = c0 + tx;
        if (r < rows && c < cols) t[yy][tx] = A[r * lda + c];
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t c = c0 + yy, r = r0 + tx;
        if (r < rows && c < cols) B[c * ldb + r] = t[tx][yy];
    }
}

inline unsigned blocks_for(int64_t work, int per = 256, int64_t cap = 65535 * 8) {
    int64_t g = (work + per - 1) / per;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace

void hidden_f64(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n,
                int64_t ldx, const double *W, int64_t ldw, const double *b,
                const double *a, int64_t L, int act, double *Ht, int64_t ldh) {
    dim3 grid((unsigned)((N + TB - 1) / TB), (unsigned)((L + TB - 1) / TB));
    if (xdt == ELM_F64)
        hidden_f64_kernel<double><<<grid, NT, 0, s>>>((const double *)X, N, n, ldx, W, ldw,
                                                      b, a, L, act, Ht, ldh);
    else
        hidden_f64_kernel<float><<<grid, NT, 0, s>>>((const float *)X, N, n, ldx, W, ldw,
                                                     b, a, L, act, Ht, ldh);
    ELM_CHECK_LAUNCH();
}

int gram_f64_nsplit(int64_t L, int64_t m, int64_t N, int sms) {
    int64_t T = (L + m + TB - 1) / TB;
    int64_t tiles = T * (T + 1) / 2;
    int64_t want = (2 * (int64_t)sms + tiles - 1) / tiles;
    int64_t cap = (N + 1023) / 1024;
    int64_t ns = want < cap ? want : cap;
    return (int)(ns < 1 ? 1 : (ns > 64 ? 64 : ns));
}

size_t gram_f64_ws(int64_t L, int64_t m, int nsplit) {
    return (size_t)nsplit * (size_t)(L + m) * (size_t)(L + m);
}

void gram_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
              int64_t N, const double *T, int64_t ldt, int64_t m, double *S,
              int64_t lds, double *Z, int64_t ldz, double *part, int nsplit) {
    int64_t Tn = (L + m + TB - 1) / TB;
    int64_t chunk = ((N + nsplit - 1) / nsplit + TK - 1) / TK * TK;
    dim3 grid((unsigned)(Tn * (Tn + 1) / 2), (unsigned)nsplit);
    gram_f64_kernel<<<grid, NT, 0, s>>>(Ht, ldh, L, N, T, ldt, m, part, chunk);
    ELM_CHECK_LAUNCH();
    int64_t Lt = L + m;
    gram_reduce_kernel<<<blocks_for(Lt * Lt), 256, 0, s>>>(part, nsplit, L, m, S, lds,
                                                            Z, ldz);
    ELM_CHECK_LAUNCH();
}

// Products of a tall r x q matrix A (row-major, lda) with a few columns
// (m <= 32 per pass, RC a compile-time count >= the pass width): memory-bound
// on A, so A is read once, coalesced.
// part[s, i, c] = sum over the rows k of split s of A[k, i] Y[k, c0 + c]:
// thread per column i, 64 rows of Y staged in shared memory at a time.
template <int RC>
__global__ void __launch_bounds__(256)
atv_kernel(const double *__restrict__ A, int64_t k, int64_t q, int64_t lda,
           const double *__restrict__ Y, int64_t ldy, int64_t m, int64_t c0, int mc,
           int64_t kchunk, double *__restrict__ part) {
    __shared__ double ys[64][RC];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t kb = (int64_t)blockIdx.y * kchunk, ke = kb + kchunk < k ? kb + kchunk : k;
    double acc[RC];
#pragma unroll
    for (int c = 0; c < RC; c++) acc[c] = 0.0;
    for (int64_t k0 = kb; k0 < ke; k0 += 64) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * RC; e += 256) {
            const int kk = e / RC, c = e % RC;
            ys[kk][c] = (k0 + kk < ke && c < mc) ? Y[(k0 + kk) * ldy + c0 + c] : 0.0;
        }
        __syncthreads();
        if (i < q) {
            const int n = (int)(ke - k0 < 64 ? ke - k0 : 64);
            for (int kk = 0; kk < n; kk++) {
                const double a = A[(k0 + kk) * lda + i];
#pragma unroll
                for (int c = 0; c < RC; c++) acc[c] = fma(a, ys[kk][c], acc[c]);
            }
        }
    }
    if (i < q)
#pragma unroll
        for (int c = 0; c < RC; c++)
            if (c < mc) part[((int64_t)blockIdx.y * q + i) * m + c0 + c] = acc[c];
}

// Y[k, c0 + c] -= sum_i A[k, i] V[i, c0 + c]: warp per row k, lanes over i,
// a fixed shuffle tree.
template <int RC>
__global__ void __launch_bounds__(256)
av_sub_kernel(const double *__restrict__ A, int64_t k, int64_t q, int64_t lda,
              const double *__restrict__ V, int64_t ldv, int64_t c0, int mc,
              double *__restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= k) return;   // warp-uniform
    double acc[RC];
#pragma unroll
    for (int c = 0; c < RC; c++) acc[c] = 0.0;
    for (int64_t i = lane; i < q; i += 32) {
        const double a = A[row * lda + i];
#pragma unroll
        for (int c = 0; c < RC; c++)
            if (c < mc) acc[c] = fma(a, V[i * ldv + c0 + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < RC; c++) {
        double v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && c < mc) Y[row * ldy + c0 + c] -= v;
    }
}

// I + A^T A for A (k x q, row-major, stride lda): lower TB x TB tiles of
// the q x q result, the k range split into S contiguous pieces (one CTA per
// tile and piece), each piece's tile written to its own buffer; both operands
// are rows of A, so every load is coalesced.
__global__ void __launch_bounds__(NT)
syrk_f64_kernel(const double *__restrict__ A, int64_t k, int64_t q, int64_t lda,
                int64_t kchunk, double *__restrict__ part) {
    __shared__ double As[TK][TB + 1];
    __shared__ double Bs[TK][TB + 1];
    const int64_t t = blockIdx.x, sp = blockIdx.y;
    int64_t J = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (J * (J + 1) / 2 > t) J--;
    while ((J + 1) * (J + 2) / 2 <= t) J++;
    const int64_t I = t - J * (J + 1) / 2;
    const int64_t i0 = J * TB, j0 = I * TB;
    const int64_t kb = sp * kchunk, ke = kb + kchunk < k ? kb + kchunk : k;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TB; e += NT) {
            const int kk = e / TB, c = e % TB;
            const int64_t kr = k0 + kk;
            As[kk][c] = (kr < ke && i0 + c < q) ? A[kr * lda + i0 + c] : 0.0;
            Bs[kk][c] = (kr < ke && j0 + c < q) ? A[kr * lda + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double u[4], v[4];
#pragma unroll
            for (int w = 0; w < 4; w++) {
                u[w] = As[kk][ty + 16 * w];
                v[w] = Bs[kk][tx + 16 * w];
            }
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = fma(u[a], v[b], acc[a][b]);
        }
        __syncthreads();
    }
    double *out = part + (sp * (int64_t)gridDim.x + t) * (TB * TB);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) out[(ty + 16 * a) * TB + tx + 16 * b] = acc[a][b];
}

// C = I + sum of the S pieces, added in piece order, both triangles.
__global__ void syrk_sum_kernel(const double *__restrict__ part, int S, int64_t ntiles, int64_t q,
                                double *__restrict__ C, int64_t ldc) {
    const int64_t t = blockIdx.x;
    int64_t J = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (J * (J + 1) / 2 > t) J--;
    while ((J + 1) * (J + 2) / 2 <= t) J++;
    const int64_t I = t - J * (J + 1) / 2;
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int64_t i = J * TB + e / TB, j = I * TB + e % TB;
        if (i >= q || j >= q || j > i) continue;
        double v = i == j ? 1.0 : 0.0;
        for (int sp = 0; sp < S; sp++) v += part[(sp * ntiles + t) * (TB * TB) + e];
        C[i * ldc + j] = v;
        C[j * ldc + i] = v;
    }
}

void gemm_f64(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t sAm, int64_t sAk, const double *B,
              int64_t sBk, int64_t sBn, double beta, double *C, int64_t ldc) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((unsigned)((N + TB - 1) / TB), (unsigned)((M + TB - 1) / TB));
    gemm_f64_kernel<<<grid, NT, 0, s>>>(M, N, K, alpha, A, sAm, sAk, B, sBk, sBn, beta, C,
                                        ldc);
    ELM_CHECK_LAUNCH();
}

int syrk_f64_splits(int64_t k, int64_t q, int sms) {
    const int64_t T = (q + TB - 1) / TB, tiles = T * (T + 1) / 2;
    int64_t S = (4 * (int64_t)sms + tiles - 1) / tiles;   // about four CTAs per SM
    const int64_t cap = (k + 255) / 256;                    // at least 256 rows a piece
    if (S > cap) S = cap;
    return (int)(S < 1 ? 1 : S);
}

size_t syrk_f64_ws(int64_t q, int S) {
    const int64_t T = (q + TB - 1) / TB;
    return (size_t)S * (T * (T + 1) / 2) * TB * TB;
}

void syrk_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda, double *C,
              int64_t ldc, double *part, int S) {
    if (q <= 0) return;
    const int64_t T = (q + TB - 1) / TB, tiles = T * (T + 1) / 2;
    const int64_t kchunk = ((k + S - 1) / S + TK - 1) / TK * TK;
    syrk_f64_kernel<<<dim3((unsigned)tiles, (unsigned)S), NT, 0, s>>>(A, k, q, lda, kchunk, part);
    ELM_CHECK_LAUNCH();
    syrk_sum_kernel<<<(unsigned)tiles, 256, 0, s>>>(part, S, tiles, q, C, ldc);
    ELM_CHECK_LAUNCH();
}

void resid_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
               int64_t N, const double *beta, int64_t m, const double *T,
               int64_t ldt, double *R) {
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((m + RC - 1) / RC));
    resid_f64_kernel<<<grid, 128, 0, s>>>(Ht, ldh, L, N, beta, m, T, ldt, R);
    ELM_CHECK_LAUNCH();
}

int htr_f64_nsplit(int64_t L, int64_t N, int sms) {
    int64_t blocks = (L + 7) / 8;
    int64_t want = (4 * (int64_t)sms + blocks - 1) / blocks;
    int64_t cap = (N + 4095) / 4096;
    int64_t ns = want < cap ? want : cap;
    return (int)(ns < 1 ? 1 : (ns > 128 ? 128 : ns));
}

size_t htr_f64_ws(int64_t L, int64_t m, int nsplit) { return (size_t)nsplit * L * m; }

void htr_f64(cudaStream_t s, const double *Ht, int64_t ldh, int64_t L,
             int64_t N, const double *R, int64_t m, double *G, double *part,
             int nsplit) {
    int64_t chunk = ((N + nsplit - 1) / nsplit + 255) / 256 * 256;
    dim3 grid((unsigned)((L + 7) / 8), (unsigned)nsplit, (unsigned)((m + RC - 1) / RC));
    htr_f64_kernel<<<grid, 256, 0, s>>>(Ht, ldh, L, N, R, m, part, chunk);
    ELM_CHECK_LAUNCH();
    split_sum_kernel<<<blocks_for(L * m), 256, 0, s>>>(part, nsplit, L * m, G);
    ELM_CHECK_LAUNCH();
}

// targets per pass: the smallest compile-time count covering m (32 above)
template <class F>
static void with_rc(int64_t m, F &&f) {
    if (m <= 2) f(std::integral_constant<int, 2>());
    else if (m <= 4) f(std::integral_constant<int, 4>());
    else if (m <= 6) f(std::integral_constant<int, 6>());
    else if (m <= 8) f(std::integral_constant<int, 8>());
    else if (m <= 10) f(std::integral_constant<int, 10>());
    else if (m <= 12) f(std::integral_constant<int, 12>());
    else if (m <= 16) f(std::integral_constant<int, 16>());
    else if (m <= 20) f(std::integral_constant<int, 20>());
    else if (m <= 26) f(std::integral_constant<int, 26>());
    else f(std::integral_constant<int, 32>());
}

int atv_splits(int64_t k, int64_t q, int sms) {
    const int64_t cols = (q + 255) / 256;
    int64_t S = (4 * (int64_t)sms + cols - 1) / cols;
    const int64_t cap = (k + 63) / 64;   // at least 64 rows a split
    if (S > cap) S = cap;
    return (int)(S < 1 ? 1 : S);
}

void atv_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda, const double *Y,
             int64_t m, double *out, double *part, int S) {
    if (q <= 0 || m <= 0) return;
    const int64_t kchunk = (k + S - 1) / S;
    for (int64_t c0 = 0; c0 < m; c0 += 32) {
        const int64_t mc = m - c0 < 32 ? m - c0 : 32;
        with_rc(mc, [&](auto rc) {
            constexpr int RC = decltype(rc)::value;
            atv_kernel<RC><<<dim3((unsigned)((q + 255) / 256), (unsigned)S), 256, 0, s>>>(
                A, k, q, lda, Y, m, m, c0, (int)mc, kchunk, part);
        });
        ELM_CHECK_LAUNCH();
    }
    split_sum_kernel<<<blocks_for(q * m), 256, 0, s>>>(part, S, q * m, out);
    ELM_CHECK_LAUNCH();
}

void av_sub_f64(cudaStream_t s, const double *A, int64_t k, int64_t q, int64_t lda,
                const double *V, int64_t m, double *Y) {
    if (k <= 0 || m <= 0) return;
    for (int64_t c0 = 0; c0 < m; c0 += 32) {
        const int64_t mc = m - c0 < 32 ? m - c0 : 32;
        with_rc(mc, [&](auto rc) {
            constexpr int RC = decltype(rc)::value;
            av_sub_kernel<RC><<<(unsigned)((k + 7) / 8), 256, 0, s>>>(A, k, q, lda, V, m, c0,
                                                                      (int)mc, Y, m);
        });
        ELM_CHECK_LAUNCH();
    }
}

void resid_df(cudaStream_t s, const void *H, int64_t L, int64_t N, const double *beta,
              int64_t m, const double *T, int64_t ldt, void *Rd, void *betaT) {
    for (int64_t c0 = 0; c0 < m; c0 += 32) {   // targets in passes of up to 32
        const int64_t mc = m - c0 < 32 ? m - c0 : 32;
        beta_pairs_kernel<<<blocks_for(L * mc), 256, 0, s>>>(beta, L, m, c0, mc, (df::F2 *)betaT);
        ELM_CHECK_LAUNCH();
        with_rc(mc, [&](auto rc) {
            constexpr int RC = decltype(rc)::value;
            constexpr int SPW = spw_for<RC>();
            resid_df_kernel<RC><<<(unsigned)((N + 8 * SPW - 1) / (8 * SPW)), 256, 0, s>>>(
                (const df::F2 *)H, L, N, (const df::F2 *)betaT, m, c0, (int)mc, T, ldt,
                (df::F2 *)Rd);
        });
        ELM_CHECK_LAUNCH();
    }
}

int htr_df_nsplit(int64_t L, int64_t N, int sms) {
    const int64_t blocks = (L + 255) / 256;
    int64_t ns = (8 * (int64_t)sms + blocks - 1) / blocks;
    const int64_t cap = (N + HT_ROWS - 1) / HT_ROWS;
    if (ns > cap) ns = cap;
    return (int)(ns < 1 ? 1 : ns);
}

void htr_df(cudaStream_t s, const void *H, int64_t L, int64_t N, const void *Rd, int64_t m,
            double *G, double *part, int nsplit) {
    const int64_t chunk = ((N + nsplit - 1) / nsplit + HT_ROWS - 1) / HT_ROWS * HT_ROWS;
    for (int64_t c0 = 0; c0 < m; c0 += 32) {
        const int64_t mc = m - c0 < 32 ? m - c0 : 32;
        with_rc(mc, [&](auto rc) {
            constexpr int RC = decltype(rc)::value;
            dim3 grid((unsigned)((L + 255) / 256), (unsigned)nsplit);
            htr_df_kernel<RC><<<grid, 256, 0, s>>>((const df::F2 *)H, L, N, (const df::F2 *)Rd,
                                                   m, c0, (int)mc, part, chunk);
        });
        ELM_CHECK_LAUNCH();
    }
    split_sum_kernel<<<blocks_for(L * m), 256, 0, s>>>(part, nsplit, L * m, G);
    ELM_CHECK_LAUNCH();
}

void predict_f64(cudaStream_t s, const void *X, int xdt, int64_t N, int64_t n,
                 int64_t ldx, const double *W, int64_t ldw, const double *b,
                 const double *a, int64_t L, int act, const double *beta,
                 int64_t ldb, int64_t m, double *Y, int64_t ldy) {
    // one pass handles PC target columns
    for (int64_t c0 = 0; c0 < m; c0 += PC) {
        int64_t mc = m - c0 < PC ? m - c0 : PC;
        dim3 grid((unsigned)((N + TB - 1) / TB));
        if (xdt == ELM_F64)
            predict_f64_kernel<double><<<grid, NT, 0, s>>>(
                (const double *)X, N, n, ldx, W, ldw, b, a, L, act, beta + c0, ldb, mc,
                Y + c0, ldy);
        else
            predict_f64_kernel<float><<<grid, NT, 0, s>>>(
                (const float *)X, N, n, ldx, W, ldw, b, a, L, act, beta + c0, ldb, mc,
                Y + c0, ldy);
        ELM_CHECK_LAUNCH();
    }
}

void sumsq(cudaStream_t s, const double *x, int64_t rows, int64_t cols, int64_t ld,
           double *out) {
    sumsq_kernel<<<1, 256, 0, s>>>(x, rows, cols, ld, out);
    ELM_CHECK_LAUNCH();
}

void check_finite(cudaStream_t s, const void *x, int xdt, int64_t rows, int64_t cols,
                  int64_t ld, int32_t *flag) {
    unsigned g = blocks_for(rows * 32, 256, 4096);
    if (xdt == ELM_F64)
        check_finite_kernel<double><<<g, 256, 0, s>>>((const double *)x, rows, cols, ld, flag);
    else
        check_finite_kernel<float><<<g, 256, 0, s>>>((const float *)x, rows, cols, ld, flag);
    ELM_CHECK_LAUNCH();
}

void gather_rows(cudaStream_t s, const double *src, int64_t lds, const int32_t *perm,
                 const int64_t *r_dev, int64_t rmax, int64_t m, double *dst, int64_t ldd) {
    gather_rows_kernel<<<blocks_for(rmax * m), 256, 0, s>>>(src, lds, perm, r_dev, rmax, m,
                                                            dst, ldd);
    ELM_CHECK_LAUNCH();
}

void scatter_rows(cudaStream_t s, const double *src, int64_t m, const int32_t *perm,
                  int64_t L, double *beta, int64_t ldb, double alpha, int accumulate) {
    scatter_rows_kernel<<<blocks_for(L * m), 256, 0, s>>>(src, m, perm, L, beta, ldb, alpha,
                                                          accumulate);
    ELM_CHECK_LAUNCH();
}

void axpy_norms(cudaStream_t s, double *beta, const double *dB, int64_t count, double *out) {
    axpy_norms_kernel<<<1, 256, 0, s>>>(beta, dB, count, out);
    ELM_CHECK_LAUNCH();
}

void sub_rows(cudaStream_t s, const double *A, int64_t lda, const double *B, int64_t rows,
              int64_t m, double *out) {
    sub_rows_kernel<<<blocks_for(rows * m), 256, 0, s>>>(A, lda, B, rows, m, out);
    ELM_CHECK_LAUNCH();
}

void act_rows_f64(cudaStream_t s, double *Ht, int64_t ldh, int64_t L, int64_t N, const double *b,
                  const double *a, int act) {
    if (L <= 0 || N <= 0) return;
    const dim3 g((unsigned)((N + 255) / 256), (unsigned)L);
    act_rows_f64_kernel<<<g, 256, 0, s>>>(Ht, ldh, N, b, a, act);
    ELM_CHECK_LAUNCH();
}

void transpose_f64(cudaStream_t s, const double *A, int64_t rows, int64_t cols, int64_t lda,
                   double *B, int64_t ldb) {
    if (rows <= 0 || cols <= 0) return;
    // rows in slices of at most 65535 row blocks (the grid's y limit)
    constexpr int64_t RMAX = 65535 * 32;
    for (int64_t r0 = 0; r0 < rows; r0 += RMAX) {
        const int64_t rr = rows - r0 < RMAX ? rows - r0 : RMAX;
        dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rr + 31) / 32));
        transpose_f64_kernel<<<g, 256, 0, s>>>(A + r0 * lda, rr, cols, lda, B + r0, ldb);
        ELM_CHECK_LAUNCH();
    }
}

void set_identity(cudaStream_t s, double *A, int64_t n) {
    set_identity_kernel<<<blocks_for(n * n), 256, 0, s>>>(A, n);
    ELM_CHECK_LAUNCH();
}

void add_identity(cudaStream_t s, double *A, int64_t n, int64_t lda) {
    if (n <= 0) return;
    add_identity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n, lda);
    ELM_CHECK_LAUNCH();
}

}  // namespace elm
