// mra_kernels.cuh -- sm_103a kernels of the MRA log-likelihood.
//
// The GPU evaluates the same likelihood as the paper's MRA (Sec. 1.1) in a
// whitened basis: with L_A the Cholesky factor of W^l_A = C_l(Q_A, Q_A) and
// Linv_A = L_A^{-1}, the basis of any point set P against its level-l ancestor
// A_l is What^l_P = C_l(P, Q_{A_l}) Linv_{A_l}', which turns the recursion of
// the remainder covariances into
//     W^l_P   = C(P, Q_{A_l}) - sum_{k<l} What^k_P (What^k_{A_l})'
//     What^l_P = W^l_P Linv_{A_l}'
// and the prior precision of every level into the identity.  The upward pass
// then factors I + A^{m,m} instead of K^{-1} + A^{m,m}; log-determinants and
// quadratic forms are unchanged (|K^{-1} + A| / |K^{-1}| = |I + L^{-1} A L^{-T}|).
//
// One CTA of 256 threads works on one region (prior, upward pass), one chunk
// of 32 observation rows (leaf basis), one leaf (leaf posterior) or one
// (region, block pair) (leaf Gram).  r_hat knots are padded to RP (16 or 32)
// with inert padding: zero covariance rows and columns and an identity
// diagonal on the padded part of every factor, which leaves every result
// exact.  Cholesky factors, log-determinants and quadratic forms are FP64 in
// both precisions; T is the storage and product type (double, or float for
// the mixed mode).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mra_internal.h"

namespace mra {

constexpr int NT = MRA_NT;
enum { MM_SET = 0, MM_SUB = 1 };
enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOTPD = 3 };

__device__ __forceinline__ bool theta_ok(const double *th)
{
    return isfinite(th[0]) && isfinite(th[1]) && isfinite(th[2]) && th[0] > 0.0 && th[1] > 0.0 &&
           th[2] > 0.0;
}

// Exponential covariance sigma2 * exp(-|a - b| / beta) (Sec. 2.2.4 reading).
template <typename T>
__device__ __forceinline__ T cov_exp(double s2, double beta, double ax, double ay, double bx,
                                     double by);
template <>
__device__ __forceinline__ double cov_exp<double>(double s2, double beta, double ax, double ay,
                                                  double bx, double by)
{
    double dx = ax - bx, dy = ay - by;
    return s2 * exp(-sqrt(dx * dx + dy * dy) / beta);
}
template <>
__device__ __forceinline__ float cov_exp<float>(double s2, double beta, double ax, double ay,
                                                double bx, double by)
{
    float dx = (float)(ax - bx), dy = (float)(ay - by);
    return (float)s2 * expf(-sqrtf(dx * dx + dy * dy) / (float)beta);
}

// sum_k a[k] b[k] (strides sa, sb) returned in FP64.  FP64 operands: plain
// FMA chain.  FP32 operands: every product is split exactly (TwoProd with an
// FMA) and accumulated as an unevaluated float pair (TwoSum), so the result is
// accurate to ~K eps_32^2 of the terms, which keeps C + tau2 I - U U' free of
// FP32 cancellation error in the mixed mode.
__device__ __forceinline__ double dot_acc(const double *a, int sa, const double *b, int sb, int K)
{
    double s = 0.0;
    for (int k = 0; k < K; k++) s = fma(a[k * sa], b[k * sb], s);
    return s;
}
__device__ __forceinline__ double dot_acc(const float *a, int sa, const float *b, int sb, int K)
{
    float hi = 0.f, lo = 0.f;
    for (int k = 0; k < K; k++) {
        const float x = a[k * sa], y = b[k * sb];
        const float p = __fmul_rn(x, y);
        const float e = __fmaf_rn(x, y, -p);
        const float t = __fadd_rn(hi, p);
        const float z = __fsub_rn(t, hi);
        const float r = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(r, e));
    }
    return (double)hi + (double)lo;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NT / 32 ? red[lane] : 0.0;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// Singularity rule shared by every factorisation: a pivot at or below
// kSingular times the largest diagonal entry of the matrix is singular
// (coincident knots make the covariance singular, Sec. 1.2).
#define MRA_SINGULAR 1e-12

// In-place lower Cholesky of the n x n matrix A (leading dimension lda) by the
// whole CTA; a singular pivot sets *fail and is replaced by 1 so that the
// factorisation completes without NaN.  Works on shared or global memory.
static __device__ void chol_cta(double *A, int lda, int n, int *fail)
{
    __shared__ double s_scale;
    if (threadIdx.x == 0) {
        double sc = 0.0;
        for (int j = 0; j < n; j++) sc = fmax(sc, A[j * lda + j]);
        s_scale = sc;
    }
    __syncthreads();
    const double tol = MRA_SINGULAR * s_scale;
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            double d = A[j * lda + j];
            if (!(d > tol)) {
                *fail = 1;
                d = 1.0;
            }
            A[j * lda + j] = sqrt(d);
        }
        __syncthreads();
        const double ljj = A[j * lda + j];
        for (int i = j + 1 + threadIdx.x; i < n; i += NT) A[i * lda + j] /= ljj;
        __syncthreads();
        const int w = n - j - 1;
        for (int e = threadIdx.x; e < w * w; e += NT) {
            const int i = j + 1 + e / w, k = j + 1 + e % w;
            if (k <= i) A[i * lda + k] -= A[i * lda + j] * A[k * lda + j];
        }
        __syncthreads();
    }
}

// X = L^{-1} for lower-triangular L (n x n), one column per thread.
static __device__ void trinv_cta(const double *L, int ldl, double *X, int ldx, int n)
{
    for (int j = threadIdx.x; j < n; j += NT) {
        for (int i = 0; i < j; i++) X[i * ldx + j] = 0.0;
        X[j * ldx + j] = 1.0 / L[j * ldl + j];
        for (int i = j + 1; i < n; i++) {
            double s = 0.0;
            for (int t = j; t < i; t++) s += L[i * ldl + t] * X[t * ldx + j];
            X[i * ldx + j] = -s / L[i * ldl + i];
        }
    }
    __syncthreads();
}

// C (ROWS x RP) = or -= A (ROWS x K) * B (RP x K)'.  Caller synchronises.
template <typename T, int ROWS, int RP>
__device__ __forceinline__ void mm_nt(T *C, int ldc, const T *A, int lda, const T *B, int ldb,
                                      int K, int mode)
{
    constexpr int CPT = ROWS * RP / NT;
    static_assert(CPT >= 1 && (ROWS * RP) % NT == 0, "tile");
    constexpr int TPR = RP / CPT;
    const int i = threadIdx.x / TPR, j0 = threadIdx.x % TPR;
    T acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; c++) acc[c] = T(0);
    for (int t = 0; t < K; t++) {
        const T a = A[i * lda + t];
#pragma unroll
        for (int c = 0; c < CPT; c++) acc[c] += a * B[(j0 + c * TPR) * ldb + t];
    }
#pragma unroll
    for (int c = 0; c < CPT; c++) {
        T *p = C + i * ldc + j0 + c * TPR;
        *p = mode == MM_SET ? acc[c] : *p - acc[c];
    }
}

template <typename T, int RP>
__device__ __forceinline__ void load_block(T *s, const T *g)
{
    constexpr int LD = RP + 1;
    for (int e = threadIdx.x; e < RP * RP; e += NT) s[(e / RP) * LD + e % RP] = g[e];
}

__host__ __device__ __forceinline__ int npairs(int D) { return D * (D + 1) / 2; }
__host__ __device__ __forceinline__ int pidx(int k, int l) { return l * (l - 1) / 2 + k - 1; }

// ------------------------------------------------------------------ prior --
// Region i of level m (1 <= m <= M-1): What^1..What^{m-1} against its
// ancestors, then W^m = C(Q,Q) - sum_k What^k What^k', its Cholesky factor L,
// log|W^m| and Linv = L^{-1}.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_prior_bytes(int m)
{
    return (size_t)2 * RP * (RP + 1) * sizeof(double) + 4 * RP * sizeof(double) + 32 * sizeof(double) +
           16 + (size_t)(m + 1) * RP * (RP + 1) * sizeof(T);
}

template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_prior(DevTree t, Work<T> w, int m)
{
    constexpr int LD = RP + 1;
    const int i = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const double s2 = th[0], beta = th[1];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sL = (double *)smem_raw;
    double *sX = sL + RP * LD;
    double *sq = sX + RP * LD;
    double *sa = sq + 2 * RP;
    double *red = sa + 2 * RP;
    int *flag = (int *)(red + 32);
    T *sW = (T *)(flag + 4);
    T *sA = sW + RP * LD;
    T *sWh = sA + RP * LD;
    const int R = t.R;
    const int64_t g = t.lvl_off[m] + i;
    if (tid < RP) {
        sq[tid] = t.kx[g * RP + tid];
        sq[RP + tid] = t.ky[g * RP + tid];
    }
    if (tid == 0) flag[0] = 0;
    T *pb = w.prior + (size_t)b * w.prior_stride;
    __syncthreads();
    for (int l = 1; l < m; l++) {
        const int64_t ia = (int64_t)i >> (t.lgJ * (m - l));
        const int64_t ga = t.lvl_off[l] + ia;
        const T *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        if (tid < RP) {
            sa[tid] = t.kx[ga * RP + tid];
            sa[RP + tid] = t.ky[ga * RP + tid];
        }
        __syncthreads();
        for (int e = tid; e < RP * RP; e += NT) {
            const int a = e / RP, c = e % RP;
            sW[a * LD + c] = (a < R && c < R) ? cov_exp<T>(s2, beta, sq[a], sq[RP + a], sa[c], sa[RP + c])
                                              : T(0);
        }
        for (int k = 1; k < l; k++) {
            load_block<T, RP>(sA, anc + (size_t)(k - 1) * RP * RP);
            __syncthreads();
            mm_nt<T, RP, RP>(sW, LD, sWh + (k - 1) * RP * LD, LD, sA, LD, RP, MM_SUB);
            __syncthreads();
        }
        load_block<T, RP>(sA, anc + (size_t)(l - 1) * RP * RP);
        __syncthreads();
        mm_nt<T, RP, RP>(sWh + (l - 1) * RP * LD, LD, sW, LD, sA, LD, RP, MM_SET);
        __syncthreads();
    }
    for (int e = tid; e < RP * RP; e += NT) {
        const int a = e / RP, c = e % RP;
        sW[a * LD + c] = (a < R && c < R) ? cov_exp<T>(s2, beta, sq[a], sq[RP + a], sq[c], sq[RP + c])
                                          : (a == c ? T(1) : T(0));
    }
    __syncthreads();
    for (int k = 1; k < m; k++) {
        mm_nt<T, RP, RP>(sW, LD, sWh + (k - 1) * RP * LD, LD, sWh + (k - 1) * RP * LD, LD, RP, MM_SUB);
        __syncthreads();
    }
    for (int e = tid; e < RP * RP; e += NT) {
        const int a = e / RP, c = e % RP;
        sL[a * LD + c] = (double)sW[a * LD + c];
    }
    __syncthreads();
    chol_cta(sL, LD, RP, flag);
    double v = 0.0;
    for (int a = tid; a < R; a += NT) v += log(sL[a * LD + a]);
    v = block_sum(v, red);
    trinv_cta(sL, LD, sX, LD, RP);
    T *out = pb + w.prior_lvl[m] + (size_t)i * m * RP * RP;
    for (int k = 0; k < m - 1; k++)
        for (int e = tid; e < RP * RP; e += NT) out[(size_t)k * RP * RP + e] = sWh[k * RP * LD + (e / RP) * LD + e % RP];
    for (int e = tid; e < RP * RP; e += NT) out[(size_t)(m - 1) * RP * RP + e] = (T)sX[(e / RP) * LD + e % RP];
    if (tid == 0) {
        if (flag[0]) w.status[b] = ST_ENOTPD;
        if (w.reg_lw) w.reg_lw[(size_t)b * w.reglw_stride + g] = 2.0 * v;
    }
}

// -------------------------------------------------------------- leaf basis --
// A chunk of <= 32 observation rows of one level-(M-1) subtree: What^l of each
// row against the M-1 ancestors (U rows).
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_leafbasis_bytes(int M)
{
    return (size_t)2 * MRA_CH * sizeof(double) + 2 * RP * sizeof(double) +
           ((size_t)MRA_CH * (RP + 1) + (size_t)RP * (RP + 1) + (size_t)(M - 1) * MRA_CH * (RP + 1)) * sizeof(T);
}

template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_leafbasis(DevTree t, Work<T> w, const Chunk *chunks)
{
    constexpr int LD = RP + 1, CH = MRA_CH;
    const Chunk ch = chunks[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const double s2 = th[0], beta = th[1];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sp = (double *)smem_raw;
    double *sa = sp + 2 * CH;
    T *sW = (T *)(sa + 2 * RP);
    T *sA = sW + CH * LD;
    T *sU = sA + RP * LD;
    const int M = t.M, R = t.R, P = ch.parent, nr = ch.n;
    if (tid < CH) {
        sp[tid] = tid < nr ? t.sx[ch.row0 + tid] : 0.0;
        sp[CH + tid] = tid < nr ? t.sy[ch.row0 + tid] : 0.0;
    }
    const T *pb = w.prior + (size_t)b * w.prior_stride;
    for (int l = 1; l <= M - 1; l++) {
        const int64_t ia = (int64_t)P >> (t.lgJ * (M - 1 - l));
        const int64_t ga = t.lvl_off[l] + ia;
        const T *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        if (tid < RP) {
            sa[tid] = t.kx[ga * RP + tid];
            sa[RP + tid] = t.ky[ga * RP + tid];
        }
        __syncthreads();
        for (int e = tid; e < CH * RP; e += NT) {
            const int a = e / RP, c = e % RP;
            sW[a * LD + c] = (a < nr && c < R) ? cov_exp<T>(s2, beta, sp[a], sp[CH + a], sa[c], sa[RP + c])
                                               : T(0);
        }
        for (int k = 1; k < l; k++) {
            load_block<T, RP>(sA, anc + (size_t)(k - 1) * RP * RP);
            __syncthreads();
            mm_nt<T, CH, RP>(sW, LD, sU + (k - 1) * CH * LD, LD, sA, LD, RP, MM_SUB);
            __syncthreads();
        }
        load_block<T, RP>(sA, anc + (size_t)(l - 1) * RP * RP);
        __syncthreads();
        mm_nt<T, CH, RP>(sU + (l - 1) * CH * LD, LD, sW, LD, sA, LD, RP, MM_SET);
        __syncthreads();
    }
    const int UC = (M - 1) * RP;
    T *Ub = w.U + (size_t)b * w.U_stride;
    for (int e = tid; e < nr * UC; e += NT) {
        const int a = e / UC, col = e % UC, l = col / RP, c = col % RP;
        Ub[(size_t)(ch.row0 + a) * UC + col] = sU[l * CH * LD + a * LD + c];
    }
}

// ---------------------------------------------------------- leaf posterior --
// Leaf c with n <= nmax observations, all in shared memory:
// V = C(S,S) + tau2 I - U U', V = L L' (FP64), Y = L^{-1} U (in place),
// y = L^{-1} z, d = log|V|, u = y'y.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_leafpost_bytes(int M, int nmax)
{
    return (size_t)nmax * (nmax + 1) * sizeof(double) + 4 * (size_t)nmax * sizeof(double) +
           32 * sizeof(double) + 16 + (size_t)nmax * ((M - 1) * RP + 1) * sizeof(T) +
           (size_t)nmax * (nmax + 1) * sizeof(T);
}

// V = L L' (FP64, in place), then Y = L^{-1} U in the storage type T using LT,
// a T copy of L (ldlt), and y = L^{-1} z in FP64.
template <typename T>
static __device__ void leaf_factor_solve(double *V, int ldv, T *LT, int ldlt, T *U, int ldu, int UC, double *y,
                                         int n, int *flag)
{
    chol_cta(V, ldv, n, flag);
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += NT) {
        const int a = (int)(e / n), q = (int)(e % n);
        if (q <= a) LT[(size_t)a * ldlt + q] = (T)V[(size_t)a * ldv + q];
    }
    __syncthreads();
    for (int col = threadIdx.x; col <= UC; col += NT) {
        if (col < UC) {
            for (int a = 0; a < n; a++) {
                T s = U[(size_t)a * ldu + col];
                for (int q = 0; q < a; q++) s -= LT[(size_t)a * ldlt + q] * U[(size_t)q * ldu + col];
                U[(size_t)a * ldu + col] = s / LT[(size_t)a * ldlt + a];
            }
        } else {
            for (int a = 0; a < n; a++) {
                double s = y[a];
                for (int q = 0; q < a; q++) s -= V[(size_t)a * ldv + q] * y[q];
                y[a] = s / V[(size_t)a * ldv + a];
            }
        }
    }
    __syncthreads();
}

template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_leafpost_small(DevTree t, Work<T> w, const int64_t *leaves,
                                                       int nmax)
{
    const int64_t c = leaves[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const double s2 = th[0], beta = th[1], tau2 = th[2];
    const int M = t.M;
    const int64_t o0 = t.leaf_off[c];
    const int n = (int)(t.leaf_off[c + 1] - o0);
    const int UC = (M - 1) * RP, LDU = UC + 1, LDV = nmax + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sV = (double *)smem_raw;
    double *sp = sV + (size_t)nmax * LDV;
    double *sy = sp + 3 * nmax;
    double *red = sy + nmax;
    int *flag = (int *)(red + 32);
    T *sU = (T *)(flag + 4);
    T *sLT = sU + (size_t)nmax * LDU;
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)o0 * UC;
    for (int a = tid; a < n; a += NT) {
        sp[a] = t.sx[o0 + a];
        sp[nmax + a] = t.sy[o0 + a];
        sp[2 * nmax + a] = t.sz[o0 + a];
        sy[a] = t.sz[o0 + a];
    }
    if (tid == 0) flag[0] = 0;
    for (int e = tid; e < n * UC; e += NT) sU[(e / UC) * LDU + e % UC] = Ub[e];
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int a = e / n, q = e % n;
        if (q <= a) {
            const double g = dot_acc(sU + a * LDU, 1, sU + q * LDU, 1, UC);
            const double v = cov_exp<double>(s2, beta, sp[a], sp[nmax + a], sp[q], sp[nmax + q]) + (a == q ? tau2 : 0.0);
            sV[a * LDV + q] = v - g;
        }
    }
    __syncthreads();
    leaf_factor_solve<T>(sV, LDV, sLT, nmax + 1, sU, LDU, UC, sy, n, flag);
    double dv = 0.0, uv = 0.0;
    for (int a = tid; a < n; a += NT) {
        dv += log(sV[a * LDV + a]);
        uv += sy[a] * sy[a];
    }
    dv = 2.0 * block_sum(dv, red);
    uv = block_sum(uv, red);
    for (int e = tid; e < n * UC; e += NT) Ub[e] = sU[(e / UC) * LDU + e % UC];
    double *yb = w.ybuf + (size_t)b * w.y_stride + o0;
    for (int a = tid; a < n; a += NT) yb[a] = sy[a];
    if (tid == 0) {
        double *du = w.leaf_du + (size_t)b * w.leafdu_stride + 2 * c;
        du[0] = dv;
        du[1] = uv;
        if (w.reg_du) {
            double *r = w.reg_du + (size_t)b * w.regdu_stride + 2 * (t.lvl_off[M] + c);
            r[0] = dv;
            r[1] = uv;
        }
        if (flag[0]) w.status[b] = ST_ENOTPD;
    }
}

// Leaves larger than the shared-memory path: the same steps on global memory.
template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_leafpost_big(DevTree t, Work<T> w, const BigLeaf *leaves)
{
    const BigLeaf bl = leaves[blockIdx.x];
    const int64_t c = bl.leaf;
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const double s2 = th[0], beta = th[1], tau2 = th[2];
    const int M = t.M;
    const int64_t o0 = t.leaf_off[c];
    const int n = (int)(t.leaf_off[c + 1] - o0);
    const int UC = (M - 1) * RP;
    __shared__ double red[32];
    __shared__ int flag[4];
    double *V = w.Vbig + (size_t)b * w.V_stride + bl.voff;
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)o0 * UC;
    double *yb = w.ybuf + (size_t)b * w.y_stride + o0;
    const double *px = t.sx + o0, *py = t.sy + o0, *pz = t.sz + o0;
    if (tid == 0) flag[0] = 0;
    for (int a = tid; a < n; a += NT) yb[a] = pz[a];
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
        const int a = (int)(e / n), q = (int)(e % n);
        if (q <= a) {
            const double g = dot_acc(Ub + (size_t)a * UC, 1, Ub + (size_t)q * UC, 1, UC);
            const double v = cov_exp<double>(s2, beta, px[a], py[a], px[q], py[q]) + (a == q ? tau2 : 0.0);
            V[(size_t)a * n + q] = v - g;
        }
    }
    __syncthreads();
    // the T copy of the factor lives right after V in the scratch (2 n^2 doubles per big leaf)
    leaf_factor_solve<T>(V, n, (T *)(V + (size_t)n * n), n, Ub, UC, UC, yb, n, flag);
    double dv = 0.0, uv = 0.0;
    for (int a = tid; a < n; a += NT) {
        dv += log(V[(size_t)a * n + a]);
        uv += yb[a] * yb[a];
    }
    dv = 2.0 * block_sum(dv, red);
    uv = block_sum(uv, red);
    if (tid == 0) {
        double *du = w.leaf_du + (size_t)b * w.leafdu_stride + 2 * c;
        du[0] = dv;
        du[1] = uv;
        if (w.reg_du) {
            double *r = w.reg_du + (size_t)b * w.regdu_stride + 2 * (t.lvl_off[M] + c);
            r[0] = dv;
            r[1] = uv;
        }
        if (flag[0]) w.status[b] = ST_ENOTPD;
    }
}

// --------------------------------------------------------------- leaf Gram --
// Region P of level M-1: A^{k,l} = sum over the rows below P of Y^k' Y^l for
// one block pair per CTA (blockIdx.y < npairs), or (blockIdx.y == npairs) the
// vectors w^k = Y^k' y and the sums of the leaves' (d, u).
template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_leafgram(DevTree t, Work<T> w)
{
    constexpr int LD = RP + 1, CH = MRA_CH;
    constexpr int CPT = RP * RP / NT, TPR = RP / CPT;
    const int P = blockIdx.x, pr = blockIdx.y, b = blockIdx.z, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const int M = t.M, J = t.J, D = M - 1, UC = D * RP;
    const int np = npairs(D);
    const int64_t r0 = t.leaf_off[(int64_t)P * J], r1 = t.leaf_off[(int64_t)P * J + J];
    const T *Ub = w.U + (size_t)b * w.U_stride;
    if (pr < np) {
        __shared__ T sX[CH * LD], sY[CH * LD];
        int l = 1;
        while (l * (l + 1) / 2 <= pr) l++;
        const int k = pr - l * (l - 1) / 2 + 1;
        const int i = tid / TPR, j0 = tid % TPR;
        double acc64[CPT];
#pragma unroll
        for (int c = 0; c < CPT; c++) acc64[c] = 0.0;
        for (int64_t rb = r0; rb < r1; rb += CH) {
            T acc[CPT];
#pragma unroll
            for (int c = 0; c < CPT; c++) acc[c] = T(0);
            const int nr = (int)min((int64_t)CH, r1 - rb);
            for (int e = tid; e < CH * RP; e += NT) {
                const int a = e / RP, cc = e % RP;
                sX[a * LD + cc] = a < nr ? Ub[(size_t)(rb + a) * UC + (k - 1) * RP + cc] : T(0);
                sY[a * LD + cc] = a < nr ? Ub[(size_t)(rb + a) * UC + (l - 1) * RP + cc] : T(0);
            }
            __syncthreads();
            for (int a = 0; a < nr; a++) {
                const T xv = sX[a * LD + i];
#pragma unroll
                for (int c = 0; c < CPT; c++) acc[c] += xv * sY[a * LD + j0 + c * TPR];
            }
#pragma unroll
            for (int c = 0; c < CPT; c++) acc64[c] += (double)acc[c];
            __syncthreads();
        }
        T *out = w.Ain + (size_t)b * w.Ain_stride + ((size_t)P * np + pr) * RP * RP;
#pragma unroll
        for (int c = 0; c < CPT; c++) out[i * RP + j0 + c * TPR] = (T)acc64[c];
    } else {
        const double *yb = w.ybuf + (size_t)b * w.y_stride;
        double *wo = w.Ain_w + (size_t)b * w.Ainw_stride + (size_t)P * UC;
        for (int col = tid; col < UC; col += NT) {
            double s = 0.0;
            for (int64_t row = r0; row < r1; row++) s += (double)Ub[(size_t)row * UC + col] * yb[row];
            wo[col] = s;
        }
        if (tid == 0) {
            double d = 0.0, u = 0.0;
            const double *ldu = w.leaf_du + (size_t)b * w.leafdu_stride;
            for (int j = 0; j < J; j++) {
                const int64_t c = (int64_t)P * J + j;
                if (t.leaf_off[c + 1] > t.leaf_off[c]) {
                    d += ldu[2 * c];
                    u += ldu[2 * c + 1];
                }
            }
            double *du = w.Ain_du + (size_t)b * w.Aindu_stride + 2 * (size_t)P;
            du[0] = d;
            du[1] = u;
        }
    }
}

// ------------------------------------------------------------- upward pass --
// Region i of level m: A = sum of the children's ATilde (or the leaf Gram for
// m = M-1); I + A^{m,m} = Lt Lt' (FP64); Z_k = Lt^{-1} A^{m,k}, z = Lt^{-1} w^m;
// ATilde^{k,l} = A^{k,l} - Z_k' Z_l (k <= l < m); wTilde^k = w^k - Z_k' z;
// d += log|I + A^{m,m}|, u -= z'z.  At the root, loglik = -(d + u + n log 2pi)/2.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_up_bytes(int m)
{
    return (size_t)RP * (RP + 1) * sizeof(double) + (size_t)m * RP * sizeof(double) + RP * sizeof(double) +
           32 * sizeof(double) + 16 + (size_t)(2 * m) * RP * (RP + 1) * sizeof(T);
}

template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_up(DevTree t, Work<T> w, int m)
{
    constexpr int LD = RP + 1;
    constexpr int CPT = RP * RP / NT, TPR = RP / CPT;
    const int i = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) {
        if (m == 1 && tid == 0) {
            w.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
            w.status[b] = ST_EINVAL;
        }
        return;
    }
    const int M = t.M, J = t.J;
    const bool direct = (m == M - 1);
    const int nsrc = direct ? 1 : J;
    const int np = npairs(m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sL = (double *)smem_raw;
    double *sw = sL + RP * LD;
    double *sz = sw + m * RP;
    double *red = sz + RP;
    int *flag = (int *)(red + 32);
    T *sC = (T *)(flag + 4);
    T *sZ = sC + (size_t)m * RP * LD;
    T *sLT = sZ + (size_t)(m - 1) * RP * LD;
    const T *blk[4];
    const double *wv[4], *dus[4];
    for (int s = 0; s < nsrc; s++) {
        if (direct) {
            blk[s] = w.Ain + (size_t)b * w.Ain_stride + (size_t)i * np * RP * RP;
            wv[s] = w.Ain_w + (size_t)b * w.Ainw_stride + (size_t)i * m * RP;
            dus[s] = w.Ain_du + (size_t)b * w.Aindu_stride + 2 * (size_t)i;
        } else {
            const int64_t ch = (int64_t)i * J + s;
            blk[s] = w.Atil[m + 1] + (size_t)b * w.Atil_stride[m + 1] + (size_t)ch * np * RP * RP;
            wv[s] = w.Atil_w[m + 1] + (size_t)b * w.Atilw_stride[m + 1] + (size_t)ch * m * RP;
            dus[s] = w.Atil_du[m + 1] + (size_t)b * w.Atildu_stride[m + 1] + 2 * (size_t)ch;
        }
    }
    if (tid == 0) flag[0] = 0;
    for (int k = 1; k <= m; k++) {
        const size_t off = (size_t)pidx(k, m) * RP * RP;
        for (int e = tid; e < RP * RP; e += NT) {
            T v = T(0);
            for (int s = 0; s < nsrc; s++) v += blk[s][off + e];
            sC[(size_t)(k - 1) * RP * LD + (e / RP) * LD + e % RP] = v;
        }
    }
    for (int e = tid; e < m * RP; e += NT) {
        double v = 0.0;
        for (int s = 0; s < nsrc; s++) v += wv[s][e];
        sw[e] = v;
    }
    double dsum = 0.0, usum = 0.0;
    for (int s = 0; s < nsrc; s++) {
        dsum += dus[s][0];
        usum += dus[s][1];
    }
    __syncthreads();
    const T *Cm = sC + (size_t)(m - 1) * RP * LD;
    for (int e = tid; e < RP * RP; e += NT) {
        const int a = e / RP, c = e % RP;
        sL[a * LD + c] = (double)Cm[a * LD + c] + (a == c ? 1.0 : 0.0);
    }
    __syncthreads();
    chol_cta(sL, LD, RP, flag);
    double ld = 0.0;
    for (int a = tid; a < RP; a += NT) ld += log(sL[a * LD + a]);
    ld = 2.0 * block_sum(ld, red);
    for (int e = tid; e < RP * RP; e += NT) sLT[(e / RP) * LD + e % RP] = (T)sL[(e / RP) * LD + e % RP];
    __syncthreads();
    // Z_k[a][bc] = (Lt^{-1} A^{m,k})[a][bc], A^{m,k}[a][bc] = A^{k,m}[bc][a]
    const int ncol = (m - 1) * RP;
    for (int col = tid; col <= ncol; col += NT) {
        if (col < ncol) {
            const int k = col / RP, bc = col % RP;
            const T *Ck = sC + (size_t)k * RP * LD;
            T *Zk = sZ + (size_t)k * RP * LD;
            for (int a = 0; a < RP; a++) {
                T s = Ck[bc * LD + a];
                for (int q = 0; q < a; q++) s -= sLT[a * LD + q] * Zk[q * LD + bc];
                Zk[a * LD + bc] = s / sLT[a * LD + a];
            }
        } else {
            for (int a = 0; a < RP; a++) {
                double s = sw[(m - 1) * RP + a];
                for (int q = 0; q < a; q++) s -= sL[a * LD + q] * sz[q];
                sz[a] = s / sL[a * LD + a];
            }
        }
    }
    __syncthreads();
    double q2 = 0.0;
    for (int a = tid; a < RP; a += NT) q2 += sz[a] * sz[a];
    q2 = block_sum(q2, red);
    const double dR = dsum + ld, uR = usum - q2;
    const int64_t g = t.lvl_off[m] + i;
    if (m > 1) {
        const int npo = npairs(m - 1);
        T *out = w.Atil[m] + (size_t)b * w.Atil_stride[m] + (size_t)i * npo * RP * RP;
        const int ii = tid / TPR, j0 = tid % TPR;
        for (int l = 1; l <= m - 1; l++) {
            for (int k = 1; k <= l; k++) {
                const T *Zk = sZ + (size_t)(k - 1) * RP * LD, *Zl = sZ + (size_t)(l - 1) * RP * LD;
                T acc[CPT];
#pragma unroll
                for (int c = 0; c < CPT; c++) acc[c] = T(0);
                for (int a = 0; a < RP; a++) {
                    const T zv = Zk[a * LD + ii];
#pragma unroll
                    for (int c = 0; c < CPT; c++) acc[c] += zv * Zl[a * LD + j0 + c * TPR];
                }
                const size_t off = (size_t)pidx(k, l) * RP * RP;
#pragma unroll
                for (int c = 0; c < CPT; c++) {
                    const int e = ii * RP + j0 + c * TPR;
                    T v = T(0);
                    for (int s = 0; s < nsrc; s++) v += blk[s][off + e];
                    out[off + e] = v - acc[c];
                }
            }
        }
        double *wo = w.Atil_w[m] + (size_t)b * w.Atilw_stride[m] + (size_t)i * (m - 1) * RP;
        for (int e = tid; e < (m - 1) * RP; e += NT) {
            const int k = e / RP, a = e % RP;
            const T *Zk = sZ + (size_t)k * RP * LD;
            double s = 0.0;
            for (int q = 0; q < RP; q++) s += (double)Zk[q * LD + a] * sz[q];
            wo[e] = sw[e] - s;
        }
        if (tid == 0) {
            double *du = w.Atil_du[m] + (size_t)b * w.Atildu_stride[m] + 2 * (size_t)i;
            du[0] = dR;
            du[1] = uR;
        }
    }
    if (tid == 0) {
        if (flag[0]) w.status[b] = ST_ENOTPD;
        if (w.reg_du) {
            double *r = w.reg_du + (size_t)b * w.regdu_stride + 2 * g;
            r[0] = dR;
            r[1] = uR;
        }
        if (m == 1) {
            const double ll = -0.5 * (dR + uR + (double)t.n_used * 1.8378770664093454836);
            w.loglik[b] = w.status[b] == ST_OK ? ll : __longlong_as_double(0x7ff8000000000000LL);
        }
    }
}

// M = 1: the root is the single leaf.
template <typename T>
__global__ void k_root_single(DevTree t, Work<T> w)
{
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) {
        w.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
        w.status[b] = ST_EINVAL;
        return;
    }
    const double *du = w.leaf_du + (size_t)b * w.leafdu_stride;
    const double ll = -0.5 * (du[0] + du[1] + (double)t.n_used * 1.8378770664093454836);
    w.loglik[b] = w.status[b] == ST_OK ? ll : __longlong_as_double(0x7ff8000000000000LL);
}

} // namespace mra
