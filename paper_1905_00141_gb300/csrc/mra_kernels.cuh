// mra_kernels.cuh -- sm_103a kernels of the MRA log-likelihood.
//
// The GPU evaluates the likelihood of the paper's MRA (Sec. 1.1) in a whitened
// basis.  With L_A the Cholesky factor of W^l_A = C_l(Q_A, Q_A) and
// Linv_A = L_A^{-1}, the basis of a point set P against its level-l ancestor
// A_l is What^l_P = C_l(P, Q_{A_l}) Linv_{A_l}', and the recursion of the
// remainder covariances becomes
//     W^l_P    = C(P, Q_{A_l}) - sum_{k<l} What^k_P (What^k_{A_l})'
//     What^l_P = W^l_P Linv_{A_l}'
// with an identity prior precision at every level.  The upward pass then
// factors I + A^{m,m}; log-determinants and quadratic forms are unchanged
// (|K^{-1} + A| / |K^{-1}| = |I + L^{-1} A L^{-T}|).
//
// Work decomposition (256 threads per CTA): one CTA per region for the prior
// and the upward pass, one per chunk of observation rows for the leaf basis,
// one per leaf for the leaf posterior, one per (level-(M-1) region, block
// column) for the leaf Gram.  r_hat knots are padded to RP (16 or 32) with
// inert padding (zero covariance rows and columns, identity on the padded
// diagonal of every factor), which leaves every result exact.
//
// Precision: T is the storage and product type (double, or float in the mixed
// mode).  Cholesky factors, log-determinants, quadratic forms and the
// accumulation of the leaf-level y vectors are FP64 in both modes.  In the
// mixed mode the leaf covariance C + tau2 I - U U' is formed with exact FP32
// products summed as unevaluated float pairs and an exact leading subtraction,
// so its FP32 rounding is relative to V itself and not to C.
//
// Operand layouts in shared memory are "k-major": a row-block X (rows x K) is
// stored as X[k][row], so the inner product loops read contiguous vectors.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ff_math.h"
#include "mra_internal.h"

namespace mra {

constexpr int NT = MRA_NT;
enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOTPD = 3 };

// Singularity rule shared by every factorisation: a pivot at or below
// MRA_SINGULAR times the largest diagonal entry of the matrix is singular
// (coincident knots make the covariance singular, Sec. 1.2).
#define MRA_SINGULAR 1e-12

__host__ __device__ __forceinline__ int npairs(int D) { return D * (D + 1) / 2; }
__host__ __device__ __forceinline__ int pidx(int k, int l) { return l * (l - 1) / 2 + k - 1; }
__host__ __device__ __forceinline__ constexpr int tri_count(int w) { return w * (w + 1) / 2; }

// finite and > 0, from the bits (integer operations: FP64 compares cost ~230
// cycles of latency each on this GPU, at the head of every CTA)
__device__ __forceinline__ bool pos_finite(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return b - 1ull < 0x7FEFFFFFFFFFFFFFull; // +0 < v < +inf, no NaN, no sign bit
}
__device__ __forceinline__ bool theta_ok(const double *th)
{
    return pos_finite(th[0]) && pos_finite(th[1]) && pos_finite(th[2]);
}

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000LL); }

// Covariance parameters in the storage type.
template <typename T>
struct CovP {
    T s2, ib; // sigma2 and 1/beta
    __device__ CovP(double sigma2, double inv_beta) : s2((T)sigma2), ib((T)inv_beta) {}
};

// Exponential covariance sigma2 * exp(-|d| / beta) of a coordinate difference
// (Sec. 2.2.4 reading of "exponential covariance function").
__device__ __forceinline__ double cov_d(const CovP<double> &c, double dx, double dy)
{
    return c.s2 * exp(-sqrt(dx * dx + dy * dy) * c.ib);
}
__device__ __forceinline__ float cov_d(const CovP<float> &c, float dx, float dy)
{
    return c.s2 * expf(-sqrtf(dx * dx + dy * dy) * c.ib);
}

// ------------------------------------------------------------ small tools --
template <typename T, int N>
__device__ __forceinline__ void ldv(T (&r)[N], const T *p)
{
    if constexpr (sizeof(T) == 4 && N == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if constexpr (sizeof(T) == 8 && N == 2) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        r[0] = v.x; r[1] = v.y;
    } else if constexpr (sizeof(T) == 4 && N == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        r[0] = v.x; r[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; i++) r[i] = p[i];
    }
}

// Copy n elements (a multiple of 16 bytes, 16-byte aligned on both sides)
// from global to shared memory.
template <typename T>
__device__ __forceinline__ void copy_g2s(T *s, const T *g, int n)
{
    const int4 *src = reinterpret_cast<const int4 *>(g);
    int4 *dst = reinterpret_cast<int4 *>(s);
    const int nv = n * (int)sizeof(T) / 16;
    for (int e = threadIdx.x; e < nv; e += NT) dst[e] = src[e];
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only); each
// thread waits for its own groups, a barrier then publishes them.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// n elements (a multiple of 16 bytes, 16-byte aligned on both sides)
template <typename T>
__device__ __forceinline__ void copy_g2s_async(T *s, const T *g, int n)
{
    const int nv = n * (int)sizeof(T) / 16;
    const char *src = reinterpret_cast<const char *>(g);
    char *dst = reinterpret_cast<char *>(s);
    for (int e = threadIdx.x; e < nv; e += NT) cp_async16(dst + 16 * e, src + 16 * e);
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NT / 32 ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// Thread tile of a ROWS x COLS output spread over NT threads.
template <int ROWS, int COLS>
struct Tile {
    static constexpr int OUT = ROWS * COLS / NT;
    static constexpr int CT = OUT % 4 == 0 ? 4 : (OUT % 2 == 0 ? 2 : 1);
    static constexpr int RT = OUT / CT;
    static constexpr int TX = COLS / CT;
    static_assert(OUT >= 1 && RT * CT == OUT && (ROWS / RT) * TX == NT, "tile shape");
    __device__ static int r0() { return (threadIdx.x / TX) * RT; }
    __device__ static int c0() { return (threadIdx.x % TX) * CT; }
};

// acc[r][c] += sum_t A[t][r0 + r] * B[t][c0 + c]  (both operands k-major)
template <typename T, int ROWS, int COLS>
__device__ __forceinline__ void tile_fma(T (&acc)[Tile<ROWS, COLS>::RT][Tile<ROWS, COLS>::CT], const T *A,
                                         int lda, const T *B, int ldb, int K)
{
    using TL = Tile<ROWS, COLS>;
    const int r0 = TL::r0(), c0 = TL::c0();
#pragma unroll 4
    for (int t = 0; t < K; t++) {
        T a[TL::RT], b[TL::CT];
        ldv<T, TL::RT>(a, A + t * lda + r0);
        ldv<T, TL::CT>(b, B + t * ldb + c0);
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
}

template <typename T, int RT, int CT>
__device__ __forceinline__ void tile_zero(T (&acc)[RT][CT])
{
#pragma unroll
    for (int r = 0; r < RT; r++)
#pragma unroll
        for (int c = 0; c < CT; c++) acc[r][c] = T(0);
}

// Exact FP32 product sum: every product split by an FMA (TwoProd) and the
// running sum kept as an unevaluated pair (hi, lo) by TwoSum.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add_prod(FF &s, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(t, s.hi);
    const float r = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(r, e));
}
__device__ __forceinline__ void ff_add(FF &s, float p)
{
    const float t = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(t, s.hi);
    const float r = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, r);
}

// sum_k a[k] b[k] returned as (hi, lo): FP32 pairs exact, FP64 plain.
__device__ __forceinline__ void ff_merge(FF &s, const FF &o)
{
    ff_add(s, o.hi);
    s.lo = __fadd_rn(s.lo, o.lo);
}
// acc[r][c] = sum_t A[t][r0 + r] * B[t][c0 + c] for rows of whitened basis
// functions, to an absolute error near 1e-11 sigma2.  Since
// sum_k |What^k(x)|^2 <= C(x, x) = sigma2 (Sec. 1.1: the remainder covariance
// stays positive), Cauchy-Schwarz bounds every partial sum of |a_t b_t| by
// sigma2, so the grid accumulation of ff_math.h applies with
// Cq = grid_constant(sigma2): four FP32 operations a product instead of the
// ten of a float-pair TwoSum accumulation of TwoProd products.
template <int ROWS, int COLS>
__device__ __forceinline__ void tile_fma_ff(FF (&acc)[Tile<ROWS, COLS>::RT][Tile<ROWS, COLS>::CT], const float *A,
                                            int lda, const float *B, int ldb, int K, float Cq)
{
    using TL = Tile<ROWS, COLS>;
    const int r0 = TL::r0(), c0 = TL::c0();
    grid_acc g[TL::RT][TL::CT];
#pragma unroll
    for (int r = 0; r < TL::RT; r++)
#pragma unroll
        for (int c = 0; c < TL::CT; c++) grid_init(g[r][c], Cq);
    for (int t = 0; t < K; t++) {
        float a[TL::RT], b[TL::CT];
        ldv<float, TL::RT>(a, A + t * lda + r0);
        ldv<float, TL::CT>(b, B + t * ldb + c0);
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) grid_add(g[r][c], a[r], b[c]);
    }
#pragma unroll
    for (int r = 0; r < TL::RT; r++)
#pragma unroll
        for (int c = 0; c < TL::CT; c++) {
            const ff v = grid_value(g[r][c], Cq);
            acc[r][c] = FF{v.hi, v.lo};
        }
}

// The grid accumulation of tile_fma_ff over K terms without its start and its
// rounding (the streaming leaf basis accumulates one staged part of K at a
// time, in the same order of terms).
template <int ROWS, int COLS>
__device__ __forceinline__ void tile_grid_add(grid_acc (&g)[Tile<ROWS, COLS>::RT][Tile<ROWS, COLS>::CT], const float *A,
                                              int lda, const float *B, int ldb, int K)
{
    using TL = Tile<ROWS, COLS>;
    const int r0 = TL::r0(), c0 = TL::c0();
    for (int t = 0; t < K; t++) {
        float a[TL::RT], b[TL::CT];
        ldv<float, TL::RT>(a, A + t * lda + r0);
        ldv<float, TL::CT>(b, B + t * ldb + c0);
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) grid_add(g[r][c], a[r], b[c]);
    }
}

// The remainder C(P, Q) - sum_k What^k(P) What^k(Q)' of one RP-column block
// (Sec. 1.1 recursion) for FP32 storage, with the covariance in float pairs
// and the product sum to ~1e-11 sigma2 (tile_fma_ff): the prior evaluates it
// at knots and the leaf basis at observations, and the two must agree far
// below FP32 relative to sigma2 where the remainder is small (deep levels,
// long ranges).  P coordinates at pp[a], pp[ldp + a] (nP valid rows), Q at
// pq[j], pq[RP + j] (R valid); sigma2 and 1/beta as float pairs (s2f, ibf),
// Cq = grid_constant(sigma2).  out[r][c] is entry (r0 + r, c0 + c) rounded to
// FP32.
template <int ROWS, int RP>
__device__ __forceinline__ void remainder_ff(float (&out)[Tile<ROWS, RP>::RT][Tile<ROWS, RP>::CT], const float *Ak,
                                             int lda, const float *Bk, int K, const float *pp, int ldp, int nP,
                                             const float *pq, int R, ff s2f, ff ibf, float Cq)
{
    using TL = Tile<ROWS, RP>;
    FF fa[TL::RT][TL::CT];
    tile_fma_ff<ROWS, RP>(fa, Ak, lda, Bk, RP, K, Cq);
    const int r0 = TL::r0(), c0 = TL::c0();
#pragma unroll
    for (int r = 0; r < TL::RT; r++)
#pragma unroll
        for (int c = 0; c < TL::CT; c++) {
            const int a = r0 + r, j = c0 + c;
            ff cv = ff{0.f, 0.f};
            if (a < nP && j < R)
                cv = ff_cov_exp(s2f, ibf, pp[a], pp[ldp + a], pq[j], pq[RP + j]);
            // rounded to FP32: the leading parts subtract exactly when they
            // are close (Sterbenz), the trailing parts only move the last bit
            out[r][c] = FADD(FSUB(cv.hi, fa[r][c].hi), FSUB(cv.lo, fa[r][c].lo));
        }
}

__device__ __forceinline__ void dot2(const float *a, const float *b, int K, float &hi, float &lo)
{
    // four independent pairs for instruction-level parallelism, merged exactly
    FF s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f}, s3{0.f, 0.f};
    int k = 0;
    for (; k + 4 <= K; k += 4) {
        ff_add_prod(s0, a[k], b[k]);
        ff_add_prod(s1, a[k + 1], b[k + 1]);
        ff_add_prod(s2, a[k + 2], b[k + 2]);
        ff_add_prod(s3, a[k + 3], b[k + 3]);
    }
    for (; k < K; k++) ff_add_prod(s0, a[k], b[k]);
    ff_merge(s0, s1);
    ff_merge(s2, s3);
    ff_merge(s0, s2);
    hi = s0.hi;
    lo = s0.lo;
}
__device__ __forceinline__ void dot2(const double *a, const double *b, int K, double &hi, double &lo)
{
    double s = 0.0;
    for (int k = 0; k < K; k++) s = fma(a[k], b[k], s);
    hi = s;
    lo = 0.0;
}

// The four sums a_i . q_j (i, j in {0, 1}) over K terms (K a multiple of 8,
// rows 16-byte aligned).  FP32: each group of 8 products is summed by an FMA
// chain in FP32 and the group sums are accumulated as float pairs (TwoSum), so
// the rounding is that of an 8-term FP32 sum per group -- the order of the
// error already carried by the FP32 operands -- while the 2x2 block reuses
// every loaded element twice.  FP64: plain FMA chains.
__device__ __forceinline__ void dot2x2(const float *a0, const float *a1, const float *q0, const float *q1, int K,
                                       float (&hi)[2][2], float (&lo)[2][2])
{
    FF s[2][2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) s[i][j] = FF{0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 8) {
        float p[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int k = k0; k < k0 + 8; k += 4) {
            const float4 x[2] = {*(const float4 *)(a0 + k), *(const float4 *)(a1 + k)};
            const float4 y[2] = {*(const float4 *)(q0 + k), *(const float4 *)(q1 + k)};
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    p[i][j] = __fmaf_rn(x[i].x, y[j].x, p[i][j]);
                    p[i][j] = __fmaf_rn(x[i].y, y[j].y, p[i][j]);
                    p[i][j] = __fmaf_rn(x[i].z, y[j].z, p[i][j]);
                    p[i][j] = __fmaf_rn(x[i].w, y[j].w, p[i][j]);
                }
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) ff_add(s[i][j], p[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const float t = __fadd_rn(s[i][j].hi, s[i][j].lo);
            hi[i][j] = t;
            lo[i][j] = __fsub_rn(s[i][j].lo, __fsub_rn(t, s[i][j].hi));
        }
}
// As dot2x2 to float-float accuracy, for leaves whose covariance loses many
// digits to cancellation (tight clusters of observations): the rows are
// whitened basis rows, so every partial sum of |products| is below sigma2 and
// the grid accumulation of ff_math.h applies (Cq = grid_constant(sigma2)).
__device__ __forceinline__ void dot2x2_exact(const float *a0, const float *a1, const float *q0, const float *q1,
                                             int K, float Cq, float (&hi)[2][2], float (&lo)[2][2])
{
    grid_acc g[2][2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) grid_init(g[i][j], Cq);
    for (int k = 0; k < K; k += 4) {
        const float4 x4[2] = {*(const float4 *)(a0 + k), *(const float4 *)(a1 + k)};
        const float4 y4[2] = {*(const float4 *)(q0 + k), *(const float4 *)(q1 + k)};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float x[2] = {(&x4[0].x)[e], (&x4[1].x)[e]}, y[2] = {(&y4[0].x)[e], (&y4[1].x)[e]};
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) grid_add(g[i][j], x[i], y[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const ff v = grid_value(g[i][j], Cq);
            hi[i][j] = v.hi;
            lo[i][j] = v.lo;
        }
}
__device__ __forceinline__ void dot2x2(const double *a0, const double *a1, const double *q0, const double *q1, int K,
                                       double (&hi)[2][2], double (&lo)[2][2])
{
    double p[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k = 0; k < K; k++) {
        const double x[2] = {a0[k], a1[k]}, y[2] = {q0[k], q1[k]};
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) p[i][j] = fma(x[i], y[j], p[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            hi[i][j] = p[i][j];
            lo[i][j] = 0.0;
        }
}
// The grid accumulation of dot2x2_exact over K terms without its start and
// its rounding (large leaves of deep trees read their rows in parts).
__device__ __forceinline__ void dot2x2_grid_add(grid_acc (&g)[2][2], const float *a0, const float *a1, const float *q0,
                                                const float *q1, int K)
{
    for (int k = 0; k < K; k += 4) {
        const float4 x4[2] = {*(const float4 *)(a0 + k), *(const float4 *)(a1 + k)};
        const float4 y4[2] = {*(const float4 *)(q0 + k), *(const float4 *)(q1 + k)};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float x[2] = {(&x4[0].x)[e], (&x4[1].x)[e]}, y[2] = {(&y4[0].x)[e], (&y4[1].x)[e]};
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) grid_add(g[i][j], x[i], y[j]);
        }
    }
}
__device__ __forceinline__ void dot2x2_exact(const double *a0, const double *a1, const double *q0, const double *q1,
                                             int K, float, double (&hi)[2][2], double (&lo)[2][2])
{
    dot2x2(a0, a1, q0, q1, K, hi, lo);
}

// C - (hi + lo) with the leading subtraction done first: when C and hi agree
// to a factor of two the difference is exact, so the rounding left is
// relative to the (small) result.
__device__ __forceinline__ double cancel_sub(float c, float hi, float lo)
{
    return (double)__fsub_rn(__fsub_rn(c, hi), lo);
}
__device__ __forceinline__ double cancel_sub(double c, double hi, double lo) { return (c - hi) - lo; }
__device__ __forceinline__ double cancel_sub(double c, float hi, float lo) { return (c - (double)hi) - (double)lo; }

// FP64 exponential covariance for the leaf covariance V, whose small
// eigenvalues (~tau2) are far below C's entries (~sigma2): C must carry more
// than FP32 accuracy there.
__device__ __forceinline__ double cov64(double s2, double ib, double dx, double dy)
{
    return s2 * exp(-sqrt(dx * dx + dy * dy) * ib);
}

// sigma2 and 1/beta for a CTA, in shared memory, by threads 0 and 1 side by
// side.  FP64 mode: 1/beta as a double.  Mixed modes: both as float pairs,
// 1/beta by a float-pair reciprocal on the FP32 pipe (an FP64 division costs
// ~440 cycles of latency on this GPU, at the head of every CTA), and s_ib its
// leading float (what the FP32 covariance of the fast mode uses).
template <typename T>
__device__ __forceinline__ void set_cov_params(const double *th, double *s_ib, ff *s_par)
{
    if constexpr (sizeof(T) == 4) {
        if (threadIdx.x == 0) s_par[0] = ff_from_double(th[0]);
        if (threadIdx.x == 1) {
            const ff ib = ff_rcp(ff_from_double(th[1]));
            s_par[1] = ib;
            *s_ib = (double)ib.hi;
        }
    } else {
        if (threadIdx.x == 0) s_par[0] = ff_from_double(th[0]);
        if (threadIdx.x == 1) {
            *s_ib = 1.0 / th[1];
            s_par[1] = ff_from_double(*s_ib);
        }
    }
}

// ------------------------------------------------------------- Cholesky --
// Factor arithmetic: F = double in the FP64 mode, F = ff (float pair, ~48-bit
// mantissa, FP32 pipe) in the mixed mode.  On GB300 a warp-wide FP64
// instruction holds its sub-partition's FP64 unit for ~64 cycles, so the
// serial chains of a small Cholesky (pivots, triangular solves) run much
// faster in float pairs at comparable accuracy.
template <typename T> struct FacT { using type = double; };
template <> struct FacT<float> { using type = ff; };

__device__ __forceinline__ double f_mul(double a, double b) { return a * b; }
__device__ __forceinline__ ff f_mul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double f_sub(double a, double b) { return a - b; }
__device__ __forceinline__ ff f_sub(ff a, ff b) { return ff_sub(a, b); }
// the subtraction of a factorisation update (absolute accuracy suffices)
__device__ __forceinline__ double f_sub_upd(double a, double b) { return a - b; }
__device__ __forceinline__ ff f_sub_upd(ff a, ff b) { return ff_sub_sloppy(a, b); }
__device__ __forceinline__ double f_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff f_add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ double f_sqr(double a) { return a * a; }
__device__ __forceinline__ ff f_sqr(ff a) { return ff_sqr(a); }
__device__ __forceinline__ double f_rsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ ff f_rsqrt(ff a) { return ff_rsqrt(a); }
__device__ __forceinline__ double f_hi(double a) { return a; }
__device__ __forceinline__ float f_hi(ff a) { return a.hi; }
__device__ __forceinline__ double f_dbl(double a) { return a; }
__device__ __forceinline__ double f_dbl(ff a) { return ff_to_double(a); }
template <typename F> __device__ __forceinline__ F f_of(double v);
template <> __device__ __forceinline__ double f_of<double>(double v) { return v; }
template <> __device__ __forceinline__ ff f_of<ff>(double v) { return ff_from_double(v); }
template <typename F> __device__ __forceinline__ F f_of_f(float v);
template <> __device__ __forceinline__ double f_of_f<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ ff f_of_f<ff>(float v) { return ff{v, 0.f}; }
__device__ __forceinline__ double f_shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ ff f_shfl(ff v, int src)
{
    return ff{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ double f_shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ ff f_shfl_xor(ff v, int m)
{
    return ff{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// Lower-triangle positions (i, k), k <= i < n, are ordered by decreasing k
// (e = 0 is (n-1, n-1)), so the positions still updated at column j are the
// first tri(n-1-j) of the order.
// Cholesky of a small (n <= 64) symmetric matrix in shared memory by the
// whole CTA, one barrier per column.  Input: the lower triangle of A.  Output:
// the factor L in the UPPER triangle, transposed (A[j][i] = L[i][j], i >= j,
// diagonal included), and rs[j] = 1 / L_jj; the lower triangle is left as
// scratch.  Thread t owns the lower-triangle positions t, t + NT, ... of the
// pair order of build_pairs and keeps their values in registers through all
// column steps; only an entry that becomes part of the next pivot column is
// written back to shared memory.  The owner of the next diagonal entry also
// forms its reciprocal square root (and its square), so each pivot is ready at
// the barrier.  A pivot at or below `rel` times the largest diagonal entry is
// singular: it sets *fail and is replaced by 1.  rs, r2s: n + 1 entries of
// shared scratch.  S = pairs per thread (ceil(n(n+1)/2 / NT)).
template <typename F, int S>
static __device__ void chol_small(F *A, int lda, int n, F *rs, F *r2s, int *fail, double rel)
{
    int pi[S], pk[S];
    F val[S];
    const int P = tri_count(n);
#pragma unroll
    for (int s = 0; s < S; s++) {
        const int e = threadIdx.x + s * NT;
        pi[s] = -1;
        pk[s] = -1;
        if (e < P) {
            int w = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f) + 1;
            while (tri_count(w) <= e) w++;
            while (w > 1 && tri_count(w - 1) > e) w--;
            pk[s] = n - w;
            pi[s] = pk[s] + (e - tri_count(w - 1));
            val[s] = A[pi[s] * lda + pk[s]];
        }
    }
    if (threadIdx.x < 32) {
        double sc = 0.0;
        for (int j = threadIdx.x; j < n; j += 32) sc = fmax(sc, (double)f_hi(A[j * lda + j]));
        for (int o = 16; o; o >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
        if (threadIdx.x == 0) {
            const double tol = rel * sc;
            F d = A[0];
            if (!((double)f_hi(d) > tol)) {
                *fail = 1;
                d = f_of<F>(1.0);
                A[0] = d;
            }
            rs[0] = f_rsqrt(d);
            r2s[0] = f_sqr(rs[0]);
            rs[n] = f_of<F>(tol);
        }
    }
    __syncthreads();
    const double tol = (double)f_hi(rs[n]);
    for (int j = 0; j < n; j++) {
        const F r = rs[j], r2 = r2s[j];
        for (int i = j + threadIdx.x; i < n; i += NT) A[j * lda + i] = f_mul(A[i * lda + j], r);
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int i = pi[s], k = pk[s];
            if (k > j) {
                F v = f_sub_upd(val[s], f_mul(f_mul(A[i * lda + j], A[k * lda + j]), r2));
                if (k == j + 1) {
                    if (i == k) {
                        if (!((double)f_hi(v) > tol)) {
                            *fail = 1;
                            v = f_of<F>(1.0);
                        }
                        const F rk = f_rsqrt(v);
                        rs[k] = rk;
                        r2s[k] = f_sqr(rk);
                    }
                    A[i * lda + k] = v;
                }
                val[s] = v;
            }
        }
        __syncthreads();
    }
}

// One step of an error-free dot product in float pairs (Ogita, Rump and
// Oishi's Dot2, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// the leading product is split exactly by an FMA (TwoProd), added to the
// running sum exactly (TwoSum), and both rounding errors plus the cross terms
// of the pairs' trailing parts go into a compensation term c.  The value of the
// sum is s + c; it is as accurate as if computed in twice the FP32 precision.
struct Dot2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(ff a, ff b)
    {
        const float p = __fmul_rn(a.hi, b.hi);
        const float pe = __fmaf_rn(a.hi, b.hi, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        // the four small terms first: one dependent addition per step on c
        c = __fadd_rn(c, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fadd_rn(pe, se))));
    }
    __device__ __forceinline__ void merge(const Dot2 &o)
    {
        const ff u = two_sum(s, o.s);
        s = u.hi;
        c = __fadd_rn(__fadd_rn(c, o.c), u.lo);
    }
    __device__ __forceinline__ ff value() const { return two_sum(s, c); }
};

// Cholesky of a small (n <= NMAX <= 64) symmetric matrix in shared memory by
// the whole CTA in float pairs, blocked by 8 columns: the same input and
// output as chol_small (input: the lower triangle of A; output: L in the upper
// triangle, transposed, A[j][i] = L[i][j] for i >= j, and rs[j] = 1 / L_jj;
// the same singularity rule), two barriers per block instead of one per
// column.  For each block of columns [c0, c0 + 8):
//   - warp 0 factors the panel (rows c0..n-1 of those columns) in registers,
//     lane l holding rows c0 + l (+ 32): column c0 + j is
//     A_ij - sum_{p<j} L_i,c0+p L_c0+j,c0+p (row c0 + j broadcast by
//     shuffles, the sum error-free in pairs by Dot2), lane j takes the pivot and
//     the column is scaled by its reciprocal square root;
//   - every thread then applies the panel to the trailing lower triangle,
//     A_ik -= sum_p L_i,c0+p L_k,c0+p (Dot2 over the block's 8 columns).
// The pivot chain (reciprocal square root, scaling, the next diagonal) stays in
// one warp's registers; the CTA-wide update needs no per-column barrier.
template <int NMAX>
static __device__ void chol_blocked(ff *A, int lda, int n, ff *rs, int *fail, double rel, double *red)
{
    static_assert(NMAX <= 64, "two rows per lane at most");
    constexpr int BS = 8, RPL = NMAX > 32 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the singularity test in FP32 (an FP64 compare on the pivot chain costs
    // ~230 cycles per column on this GPU)
    float *tolp = reinterpret_cast<float *>(red);
    if (warp == 0) {
        float sc = 0.f;
        for (int j = lane; j < n; j += 32) sc = fmaxf(sc, A[j * lda + j].hi);
        for (int o = 16; o; o >>= 1) sc = fmaxf(sc, __shfl_xor_sync(0xffffffffu, sc, o));
        if (lane == 0) tolp[0] = (float)rel * sc;
    }
    for (int c0 = 0; c0 < n; c0 += BS) {
        const int w = min(BS, n - c0);
        if (warp == 0) {
            const float tol = tolp[0];
            ff a[RPL][BS];
#pragma unroll
            for (int q = 0; q < RPL; q++) {
                const int i = c0 + lane + 32 * q;
#pragma unroll
                for (int p = 0; p < BS; p++) a[q][p] = (i < n && p < w && c0 + p <= i) ? A[i * lda + c0 + p] : ff{0.f, 0.f};
            }
#pragma unroll
            for (int j = 0; j < BS; j++) {
                if (j < w) {
                    // row c0 + j is lane j's first row
                    ff s[RPL];
#pragma unroll
                    for (int q = 0; q < RPL; q++) {
                        Dot2 d;
#pragma unroll
                        for (int p = 0; p < j; p++) d.add(a[q][p], f_shfl(a[0][p], j));
                        s[q] = ff_sub_sloppy(a[q][j], d.value());
                    }
                    ff r = ff{0.f, 0.f};
                    if (lane == j) {
                        ff dj = s[0];
                        if (!(dj.hi > tol)) {
                            *fail = 1;
                            dj = ff{1.f, 0.f};
                        }
                        r = ff_rsqrt(dj);
                        rs[c0 + j] = r;
                        a[0][j] = ff_mul(dj, r);
                    }
                    r = f_shfl(r, j);
#pragma unroll
                    for (int q = 0; q < RPL; q++) {
                        const int i = c0 + lane + 32 * q;
                        if (i > c0 + j && i < n) a[q][j] = ff_mul(s[q], r);
                    }
                }
            }
            // the panel's columns of L, transposed into the upper triangle
#pragma unroll
            for (int q = 0; q < RPL; q++) {
                const int i = c0 + lane + 32 * q;
#pragma unroll
                for (int p = 0; p < BS; p++)
                    if (i < n && p < w && c0 + p <= i) A[(c0 + p) * lda + i] = a[q][p];
            }
        }
        __syncthreads();
        // trailing lower triangle: rows and columns from c0 + w on
        const int t0 = c0 + w, tn = n - t0;
        if (tn > 0) {
            for (int e = threadIdx.x; e < tri_count(tn); e += NT) {
                int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (tri_count(ii + 1) <= e) ii++;
                while (ii > 0 && tri_count(ii) > e) ii--;
                const int i = t0 + ii, k = t0 + (e - tri_count(ii));
                Dot2 d;
#pragma unroll
                for (int p = 0; p < BS; p++)
                    if (p < w) d.add(A[(c0 + p) * lda + i], A[(c0 + p) * lda + k]);
                A[i * lda + k] = ff_sub_sloppy(A[i * lda + k], d.value());
            }
            __syncthreads();
        }
    }
}

// 2 sum_j log L_jj of a chol_small factor, by warp 0.  FP64: the pivots are
// multiplied as mantissas with a running exponent and one log is taken.
// Float pairs: each lane splits its pivots into exponent and mantissa in
// [1, 2) and sums logf of the mantissas (absolute error ~4e-8 per pivot).
__device__ __forceinline__ double logdet_small(const double *A, int lda, int n, double *out)
{
    if (threadIdx.x < 32) {
        double prod = 1.0;
        int ex = 0;
        for (int j = threadIdx.x; j < n; j += 32) {
            int e;
            prod = frexp(prod * A[j * lda + j], &e);
            ex += e;
        }
        for (int o = 16; o; o >>= 1) {
            const double q = __shfl_xor_sync(0xffffffffu, prod, o);
            const int eo = __shfl_xor_sync(0xffffffffu, ex, o);
            int e;
            prod = frexp(prod * q, &e);
            ex += eo + e;
        }
        if (threadIdx.x == 0) *out = 2.0 * (log(prod) + (double)ex * 0.69314718055994530942);
    }
    __syncthreads();
    const double v = *out;
    __syncthreads();
    return v;
}
__device__ __forceinline__ double logdet_small(const ff *A, int lda, int n, double *out)
{
    if (threadIdx.x < 32) {
        ff s{0.f, 0.f};
        int ex = 0;
        for (int j = threadIdx.x; j < n; j += 32) {
            const ff p = A[j * lda + j];
            int e;
            const float m = 2.0f * frexpf(p.hi, &e); // p.hi = m 2^(e-1), m in [1, 2)
            ex += e - 1;
            s = ff_add(s, ff{logf(m), p.lo / p.hi});
        }
        for (int o = 16; o; o >>= 1) {
            s = ff_add(s, f_shfl_xor(s, o));
            ex += __shfl_xor_sync(0xffffffffu, ex, o);
        }
        if (threadIdx.x == 0) *out = 2.0 * (ff_to_double(s) + (double)ex * 0.69314718055994530942);
    }
    __syncthreads();
    const double v = *out;
    __syncthreads();
    return v;
}

// The leading float of a factor entry, as a factor-type value (float pairs:
// the pair (hi, 0); FP64: the value itself).
__device__ __forceinline__ ff f_lead(ff a) { return ff{a.hi, 0.f}; }
__device__ __forceinline__ double f_lead(double a) { return a; }

// y <- L^{-1} y with the chol_small factor (L[a][q] = A[q][a]) and rs = 1/L_jj,
// by warp 0, right-looking: lane a (and a + 32) owns y[a]; after y[q] is
// final it is broadcast and every later row subtracts its share.  With LEAD,
// the operator is the leading floats of L and rs (the FP32 factor the solves
// of the storage-type right-hand sides use), applied in float-pair arithmetic:
// y then belongs to the same operator as those solves, which keeps the
// quadratic forms of the upward pass consistent with the Gram blocks.
template <typename F, bool LEAD = false>
__device__ void fwd_solve_vec(const F *A, int lda, const F *rs, int n, F *y)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        F y0 = lane < n ? y[lane] : f_of<F>(0.0);
        F y1 = lane + 32 < n ? y[lane + 32] : f_of<F>(0.0);
        for (int q = 0; q < n; q++) {
            const bool mine0 = (q == lane), mine1 = (q == lane + 32);
            const F rq = LEAD ? f_lead(rs[q]) : rs[q];
            if (mine0) y0 = f_mul(y0, rq);
            if (mine1) y1 = f_mul(y1, rq);
            const F yq = q < 32 ? f_shfl(y0, q) : f_shfl(y1, q - 32);
            if (lane > q && lane < n) {
                const F l = A[q * lda + lane];
                y0 = f_sub(y0, f_mul(LEAD ? f_lead(l) : l, yq));
            }
            if (lane + 32 > q && lane + 32 < n) {
                const F l = A[q * lda + lane + 32];
                y1 = f_sub(y1, f_mul(LEAD ? f_lead(l) : l, yq));
            }
        }
        if (lane < n) y[lane] = y0;
        if (lane + 32 < n) y[lane + 32] = y1;
    }
    __syncthreads();
}

// y <- L^{-1} y as fwd_solve_vec<F, true> (the leading floats of L and rs,
// applied in factor arithmetic; the same operations, so the same result) for
// n <= N <= 32, with lane a's row of L and its reciprocal pivot loaded into
// registers first: each step is a scale, one shuffle and one update per lane,
// with no shared-memory load on the chain.  By warp 0; ends with a barrier.
template <typename F, int N>
__device__ void fwd_solve_vec_lead_warp(const F *A, int lda, const F *rs, int n, F *y)
{
    static_assert(N <= 32, "one row per lane");
    {
        const int lane = threadIdx.x & 31;
        F Lr[N];
#pragma unroll
        for (int q = 0; q < N; q++) Lr[q] = (q < lane && lane < n) ? f_lead(A[q * lda + lane]) : f_of<F>(0.0);
        const F rl = lane < n ? f_lead(rs[lane]) : f_of<F>(0.0);
        F yl = lane < n ? y[lane] : f_of<F>(0.0);
#pragma unroll
        for (int q = 0; q < N; q++) {
            if (q < n) {
                if (lane == q) yl = f_mul(yl, rl);
                const F yq = f_shfl(yl, q);
                if (lane > q && lane < n) yl = f_sub(yl, f_mul(Lr[q], yq));
            }
        }
        if (lane < n) y[lane] = yl;
    }
}
template <typename F, int N>
__device__ void fwd_solve_vec_lead(const F *A, int lda, const F *rs, int n, F *y)
{
    if (threadIdx.x < 32) fwd_solve_vec_lead_warp<F, N>(A, lda, rs, n, y);
    __syncthreads();
}

// sum_k a_k b_k with a in the storage type and b in the factor type: float x
// float-pair products exact in their leading part (TwoProd), the trailing
// part summed in FP32; FP64: plain FMA.
template <typename T, typename F> struct DotTF;
template <> struct DotTF<float, ff> {
    FF s{0.f, 0.f};
    float side = 0.f;
    __device__ __forceinline__ void add(float a, ff b)
    {
        ff_add_prod(s, a, b.hi);
        side = __fmaf_rn(a, b.lo, side);
    }
    __device__ __forceinline__ ff value() const { return fast_two_sum(s.hi, __fadd_rn(s.lo, side)); }
};
template <> struct DotTF<double, double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ ff f_of_ff(ff v) { return v; }
__device__ __forceinline__ ff f_of_ff(double v) { return ff_from_double(v); }
__device__ __forceinline__ double f_of_T(double v) { return v; }
__device__ __forceinline__ ff f_of_T(float v) { return ff{v, 0.f}; }

template <typename F>
__device__ __forceinline__ F warp_sum_f(F v)
{
    for (int o = 16; o; o >>= 1) v = f_add(v, f_shfl_xor(v, o));
    return v;
}

// L^{-1} of the chol_small factor (L[k][i] = A[i][k], n <= NMAX <= 64),
// written column-major into out (ld ldo: out[col * ldo + i] = (L^{-1})[i][col],
// zeros above the diagonal), which is also the k-major layout of L^{-1} as a
// left GEMM operand; out may be global or shared memory, not aliasing A.
// Warps own columns (col = warp + 8c), lanes own rows (lane, lane + 32): at
// step i row i of every column is final, one shuffle broadcasts it and each
// lane updates its later rows with L[k][i], read once per step for all the
// warp's columns.  Reads of A and writes of out are lane-contiguous.
template <typename T, int NMAX, typename F>
__device__ void trinv_warp(const F *A, int lda, const F *rs, T *out, int ldo, int n)
{
    constexpr int NW = NT / 32, RPL = NMAX > 32 ? 2 : 1, CPW = (NMAX + NW - 1) / NW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T x[CPW][RPL];
#pragma unroll
    for (int c = 0; c < CPW; c++)
#pragma unroll
        for (int r = 0; r < RPL; r++) x[c][r] = (lane + 32 * r == warp + NW * c) ? T(1) : T(0);
    for (int i = warp; i < n; i++) {
        T l[RPL];
#pragma unroll
        for (int r = 0; r < RPL; r++) {
            const int k = lane + 32 * r;
            l[r] = (k > i && k < n) ? (T)f_hi(A[i * lda + k]) : T(0);
        }
        const T ri = (T)f_hi(rs[i]);
#pragma unroll
        for (int c = 0; c < CPW; c++) {
            const T own = (RPL == 1 || i < 32) ? x[c][0] : x[c][RPL - 1];
            const T xi = __shfl_sync(0xffffffffu, own, i & 31) * ri;
#pragma unroll
            for (int r = 0; r < RPL; r++) x[c][r] = (lane + 32 * r == i) ? xi : fma(-l[r], xi, x[c][r]);
        }
    }
#pragma unroll
    for (int c = 0; c < CPW; c++) {
        const int col = warp + NW * c;
        if (col < n)
#pragma unroll
            for (int r = 0; r < RPL; r++)
                if (lane + 32 * r < n) out[(size_t)col * ldo + lane + 32 * r] = x[c][r];
    }
    __syncthreads();
}

// X = L^{-1} B for ncol right-hand sides, L the chol_small factor of order
// N <= 32 (L[k][i] = A[i][k]).  Element a of column col of B is read at
// src[col * cs + a * ls], element a of column col of X is written to
// X[a * ldx + col] (X may be B itself when B is stored that way).  Only the
// leading nrow <= N rows take part (rows beyond are left as garbage).  Warps
// own columns (col = warp + 8j, four at a time), lanes own rows; each lane
// keeps its row of L and its reciprocal pivot in registers, and at step i the
// owner of row i scales x_i and one shuffle broadcasts it.
// The columns of fwd_solve_warp by the warps w0 .. w0 + nw - 1 of the CTA
// (column col by warp w0 + col % nw); no barrier.
template <typename T, int N, typename F>
__device__ void fwd_solve_warps(const F *A, int lda, const F *rs, const T *src, int cs, int ls, T *X, int ldx,
                                int ncol, int nrow, int w0, int NW)
{
    static_assert(N <= 32, "one row per lane");
    constexpr int CB = 4;
    const int warp = (threadIdx.x >> 5) - w0, lane = threadIdx.x & 31;
    if (warp < 0 || warp >= NW) return;
    T Lr[N];
#pragma unroll
    for (int i = 0; i < N; i++) Lr[i] = (lane > i && lane < N) ? (T)f_hi(A[i * lda + lane]) : T(0);
    const T rl = lane < N ? (T)f_hi(rs[lane]) : T(0);
    for (int j0 = 0; warp + NW * j0 < ncol; j0 += CB) {
        T x[CB];
#pragma unroll
        for (int cc = 0; cc < CB; cc++) {
            const int col = warp + NW * (j0 + cc);
            x[cc] = (col < ncol && lane < N) ? src[(size_t)col * cs + (size_t)lane * ls] : T(0);
        }
#pragma unroll
        for (int i = 0; i < N; i++)
            if (i < nrow)
#pragma unroll
                for (int cc = 0; cc < CB; cc++) {
                    const T xi = __shfl_sync(0xffffffffu, x[cc] * rl, i);
                    x[cc] = lane == i ? xi : fma(-Lr[i], xi, x[cc]);
                }
#pragma unroll
        for (int cc = 0; cc < CB; cc++) {
            const int col = warp + NW * (j0 + cc);
            if (col < ncol && lane < N) X[(size_t)lane * ldx + col] = x[cc];
        }
    }
}
template <typename T, int N, typename F>
__device__ void fwd_solve_warp(const F *A, int lda, const F *rs, const T *src, int cs, int ls, T *X, int ldx,
                               int ncol, int nrow = N)
{
    fwd_solve_warps<T, N, F>(A, lda, rs, src, cs, ls, X, ldx, ncol, nrow, 0, NT / 32);
    __syncthreads();
}

// ---------------------------------------------- fixed-grid BF16 slices --
// Entries of the whitened basis at points and knots are bounded by sigma
// (sum_k |What^k(x)|^2 <= C(x, x) = sigma2), so one grid serves all of them:
// with 2^e > 2 sigma, v = q0 + ... + q4 with q_i = n_i 2^(e - 7 - 8 i),
// |n_i| <= 128 (exact BF16 values), exact for an FP32 v down to 2^(e - 40).
// Each q_i comes from rounding the remainder to its grid by adding and
// subtracting 1.5 2^(e + 16 - 8 i) (round to nearest even; the subtraction of
// q_i from the remainder is exact).  The tensor-core leaf basis sums the
// slices' products by order (mra_leafbasis_tc.cuh); the prior writes its
// regions' blocks in this form for it.
constexpr int kTcSlices = 5;
struct TcGrid {
    float mag[kTcSlices];
};
__device__ __forceinline__ TcGrid tc_grid(double sigma2)
{
    const float sg = sqrtf((float)sigma2);
    const int e = (int)((__float_as_uint(sg) >> 23) & 0xffu) - 127 + 2; // 2^e > 2 sigma
    TcGrid g;
#pragma unroll
    for (int i = 0; i < kTcSlices; i++) g.mag[i] = __fmul_rn(1.5f, __int_as_float((127 + e + 16 - 8 * i) << 23));
    return g;
}
// the slices of v as BF16 bit patterns (absolute units)
__device__ __forceinline__ void tc_slices(float v, const TcGrid &g, uint32_t (&q)[kTcSlices])
{
    float r = v;
#pragma unroll
    for (int i = 0; i < kTcSlices; i++) {
        const float qi = FSUB(FADD(r, g.mag[i]), g.mag[i]);
        r = FSUB(r, qi);
        q[i] = __float_as_uint(qi) >> 16; // <= 8 significant bits: the truncation is exact
    }
}
// Eight values of one operand row at K positions 8 g .. 8 g + 7, sliced, as
// one 16-byte core-matrix row in each of the five slice planes (plane stride
// `plane` bytes, offset `off` of the row in plane 0).
__device__ __forceinline__ void tc_put8(unsigned char *base, size_t plane, size_t off, const float (&v)[8],
                                        const TcGrid &g)
{
    uint32_t w[kTcSlices][4];
#pragma unroll
    for (int p = 0; p < 4; p++) {
        uint32_t a[kTcSlices], b[kTcSlices];
        tc_slices(v[2 * p], g, a);
        tc_slices(v[2 * p + 1], g, b);
#pragma unroll
        for (int i = 0; i < kTcSlices; i++) w[i][p] = a[i] | (b[i] << 16);
    }
#pragma unroll
    for (int i = 0; i < kTcSlices; i++)
        *reinterpret_cast<uint4 *>(base + (size_t)i * plane + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}
// Sliced operands are stored step-major for the MMAs' K = 16 steps: per step
// the five slice planes follow each other, and a plane holds the ROWS rows'
// two no-swizzle K-major core matrices (8 rows x 16 bytes): 8-row groups 256
// bytes apart (SBO), the step's two K groups 128 bytes apart (LBO).  One step
// of all slices is contiguous (one bulk copy).
template <int ROWS>
__host__ __device__ constexpr size_t tc_step_plane() { return (size_t)ROWS * 32; }
// byte offset of row r, K group g (values 8 g .. 8 g + 7), slice plane 0
template <int ROWS>
__host__ __device__ constexpr size_t tc_step_off(int r, int g)
{
    return (size_t)(g / 2) * kTcSlices * tc_step_plane<ROWS>() + (size_t)(r / 8) * 256u + (size_t)(g % 2) * 128u +
           (size_t)(r % 8) * 16u;
}
// bytes of one sliced RP x RP block (the prior's What^k of a region)
template <int RP>
__host__ __device__ constexpr size_t tc_block_bytes() { return (size_t)kTcSlices * RP * RP * 2; }

// Bytes of the per-column Cholesky's scratch (chol_small, the FP64 kernels);
// the mixed kernels' blocked Cholesky needs none.
template <typename T, int N>
__host__ __device__ constexpr size_t chol_scratch_bytes()
{
    return sizeof(T) == 8 ? (size_t)((tri_count(N) * 2 + 15) & ~15) : 0;
}

// ------------------------------------------------------------------ prior --
// Region i of level m (1 <= m <= M-1): What^1..What^{m-1} against its
// ancestors, then W^m = C(Q,Q) - sum_k What^k What^k', its Cholesky factor L,
// log|W^m| and Linv = L^{-1}.  The ancestors' blocks are staged level by
// level: in two buffers (the next level prefetched while this one is
// computed), or in one on deep trees where two do not fit.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_prior_bytes(int m, int stages = 2)
{
    return (size_t)RP * (RP + 1) * 8 + (RP + 2) * 8 + 8 * 8 + chol_scratch_bytes<T, RP>() + 64 +
           4 * RP * sizeof(T) + (size_t)((m - 1) + stages * (m > 1 ? m - 1 : 1) + 1) * RP * RP * sizeof(T) +
           RP * sizeof(T) + 64;
}

template <typename T, int RP>
__host__ __device__ constexpr int prior_stages(int m)
{
    return smem_prior_bytes<T, RP>(m, 2) <= kSmemMax ? 2 : 1;
}

// Deep levels (one stage of the ancestor's blocks does not fit beside the
// region's own): k_prior<T, RP, KB> stages them KB at a time.  Each output
// sums the same terms in the same order, so the two give the same blocks and
// factors bit for bit.
template <typename T, int RP, int KB>
__host__ __device__ constexpr size_t smem_prior_stream_bytes(int m)
{
    return (size_t)RP * (RP + 1) * 8 + (RP + 2) * 8 + 8 * 8 + chol_scratch_bytes<T, RP>() + 64 +
           4 * RP * sizeof(T) + (size_t)((m - 1) + KB + 1) * RP * RP * sizeof(T) + RP * sizeof(T) + 64;
}

// CTAs per SM the registers must allow: in FP32 five for the two-block
// kernel, which exists to fit five where shared memory allows them, six for
// the whole-staged one (40 registers; small-RP trees fit six), one for the
// deep levels' four-block kernel (its shared memory holds one); FP64 four.
// (A kernel declared without a CTA count gets a register budget of the
// compiler's choosing, which a count of one does not reproduce.)
template <typename T, int KB>
constexpr int prior_min_ctas()
{
    return sizeof(T) != 4 ? 4 : (KB == 2 ? 5 : (KB == 0 ? 6 : 1));
}

template <typename T, int RP, int KB = 0>
__global__ void __launch_bounds__(NT, (prior_min_ctas<T, KB>())) k_prior(DevTree t, Work<T> w, int m, int stages)
{
    using TL = Tile<RP, RP>;
    using F = typename FacT<T>::type;
    const int i = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    // sigma2 and 1/beta once per CTA, read after the first barrier
    __shared__ double s_ib;
    __shared__ ff s_par[2]; // sigma2 and 1/beta as float pairs
    const float s_cq = grid_constant(th[0]);
    set_cov_params<T>(th, &s_ib, s_par);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sL = (F *)smem_raw;                  // RP x (RP+1)
    F *srs = sL + RP * (RP + 1);            // RP + 2
    double *red = (double *)(srs + RP + 2); // 8
    F *sr2 = (F *)(red + 8);                // RP + 1 (squared reciprocal pivots; FP64 only)
    int *flag = (int *)((unsigned char *)sr2 + chol_scratch_bytes<T, RP>());
    T *sq = (T *)(flag + 16);               // own knots relative to the current origin: 2 RP
    T *sa = sq + 2 * RP;                    // ancestor knots: 2 RP
    T *sU = sa + 2 * RP;                    // (m-1) blocks k-major [t][row]
    T *sB0 = sU + (size_t)(m - 1) * RP * RP; // `stages` stages of up to m-1 ancestor blocks (column-major)
    // RP x RP k-major (KB > 0: after KB staged blocks)
    T *sW = sB0 + (KB > 0 ? (size_t)KB * RP * RP : (size_t)stages * (m > 1 ? m - 1 : 1) * RP * RP);

    const int Rm = t.Rl[m]; // own knots
    const int64_t g = t.lvl_off[m] + i;
    if (tid == 0) flag[0] = 0;
    T *pb = w.prior + (size_t)b * w.prior_stride;
    const int r0 = TL::r0(), c0 = TL::c0();
    // two stages: the level-l ancestor's blocks go to stage l & 1 and level
    // l + 1 is fetched with cp.async while level l is computed; one stage:
    // each level is fetched after the previous one's last read (the barrier
    // that ends every level)
    const size_t stage = (size_t)(m > 1 ? m - 1 : 1) * RP * RP;
    auto slot = [&](int l) { return sB0 + (size_t)(stages == 2 ? (l & 1) : 0) * stage; };
    auto fetch = [&](int l) {
        const int64_t ia = anc_index(t, i, m, l);
        copy_g2s_async(slot(l), pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP, l * RP * RP);
        cp_async_commit();
    };
    if (KB == 0 && m > 1 && stages == 2) fetch(1);
    for (int l = 1; l < m; l++) {
      if constexpr (KB > 0) {
        // the ancestor's blocks KB at a time through sB0: What^1..What^{l-1}
        // against the region's own, then its Linv
        const int64_t ia = anc_index(t, i, m, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int Ra = t.Rl[l];
        const T *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        if (tid < RP) {
            const double ox = t.cx[ga], oy = t.cy[ga];
            sq[tid] = (T)(t.kx[g * RP + tid] - ox);
            sq[RP + tid] = (T)(t.ky[g * RP + tid] - oy);
            sa[tid] = (T)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (T)(t.ky[ga * RP + tid] - oy);
        }
        T acc[TL::RT][TL::CT];
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (w.exact_rem) {
                grid_acc ga4[TL::RT][TL::CT];
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) grid_init(ga4[r][c], s_cq);
                for (int k0 = 0; k0 < l - 1; k0 += KB) {
                    const int nb = min(KB, l - 1 - k0);
                    copy_g2s_async(sB0, anc + (size_t)k0 * RP * RP, nb * RP * RP);
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncthreads();
                    tile_grid_add<RP, RP>(ga4, sU + (size_t)k0 * RP * RP, RP, sB0, RP, nb * RP);
                    __syncthreads();
                }
                __syncthreads(); // sq and sa before the covariance
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) {
                        const int a = r0 + r, j = c0 + c;
                        ff cv = ff{0.f, 0.f};
                        if (a < Rm && j < Ra) cv = ff_cov_exp(s_par[0], s_par[1], sq[a], sq[RP + a], sa[j], sa[RP + j]);
                        const ff fa = grid_value(ga4[r][c], s_cq);
                        sW[(c0 + c) * RP + r0 + r] = FADD(FSUB(cv.hi, fa.hi), FSUB(cv.lo, fa.lo));
                    }
                done = true;
            }
        }
        if (!done) {
            tile_zero(acc);
            for (int k0 = 0; k0 < l - 1; k0 += KB) {
                const int nb = min(KB, l - 1 - k0);
                copy_g2s_async(sB0, anc + (size_t)k0 * RP * RP, nb * RP * RP);
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
                tile_fma<T, RP, RP>(acc, sU + (size_t)k0 * RP * RP, RP, sB0, RP, nb * RP);
                __syncthreads();
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) {
                    const int a = r0 + r, j = c0 + c;
                    const T cv = (a < Rm && j < Ra) ? cov_d(CovP<T>(th[0], s_ib), sq[a] - sa[j], sq[RP + a] - sa[RP + j]) : T(0);
                    sW[j * RP + a] = cv - acc[r][c];
                }
        }
        // What^l = W Linv' with the ancestor's Linv (its last block)
        __syncthreads();
        copy_g2s_async(sB0, anc + (size_t)(l - 1) * RP * RP, RP * RP);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        tile_zero(acc);
        tile_fma<T, RP, RP>(acc, sW, RP, sB0, RP, RP);
        T *outl = sU + (size_t)(l - 1) * RP * RP;
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) outl[(c0 + c) * RP + r0 + r] = acc[r][c];
        __syncthreads();
      } else {
        const int64_t ia = anc_index(t, i, m, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int Ra = t.Rl[l]; // the ancestor's knots
        T *sB = slot(l);
        if (stages != 2) {
            fetch(l);
            cp_async_wait<0>();
        } else if (l + 1 < m) {
            fetch(l + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        if (tid < RP) {
            const double ox = t.cx[ga], oy = t.cy[ga];
            sq[tid] = (T)(t.kx[g * RP + tid] - ox);
            sq[RP + tid] = (T)(t.ky[g * RP + tid] - oy);
            sa[tid] = (T)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (T)(t.ky[ga * RP + tid] - oy);
        }
        __syncthreads();
        T acc[TL::RT][TL::CT];
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (w.exact_rem) {
                remainder_ff<RP, RP>(acc, sU, RP, sB, (l - 1) * RP, sq, RP, Rm, sa, Ra, s_par[0], s_par[1], s_cq);
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) sW[(c0 + c) * RP + r0 + r] = acc[r][c];
                done = true;
            }
        }
        if (!done) {
            tile_zero(acc);
            tile_fma<T, RP, RP>(acc, sU, RP, sB, RP, (l - 1) * RP);
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) {
                    const int a = r0 + r, j = c0 + c;
                    const T cv = (a < Rm && j < Ra) ? cov_d(CovP<T>(th[0], s_ib), sq[a] - sa[j], sq[RP + a] - sa[RP + j]) : T(0);
                    sW[j * RP + a] = cv - acc[r][c];
                }
        }
        __syncthreads();
        tile_zero(acc);
        tile_fma<T, RP, RP>(acc, sW, RP, sB + (size_t)(l - 1) * RP * RP, RP, RP);
        T *out = sU + (size_t)(l - 1) * RP * RP;
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) out[(c0 + c) * RP + r0 + r] = acc[r][c];
        __syncthreads();
      }
    }
    // self block W^m = C(Q,Q) - sum_k What^k What^k' (identity on the padding)
    if (tid < RP) {
        const double ox = t.cx[g], oy = t.cy[g];
        sq[tid] = (T)(t.kx[g * RP + tid] - ox);
        sq[RP + tid] = (T)(t.ky[g * RP + tid] - oy);
    }
    __syncthreads();
    bool self_done = false;
    if constexpr (sizeof(T) == 4) {
        if (w.exact_rem) {
            // W^m in float pairs straight into the factorization
            FF fa[TL::RT][TL::CT];
            tile_fma_ff<RP, RP>(fa, sU, RP, sU, RP, (m - 1) * RP, s_cq);
            const ff s2f = s_par[0], ibf = s_par[1];
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) {
                    const int a = r0 + r, j = c0 + c;
                    F v;
                    if (a < Rm && j < Rm)
                        v = ff_sub_sloppy(ff_cov_exp(s2f, ibf, sq[a], sq[RP + a], sq[j], sq[RP + j]),
                                   ff{fa[r][c].hi, fa[r][c].lo});
                    else
                        v = f_of<F>(a == j ? 1.0 : 0.0);
                    sL[a * (RP + 1) + j] = v;
                }
            self_done = true;
        }
    }
    if (!self_done) {
        T acc[TL::RT][TL::CT];
        tile_zero(acc);
        tile_fma<T, RP, RP>(acc, sU, RP, sU, RP, (m - 1) * RP);
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) {
                const int a = r0 + r, j = c0 + c;
                F v;
                if (a < Rm && j < Rm)
                    v = f_of_T(cov_d(CovP<T>(th[0], s_ib), sq[a] - sq[j], sq[RP + a] - sq[RP + j]) - acc[r][c]);
                else
                    v = f_of<F>(a == j ? 1.0 : 0.0);
                sL[a * (RP + 1) + j] = v;
            }
    }
    __syncthreads();
    // W^m assembled in FP32 cannot resolve pivots below its own rounding: the
    // mixed mode calls such a factor singular at 1e-6 of the largest diagonal.
    if constexpr (sizeof(T) == 4)
        chol_blocked<RP>(sL, RP + 1, RP, srs, flag, 1e-6, red);
    else
        chol_small<F, (tri_count(RP) + NT - 1) / NT>(sL, RP + 1, RP, srs, sr2, flag, MRA_SINGULAR);
    const double ld = logdet_small(sL, RP + 1, RP, red);
    T *out = pb + w.prior_lvl[m] + (size_t)i * m * RP * RP;
    for (int e = tid; e < (m - 1) * RP * RP; e += NT) out[e] = sU[e];
    if constexpr (sizeof(T) == 4) {
        if (w.lbB && m >= 2) {
            // What^1..What^{m-1} of the region as fixed-grid BF16 slices for the
            // tensor-core leaf basis: operand rows = the region's knots j, K = the
            // basis index t (element (j, t) of block k at sU[k RP^2 + t RP + j])
            const TcGrid gr = tc_grid(th[0]);
            constexpr size_t BB = tc_block_bytes<RP>();
            unsigned char *dst = w.lbB + (size_t)b * w.lbB_stride + w.lbB_lvl[m] + (size_t)i * (m - 1) * BB;
            for (int it = tid; it < (m - 1) * RP * (RP / 8); it += NT) {
                const int k = it / (RP * (RP / 8)), rem = it % (RP * (RP / 8)), j = rem / (RP / 8), gg = rem % (RP / 8);
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = sU[(size_t)k * RP * RP + (size_t)(8 * gg + q) * RP + j];
                tc_put8(dst + (size_t)k * BB, tc_step_plane<RP>(), tc_step_off<RP>(j, gg), v, gr);
            }
        }
    }
    // Linv stored column-major: element (a, j) at j*RP + a
    trinv_warp<T, RP>(sL, RP + 1, srs, out + (size_t)(m - 1) * RP * RP, RP, RP);
    if (tid == 0) {
        if (flag[0]) w.status[b] = ST_ENOTPD;
        if (w.reg_lw) w.reg_lw[(size_t)b * w.reglw_stride + g] = ld;
    }
}

// -------------------------------------------------------------- leaf basis --
// A chunk of observation rows below one level-(M-1) region: What^l of each
// row against its M-1 ancestors, written as rows of U.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_leafbasis_bytes(int M, int stages, int CH = chunk_rows<T>())
{
    return (size_t)(2 * CH + 2 * RP) * sizeof(T) + (size_t)(M - 1) * RP * (CH + 2) * sizeof(T) +
           (size_t)stages * (M - 1) * RP * RP * sizeof(T) + (size_t)RP * (CH + 2) * sizeof(T) + 64;
}

// Two stages of ancestor blocks (prefetch of the next level) only while two
// CTAs still fit on an SM; deep trees keep one stage and the occupancy.
template <typename T, int RP>
__host__ __device__ constexpr int leafbasis_stages(int M, int CH = chunk_rows<T>())
{
    return smem_leafbasis_bytes<T, RP>(M, 2, CH) <= (size_t)110 * 1024 ? 2 : 1;
}

template <typename T, int RP, int CH>
__global__ void __launch_bounds__(NT) k_leafbasis(DevTree t, Work<T> w, const Chunk *chunks, int stages)
{
    constexpr int LDC = CH + 2; // k-major row stride (keeps the transposed write-out conflict-light)
    using TL = Tile<CH, RP>;
    const Chunk ch = chunks[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    // sigma2 and 1/beta once per CTA, read after the first barrier
    __shared__ double s_ib;
    __shared__ ff s_par[2]; // sigma2 and 1/beta as float pairs
    const float s_cq = grid_constant(th[0]);
    set_cov_params<T>(th, &s_ib, s_par);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = t.M, P = ch.parent, nr = ch.n;
    T *sp = (T *)smem_raw;                  // 2 CH rows relative to the ancestor corner
    T *sa = sp + 2 * CH;                    // 2 RP
    T *sU = sa + 2 * RP;                     // (M-1) blocks k-major [t][row], stride LDC
    T *sB0 = sU + (size_t)(M - 1) * RP * LDC;          // 1 or 2 stages of up to M-1 ancestor blocks
    T *sW = sB0 + (size_t)stages * (M - 1) * RP * RP; // RP x LDC k-major
    const T *pb = w.prior + (size_t)b * w.prior_stride;
    const int r0 = TL::r0(), c0 = TL::c0();
    // the ancestor's blocks of level l go to stage l & 1 (two stages: level
    // l + 1 is fetched with cp.async while level l is computed)
    auto fetch = [&](int l) {
        const int64_t ia = anc_index(t, P, M - 1, l);
        copy_g2s_async(sB0 + (size_t)((l & 1) * (stages - 1)) * (M - 1) * RP * RP,
                       pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP, l * RP * RP);
        cp_async_commit();
    };
    fetch(1);
    for (int l = 1; l <= M - 1; l++) {
        const int64_t ia = anc_index(t, P, M - 1, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int R = t.Rl[l]; // the ancestor's knots
        T *sB = sB0 + (size_t)((l & 1) * (stages - 1)) * (M - 1) * RP * RP;
        if (stages == 2) {
            if (l + 1 <= M - 1) {
                fetch(l + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        } else {
            if (l > 1) fetch(l); // the single stage is free after the previous level's barrier
            cp_async_wait<0>();
        }
        const double ox = t.cx[ga], oy = t.cy[ga];
        if (tid < CH) {
            sp[tid] = tid < nr ? (T)(t.sx[ch.row0 + tid] - ox) : T(0);
            sp[CH + tid] = tid < nr ? (T)(t.sy[ch.row0 + tid] - oy) : T(0);
        }
        if (tid < RP) {
            sa[tid] = (T)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (T)(t.ky[ga * RP + tid] - oy);
        }
        __syncthreads();
        T acc[TL::RT][TL::CT];
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (w.exact_rem) {
                remainder_ff<CH, RP>(acc, sU, LDC, sB, (l - 1) * RP, sp, CH, nr, sa, R, s_par[0], s_par[1], s_cq);
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) sW[(c0 + c) * LDC + r0 + r] = acc[r][c];
                done = true;
            }
        }
        if (!done) {
            tile_zero(acc);
            tile_fma<T, CH, RP>(acc, sU, LDC, sB, RP, (l - 1) * RP);
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) {
                    const int a = r0 + r, j = c0 + c;
                    const T cv = (a < nr && j < R) ? cov_d(CovP<T>(th[0], s_ib), sp[a] - sa[j], sp[CH + a] - sa[RP + j]) : T(0);
                    sW[j * LDC + a] = cv - acc[r][c];
                }
        }
        __syncthreads();
        tile_zero(acc);
        tile_fma<T, CH, RP>(acc, sW, LDC, sB + (size_t)(l - 1) * RP * RP, RP, RP);
        T *out = sU + (size_t)(l - 1) * RP * LDC;
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) out[(c0 + c) * LDC + r0 + r] = acc[r][c];
        __syncthreads();
    }
    const int UC = (M - 1) * RP;
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)ch.row0 * UC;
    for (int e = tid; e < nr * UC; e += NT) {
        const int a = e / UC, col = e % UC;
        Ub[e] = sU[(size_t)col * LDC + a];
    }
}

// The leaf basis for deep trees: the same rows-by-level recursion as
// k_leafbasis, with the level's ancestor blocks staged KB at a time instead of
// all at once, so that 16-row chunks of deep trees fit several CTAs per SM
// (27 device levels at RP = 32: one CTA per SM with 32 rows and all blocks,
// three with 16 rows and two blocks).  Every output is formed by the same
// terms in the same order as in k_leafbasis, so the two give the same U bit
// for bit.
template <typename T, int RP, int CH, int KB>
__host__ __device__ constexpr size_t smem_leafbasis_stream_bytes(int M)
{
    return (size_t)(2 * CH + 2 * RP) * sizeof(T) + (size_t)(M - 1) * RP * (CH + 2) * sizeof(T) +
           (size_t)KB * RP * RP * sizeof(T) + (size_t)RP * (CH + 2) * sizeof(T) + 64;
}

template <typename T, int RP, int CH, int KB>
__global__ void __launch_bounds__(NT) k_leafbasis_stream(DevTree t, Work<T> w, const Chunk *chunks)
{
    constexpr int LDC = CH + 2;
    using TL = Tile<CH, RP>;
    const Chunk ch = chunks[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    __shared__ double s_ib;
    __shared__ ff s_par[2]; // sigma2 and 1/beta as float pairs
    const float s_cq = grid_constant(th[0]);
    set_cov_params<T>(th, &s_ib, s_par);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = t.M, P = ch.parent, nr = ch.n;
    T *sp = (T *)smem_raw;                    // 2 CH rows relative to the ancestor corner
    T *sa = sp + 2 * CH;                      // 2 RP
    T *sU = sa + 2 * RP;                      // (M-1) blocks k-major [t][row], stride LDC
    T *sB = sU + (size_t)(M - 1) * RP * LDC;  // KB ancestor blocks
    T *sW = sB + (size_t)KB * RP * RP;        // RP x LDC k-major
    const T *pb = w.prior + (size_t)b * w.prior_stride;
    const int r0 = TL::r0(), c0 = TL::c0();
    for (int l = 1; l <= M - 1; l++) {
        const int64_t ia = anc_index(t, P, M - 1, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int R = t.Rl[l]; // the ancestor's knots
        const T *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        const double ox = t.cx[ga], oy = t.cy[ga];
        if (tid < CH) {
            sp[tid] = tid < nr ? (T)(t.sx[ch.row0 + tid] - ox) : T(0);
            sp[CH + tid] = tid < nr ? (T)(t.sy[ch.row0 + tid] - oy) : T(0);
        }
        if (tid < RP) {
            sa[tid] = (T)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (T)(t.ky[ga * RP + tid] - oy);
        }
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (w.exact_rem) {
                grid_acc g[TL::RT][TL::CT];
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) grid_init(g[r][c], s_cq);
                for (int k0 = 0; k0 < l - 1; k0 += KB) {
                    const int nb = min(KB, l - 1 - k0);
                    copy_g2s_async(sB, anc + (size_t)k0 * RP * RP, nb * RP * RP);
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncthreads();
                    tile_grid_add<CH, RP>(g, sU + (size_t)k0 * RP * LDC, LDC, sB, RP, nb * RP);
                    __syncthreads();
                }
                __syncthreads(); // sp and sa (written above) before the covariance
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) {
                        const int a = r0 + r, j = c0 + c;
                        ff cv = ff{0.f, 0.f};
                        if (a < nr && j < R) cv = ff_cov_exp(s_par[0], s_par[1], sp[a], sp[CH + a], sa[j], sa[RP + j]);
                        const ff fa = grid_value(g[r][c], s_cq);
                        sW[(c0 + c) * LDC + r0 + r] = FADD(FSUB(cv.hi, fa.hi), FSUB(cv.lo, fa.lo));
                    }
                done = true;
            }
        }
        if (!done) {
            T acc[TL::RT][TL::CT];
            tile_zero(acc);
            for (int k0 = 0; k0 < l - 1; k0 += KB) {
                const int nb = min(KB, l - 1 - k0);
                copy_g2s_async(sB, anc + (size_t)k0 * RP * RP, nb * RP * RP);
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
                tile_fma<T, CH, RP>(acc, sU + (size_t)k0 * RP * LDC, LDC, sB, RP, nb * RP);
                __syncthreads();
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) {
                    const int a = r0 + r, j = c0 + c;
                    const T cv = (a < nr && j < R) ? cov_d(CovP<T>(th[0], s_ib), sp[a] - sa[j], sp[CH + a] - sa[RP + j]) : T(0);
                    sW[j * LDC + a] = cv - acc[r][c];
                }
        }
        // What^l = W Linv' with the ancestor's Linv (its last block)
        copy_g2s_async(sB, anc + (size_t)(l - 1) * RP * RP, RP * RP);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        {
            T acc[TL::RT][TL::CT];
            tile_zero(acc);
            tile_fma<T, CH, RP>(acc, sW, LDC, sB, RP, RP);
            T *out = sU + (size_t)(l - 1) * RP * LDC;
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
#pragma unroll
                for (int c = 0; c < TL::CT; c++) out[(c0 + c) * LDC + r0 + r] = acc[r][c];
        }
        __syncthreads();
    }
    const int UC = (M - 1) * RP;
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)ch.row0 * UC;
    for (int e = tid; e < nr * UC; e += NT) {
        const int a = e / UC, col = e % UC;
        Ub[e] = sU[(size_t)col * LDC + a];
    }
}

// ---------------------------------------------------------- leaf posterior --
// Leaf c with n <= nmax observations, all in shared memory:
// V = C(S,S) + tau2 I - U U' (exact products), V = L L' (FP64),
// Y = L^{-1} U (in place, type T), y = L^{-1} z (FP64), d = log|V|, u = y'y,
// w_c = Y'y.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_leafpost_bytes(int M, int nmax)
{
    return (size_t)nmax * (nmax + 1) * 8 + (size_t)(2 * nmax + 2) * 8 + 8 * 8 +
           (size_t)((tri_count(nmax) * 2 + 15) & ~15) + 64 + (size_t)nmax * ((M - 1) * RP + 4) * sizeof(T) +
           (size_t)nmax * nmax * sizeof(T) + 2 * (size_t)nmax * 8 + 80;
}

// w[col] = sum_a Y[a][col] y[a] for UC columns, in FP64.  Mixed mode: y is a
// float pair; the products with its leading part are exact and summed as a
// float pair, those with its trailing part are summed in FP32, so w carries
// the precision of y (the upward pass cancels sum y'y against quadratic
// forms in w, which must agree to more than FP32).
template <typename T, typename F>
__device__ void gram_vec(const T *Y, int ldy, int UC, const F *y, int n, double *wout)
{
    for (int col = threadIdx.x; col < UC; col += NT) {
        if constexpr (sizeof(T) == 4) {
            FF s{0.f, 0.f};
            float sl = 0.f;
            for (int a = 0; a < n; a++) {
                const float v = Y[(size_t)a * ldy + col];
                const ff ya = f_of_ff(y[a]);
                ff_add_prod(s, v, ya.hi);
                sl = __fmaf_rn(v, ya.lo, sl);
            }
            wout[col] = (double)s.hi + ((double)s.lo + (double)sl);
        } else {
            double s = 0.0;
            for (int a = 0; a < n; a++) s = fma(Y[(size_t)a * ldy + col], (double)f_hi(y[a]), s);
            wout[col] = s;
        }
    }
}

// The posterior terms of leaf c at theta b by the whole CTA (the body of the
// shared-memory leaf kernels below); theta b is valid.  Ends with every thread
// past its last shared-memory access of the leaf.
template <typename T, int RP, int NMAX>
__device__ __forceinline__ void leafpost_small_leaf(const DevTree &t, const Work<T> &w, int64_t c, int b)
{
    constexpr int nmax = NMAX;
    using F = typename FacT<T>::type;
    const int tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    const double tau2 = th[2];
    __shared__ double s_ib; // 1/beta, one FP64 division per CTA
    const int M = t.M;
    const int64_t o0 = t.leaf_off[c];
    const int n = (int)(t.leaf_off[c + 1] - o0);
    const int UC = (M - 1) * RP, LDU = UC + 4, LDV = nmax + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sV = (F *)smem_raw;                      // nmax x (nmax+1): V, then its factor
    F *sy = sV + (size_t)nmax * LDV;            // nmax: z, then y = L^{-1} z, then V^{-1} z
    F *srs = sy + nmax;                         // nmax + 2
    double *red = (double *)(srs + nmax + 2);   // 8
    F *sr2 = (F *)(red + 8);                    // nmax + 1
    int *flag = (int *)((unsigned char *)sr2 + ((tri_count(nmax) * 2 + 15) & ~15));
    T *sU = (T *)(flag + 16);                   // nmax x LDU (rows 16-byte aligned)
    T *sLi = sU + (size_t)nmax * LDU;           // nmax x nmax: L^{-1}, column-major
    double *sp = (double *)(((uintptr_t)(sLi + (size_t)nmax * nmax) + 15) & ~(uintptr_t)15); // 2 nmax coordinates
    ff *spf = (ff *)sp;
    __shared__ ff s_par[2]; // sigma2 and 1/beta as float pairs
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)o0 * UC;
    // U rows -> shared (asynchronous 16-byte copies)
    {
        const int cpr = UC * (int)sizeof(T) / 16;
        for (int e = tid; e < n * cpr; e += NT) {
            const int a = e / cpr, q = e % cpr;
            cp_async16((char *)(sU + (size_t)a * LDU) + 16 * q, (const char *)(Ub + (size_t)a * UC) + 16 * q);
        }
        cp_async_commit();
    }
    // coordinates relative to the parent region's corner (level M-1)
    const int64_t gp = M > 1 ? t.lvl_off[M - 1] + anc_index(t, c, M, M - 1) : -1;
    const double ox = gp >= 0 ? t.cx[gp] : t.sx[o0], oy = gp >= 0 ? t.cy[gp] : t.sy[o0];
    for (int a = tid; a < n; a += NT) {
        if constexpr (sizeof(T) == 4) {
            spf[a] = ff_from_double(t.sx[o0 + a] - ox);
            spf[nmax + a] = ff_from_double(t.sy[o0 + a] - oy);
        } else {
            sp[a] = t.sx[o0 + a] - ox;
            sp[nmax + a] = t.sy[o0 + a] - oy;
        }
        sy[a] = f_of<F>(t.sz[o0 + a]);
    }
    for (int e = tid; e < nmax * nmax; e += NT) sLi[e] = T(0);
    if (tid == 0) flag[0] = 0;
    set_cov_params<T>(th, &s_ib, s_par);
    __shared__ ff s_tau2;
    if (tid == 2) s_tau2 = ff_from_double(tau2);
    cp_async_wait<0>();
    __syncthreads();
    const ff tau2f = s_tau2;
    // V = C(S,S) + tau2 I - U U' (lower triangle), in 2x2 blocks (A, Q), Q <= A
    {
        const int nb = (n + 1) >> 1;
        for (int e = tid; e < tri_count(nb); e += NT) {
            int A = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (tri_count(A + 1) <= e) A++;
            while (A > 0 && tri_count(A) > e) A--;
            const int Q = e - tri_count(A);
            const int a0 = 2 * A, q0 = 2 * Q;
            T hi[2][2], lo[2][2];
            dot2x2(sU + a0 * LDU, sU + min(a0 + 1, n - 1) * LDU, sU + q0 * LDU, sU + min(q0 + 1, n - 1) * LDU, UC,
                   hi, lo);
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const int a = a0 + i, q = q0 + j;
                    if (a >= n || q > a) continue;
                    if constexpr (sizeof(T) == 4) {
                        const ff cv = ff_cov_exp(s_par[0], s_par[1], spf[a], spf[nmax + a], spf[q], spf[nmax + q]);
                        ff v = ff_sub_sloppy(cv, ff{(float)hi[i][j], (float)lo[i][j]});
                        if (a == q) v = ff_add_sloppy(v, tau2f);
                        sV[a * LDV + q] = v;
                    } else {
                        const double cv = cov64(th[0], s_ib, sp[a] - sp[q], sp[nmax + a] - sp[nmax + q]);
                        sV[a * LDV + q] = cancel_sub(cv, hi[i][j], lo[i][j]) + (a == q ? tau2 : 0.0);
                    }
                }
        }
    }
    __syncthreads();
    // the per-column factor: with several leaves per SM the kernel is bound by
    // issue, not by one factor's latency, and the blocked factor's
    // register-resident panel costs more instructions and registers here (it
    // stays in the prior and the upward pass, whose top levels are latency
    // chains of one CTA)
    chol_small<F, (tri_count(NMAX) + NT - 1) / NT>(sV, LDV, n, srs, sr2, flag, MRA_SINGULAR);
    const double dv = logdet_small(sV, LDV, n, red);
    trinv_warp<T, NMAX>(sV, LDV, srs, sLi, nmax, n);
    // Y = L^{-1} U, block column by block column, straight to global; row r
    // of L^{-1} ends at column r, so a thread's rows r0 .. r0 + RT - 1 stop
    // the sum there (the terms skipped are exact zeros)
    {
        using TL = Tile<NMAX, RP>;
        const int r0 = TL::r0(), c0 = TL::c0();
        const int kend = min(n, r0 + TL::RT);
        for (int cb = 0; cb < UC; cb += RP) {
            T acc[TL::RT][TL::CT];
            tile_zero(acc);
            tile_fma<T, NMAX, RP>(acc, sLi, nmax, sU + cb, LDU, kend);
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
                if (r0 + r < n)
#pragma unroll
                    for (int cc = 0; cc < TL::CT; cc++) Ub[(size_t)(r0 + r) * UC + cb + c0 + cc] = acc[r][cc];
        }
    }
    // y = Linv z, u = y'y and w = Y'y = U' (Linv' y) with the same FP32 Linv
    // that forms Y = Linv U (exact products, float-pair sums): the leaf's u, w
    // and Gram blocks then all belong to one operator, so the upward pass
    // cancels them consistently
    F *sy2 = sr2; // the Cholesky's scratch is free now
    for (int r = tid; r < n; r += NT) {
        DotTF<T, F> acc;
        for (int k = 0; k <= r; k++) acc.add(sLi[k * nmax + r], sy[k]);
        sy2[r] = acc.value();
    }
    __syncthreads();
    if (tid < 32) {
        F q = f_of<F>(0.0);
        for (int a = tid; a < n; a += 32) q = f_add(q, f_sqr(sy2[a]));
        q = warp_sum_f(q);
        if (tid == 0) red[0] = f_dbl(q);
    }
    for (int k = tid; k < n; k += NT) {
        DotTF<T, F> acc;
        for (int r = k; r < n; r++) acc.add(sLi[k * nmax + r], sy2[r]);
        sy[k] = acc.value();
    }
    if (w.keep_li && b == 0) {
        // L^{-1} and y for prediction
        T *kl = w.keep_li + (size_t)c * kKeepLd * kKeepLd;
        for (int e = tid; e < n * n; e += NT) {
            const int k = e / n, r = e % n;
            kl[k * kKeepLd + r] = sLi[k * nmax + r];
        }
        for (int a = tid; a < n; a += NT) w.keep_y[(size_t)c * kKeepLd + a] = f_dbl(sy2[a]);
    }
    __syncthreads();
    const double uv = red[0];
    gram_vec(sU, LDU, UC, sy, n, w.leaf_w + (size_t)b * w.leafw_stride + (size_t)c * UC);
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

// CTAs per SM the register budget must allow in the mixed modes: as many as
// the bucket's shared memory fits on trees of M = 7 at RP = 32 (five, four
// and three for caps 32, 40 and 48).  Left to itself the compiler spends up to
// 110 registers a thread, which holds every bucket to two CTAs per SM.
template <typename T, int RP, int NMAX>
constexpr int leafpost_min_ctas()
{
    // FP64 (shared memory fits at most three): the register counts of the
    // kernels without a budget; the 64 cap runs one CTA per SM
    if (sizeof(T) != 4) return NMAX <= 48 ? 3 : 1;
    return NMAX <= 32 ? 5 : (NMAX <= 40 ? 4 : 3);
}

// One CTA per leaf of the list (grid.x), theta grid.y.
template <typename T, int RP, int NMAX>
__global__ void __launch_bounds__(NT, (leafpost_min_ctas<T, RP, NMAX>())) k_leafpost_small(DevTree t, Work<T> w,
                                                                                           const int64_t *leaves)
{
    const int b = blockIdx.y;
    if (!theta_ok(w.theta + 3 * b)) return;
    leafpost_small_leaf<T, RP, NMAX>(t, w, leaves[blockIdx.x], b);
}

// The same leaves as a work queue: a persistent grid (CTAs resident at once)
// takes the leaves of the list in order through an atomic counter per theta
// (counter[b], zero at launch), the list being ordered by decreasing size --
// the paper's dynamic scheduling by the cost of a leaf (Sec. 4.1) as greedy
// longest-first list scheduling on the GPU.  No CTA waits for another; each
// leaf is computed by the same code as above, so the results are the same bit
// for bit.
template <typename T, int RP, int NMAX>
__global__ void __launch_bounds__(NT, (leafpost_min_ctas<T, RP, NMAX>())) k_leafpost_queue(DevTree t, Work<T> w, const int64_t *leaves, int nleaves,
                                                       unsigned *counter)
{
    const int b = blockIdx.y;
    if (!theta_ok(w.theta + 3 * b)) return;
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(&counter[b], 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads(); // every thread has read s_idx (and left the last leaf's shared memory)
        if (idx >= nleaves) break;
        leafpost_small_leaf<T, RP, NMAX>(t, w, leaves[idx], b);
    }
}

// Leaves larger than the shared-memory path: the same steps on global memory.
// Cholesky with L in the LOWER triangle and rs[j] = 1/L_jj.
template <typename F>
static __device__ void chol_global(F *A, int lda, int n, F *rs, int *fail, double *sc, F *sr)
{
    if (threadIdx.x < 32) {
        double m = 0.0;
        for (int j = threadIdx.x; j < n; j += 32) m = fmax(m, (double)f_hi(A[(size_t)j * lda + j]));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) sc[0] = MRA_SINGULAR * m;
    }
    __syncthreads();
    const double tol = sc[0];
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            F d = A[(size_t)j * lda + j];
            if (!((double)f_hi(d) > tol)) {
                *fail = 1;
                d = f_of<F>(1.0);
            }
            const F r = f_rsqrt(d);
            A[(size_t)j * lda + j] = f_mul(d, r);
            rs[j] = r;
            *sr = r;
        }
        __syncthreads();
        const F r = *sr;
        for (int i = j + 1 + threadIdx.x; i < n; i += NT) A[(size_t)i * lda + j] = f_mul(A[(size_t)i * lda + j], r);
        __syncthreads();
        const int wd = n - j - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)wd * wd; e += NT) {
            const int i = j + 1 + (int)(e / wd), k = j + 1 + (int)(e % wd);
            if (k <= i)
                A[(size_t)i * lda + k] =
                    f_sub(A[(size_t)i * lda + k], f_mul(A[(size_t)i * lda + j], A[(size_t)k * lda + j]));
        }
        __syncthreads();
    }
}

// y <- L^{-1} y for a large factor in the lower triangle, by warp 0: lane a
// owns the rows a = lane (mod 32).
template <typename F>
static __device__ void fwd_solve_vec_big(const F *A, int lda, const F *rs, int n, F *y)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int q = 0; q < n; q++) {
            F yq = y[q];
            if ((q & 31) == lane) {
                yq = f_mul(yq, rs[q]);
                y[q] = yq;
            }
            yq = f_shfl(yq, q & 31);
            for (int a = q + 1 + ((lane - q - 1) & 31); a < n; a += 32)
                y[a] = f_sub(y[a], f_mul(A[(size_t)a * lda + q], yq));
            __syncwarp();
        }
    }
    __syncthreads();
}

// --------------------------------------------------------------- leaf Gram --
// Region P of level M-1: A = Y'Y over the rows below P, as 64 x 64 output
// tiles of the D x D matrix (D = (M-1) RP, blockIdx.y = upper-triangle tile);
// every 32 x 32 sub-block (k <= l) is written to the packed layout.  Rows are
// staged in chunks of 32 (double-buffered with cp.async), accumulated in T
// within a chunk and as an unevaluated pair across chunks in the mixed mode.
// Tile (0, 0) also sums the leaves' w and (d, u).
constexpr int kGramTile = 64, kGramRows = 32;

template <typename T, int RP>
__host__ __device__ constexpr size_t smem_leafgram_bytes(int M)
{
    return (size_t)2 * 2 * kGramRows * kGramTile * sizeof(T) + 64;
}

// FP32: four CTAs per SM (64 registers, no spills; 80 otherwise, which
// allows three while the shared memory fits six); FP64: two
template <typename T>
constexpr int leafgram_min_ctas()
{
    return sizeof(T) == 4 ? 4 : 2;
}

template <typename T, int RP>
__global__ void __launch_bounds__(NT, (leafgram_min_ctas<T>())) k_leafgram(DevTree t, Work<T> w, int reg0)
{
    constexpr int TS = kGramTile, RW = kGramRows;
    using TL = Tile<TS, TS>;
    constexpr int RT = TL::RT, CT = TL::CT;
    // region P of level M-1; Ain holds the regions reg0, reg0 + 1, ... of this launch
    const int P = reg0 + blockIdx.x, Pl = blockIdx.x, b = blockIdx.z, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const int M = t.M, J = t.Jl[M - 1], D = M - 1, UC = D * RP;
    const int np = npairs(D);
    // upper-triangle tile (ti <= tj) from the linear index
    const int nt = (UC + TS - 1) / TS;
    int ti = 0, rem = blockIdx.y;
    while (rem >= nt - ti) {
        rem -= nt - ti;
        ti++;
    }
    const int tj = ti + rem;
    const int ca = ti * TS, cb = tj * TS; // first column of the A and B operands
    const int wa = min(TS, UC - ca), wb = min(TS, UC - cb);
    const int64_t r0 = t.leaf_off[(int64_t)P * J], r1 = t.leaf_off[(int64_t)P * J + J];
    const T *Ub = w.U + (size_t)b * w.U_stride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sbuf = (T *)smem_raw; // 2 stages x (A: RW x TS, B: RW x TS)
    const int i0 = TL::r0(), j0 = TL::c0();
    T hi[RT][CT], lo[RT][CT];
    tile_zero(hi);
    tile_zero(lo);
    // stage a chunk of rows [rb, rb + RW) into buffer st (zero past the end)
    auto stage = [&](int64_t rb, int st) {
        T *sA = sbuf + (size_t)st * 2 * RW * TS, *sB = sA + RW * TS;
        const int nr = (int)min((int64_t)RW, r1 - rb);
        constexpr int VPR = TS * (int)sizeof(T) / 16; // 16-byte vectors per staged row
        for (int e = tid; e < 2 * RW * VPR; e += NT) {
            const int which = e / (RW * VPR), a = (e / VPR) % RW, v = e % VPR;
            const int col0 = (which ? cb : ca) + v * (16 / (int)sizeof(T));
            const int wdt = which ? wb : wa;
            T *dst = (which ? sB : sA) + a * TS + v * (16 / (int)sizeof(T));
            if (a < nr && col0 - (which ? cb : ca) < wdt)
                cp_async16(dst, Ub + (size_t)(rb + a) * UC + col0);
            else
                *reinterpret_cast<int4 *>(dst) = make_int4(0, 0, 0, 0);
        }
        cp_async_commit();
    };
    int st = 0;
    if (r0 < r1) stage(r0, 0);
    for (int64_t rb = r0; rb < r1; rb += RW, st ^= 1) {
        const int nr = (int)min((int64_t)RW, r1 - rb);
        if (rb + RW < r1) {
            stage(rb + RW, st ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *sA = sbuf + (size_t)st * 2 * RW * TS, *sB = sA + RW * TS;
        T acc[RT][CT];
        tile_zero(acc);
        tile_fma<T, TS, TS>(acc, sA, TS, sB, TS, nr);
#pragma unroll
        for (int r = 0; r < RT; r++)
#pragma unroll
            for (int c = 0; c < CT; c++) {
                if constexpr (sizeof(T) == 4) {
                    FF s{hi[r][c], lo[r][c]};
                    ff_add(s, acc[r][c]);
                    hi[r][c] = s.hi;
                    lo[r][c] = s.lo;
                } else {
                    hi[r][c] += acc[r][c];
                }
            }
        __syncthreads();
    }
    // scatter into the packed 32 x 32 (RP x RP) blocks with k <= l
    T *out = w.Ain + (size_t)b * w.Ain_stride + (size_t)Pl * np * RP * RP;
#pragma unroll
    for (int r = 0; r < RT; r++) {
        const int gr = ca + i0 + r;
        if (i0 + r >= wa) continue;
        const int k = gr / RP, ii = gr % RP;
#pragma unroll
        for (int c = 0; c < CT; c++) {
            const int gc = cb + j0 + c;
            if (j0 + c >= wb) continue;
            const int l = gc / RP, jj = gc % RP;
            if (k <= l) out[(size_t)pidx(k + 1, l + 1) * RP * RP + ii * RP + jj] = hi[r][c] + lo[r][c];
        }
    }
    if (blockIdx.y == 0) {
        const double *lw = w.leaf_w + (size_t)b * w.leafw_stride;
        const double *ldu = w.leaf_du + (size_t)b * w.leafdu_stride;
        double *wo = w.Ain_w + (size_t)b * w.Ainw_stride + (size_t)Pl * UC;
        for (int col = tid; col < UC; col += NT) {
            double s = 0.0;
            for (int j = 0; j < J; j++) {
                const int64_t c = (int64_t)P * J + j;
                if (t.leaf_off[c + 1] > t.leaf_off[c]) s += lw[(size_t)c * UC + col];
            }
            wo[col] = s;
        }
        if (tid == 0) {
            double d = 0.0, u = 0.0;
            for (int j = 0; j < J; j++) {
                const int64_t c = (int64_t)P * J + j;
                if (t.leaf_off[c + 1] > t.leaf_off[c]) {
                    d += ldu[2 * c];
                    u += ldu[2 * c + 1];
                }
            }
            double *du = w.Ain_du + (size_t)b * w.Aindu_stride + 2 * (size_t)Pl;
            du[0] = d;
            du[1] = u;
        }
    }
}

// ------------------------------------------------------------- upward pass --
// Region i of level m: A = sum of the children's ATilde (or the leaf Gram for
// m = M-1); I + A^{m,m} = Lt Lt' (FP64); Z_k = Lt^{-1} A^{m,k} (T),
// z = Lt^{-1} w^m (FP64); ATilde^{k,l} = A^{k,l} - Z_k' Z_l (k <= l < m);
// wTilde^k = w^k - Z_k' z; d += log|I + A^{m,m}|, u -= z'z.  At the root,
// loglik = -(d + u + n log 2 pi) / 2.
template <typename T, int RP>
__host__ __device__ constexpr size_t smem_up_bytes(int m)
{
    return (size_t)RP * (RP + 1) * 8 + (size_t)(m * RP) * 8 + (size_t)(RP + RP + 2 + 8) * 8 +
           chol_scratch_bytes<T, RP>() + 64 + (size_t)(2 * m - 1) * RP * RP * sizeof(T) +
           (size_t)4 * RP * sizeof(T) + 64;
}

// Deep levels (the m blocks of column m and the m - 1 of Z exceed one CTA's
// shared memory): k_up<T, RP, KB> keeps A^{m,m} and stages the right-hand
// blocks of the solve KB at a time; every column of Z is solved by the same
// operations as with all blocks staged.
template <typename T, int RP, int KB>
__host__ __device__ constexpr size_t smem_up_stream_bytes(int m)
{
    return (size_t)RP * (RP + 1) * 8 + (size_t)(m * RP) * 8 + (size_t)(RP + RP + 2 + 8) * 8 +
           chol_scratch_bytes<T, RP>() + 64 + (size_t)(KB + 1 + m - 1) * RP * RP * sizeof(T) +
           (size_t)4 * RP * sizeof(T) + 64;
}

// dst[e] = sum over the NS children of src[s][e], e < count (a multiple of
// 16 bytes), added in the order s = 0, 1, ..: 16-byte loads, two per child
// and thread in flight (the children's blocks come from L2 or HBM, and one
// region's chain of such sums is the latency of the upward pass's top levels)
template <typename T, int NS>
__device__ __forceinline__ void sum_children(T *dst, const T *const *src, size_t off, int count)
{
    constexpr int V = 16 / (int)sizeof(T);
    const T *p[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) p[s] = src[s] + off;
    const int nv = count / V;
#pragma unroll 2
    for (int e = threadIdx.x; e < nv; e += NT) {
        T a[NS][V];
#pragma unroll
        for (int s = 0; s < NS; s++) ldv<T, V>(a[s], p[s] + (size_t)e * V);
#pragma unroll
        for (int q = 0; q < V; q++) {
            T v = a[0][q];
#pragma unroll
            for (int s = 1; s < NS; s++) v += a[s][q];
            dst[(size_t)e * V + q] = v;
        }
    }
}

// The parent's blocks of the upward step: for every pair p = pidx(k, l),
// l = 1..m-1, k = 1..l, out_p = sum of the NS sources' block p minus
// Z_k' Z_l (Z rows of RP, k-major at sZ + (k-1) RP, ld ldz).  The next pair's
// source elements are loaded before this pair's product, so their latency
// hides behind the FMAs; each output is formed as in one pass per pair.
template <typename T, int RP, int NS>
__device__ __forceinline__ void up_parent_blocks(T *out, const T *const *blk, const T *sZ, int ldz, int m)
{
    using TL = Tile<RP, RP>;
    constexpr int B2 = RP * RP;
    const int i0 = TL::r0(), j0 = TL::c0();
    const int np = npairs(m - 1);
    T cur[NS][TL::RT][TL::CT], nxt[NS][TL::RT][TL::CT];
    auto load = [&](T (&v)[NS][TL::RT][TL::CT], int p) {
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int r = 0; r < TL::RT; r++)
                ldv<T, TL::CT>(v[s][r], blk[s] + (size_t)p * B2 + (i0 + r) * RP + j0);
    };
    if (np > 0) load(cur, 0);
    int k = 1, l = 1;
    for (int p = 0; p < np; p++) {
        if (p + 1 < np) load(nxt, p + 1);
        T acc[TL::RT][TL::CT];
        tile_zero(acc);
        tile_fma<T, RP, RP>(acc, sZ + (k - 1) * RP, ldz, sZ + (l - 1) * RP, ldz, RP);
#pragma unroll
        for (int r = 0; r < TL::RT; r++)
#pragma unroll
            for (int c = 0; c < TL::CT; c++) {
                T v = cur[0][r][c];
#pragma unroll
                for (int s = 1; s < NS; s++) v += cur[s][r][c];
                out[(size_t)p * B2 + (i0 + r) * RP + j0 + c] = v - acc[r][c];
            }
        if (p + 1 < np) {
#pragma unroll
            for (int s = 0; s < NS; s++)
#pragma unroll
                for (int r = 0; r < TL::RT; r++)
#pragma unroll
                    for (int c = 0; c < TL::CT; c++) cur[s][r][c] = nxt[s][r][c];
        }
        if (++k > l) {
            l++;
            k = 1;
        }
    }
}

template <typename T, int RP, int KB = 0>
__global__ void __launch_bounds__(NT) k_up(DevTree t, Work<T> w, int m, int reg0)
{
    using TL = Tile<RP, RP>;
    using F = typename FacT<T>::type;
    constexpr int B2 = RP * RP;
    // region i of level m; at m = M-1 the Ain buffer holds regions reg0, reg0 + 1, ...
    const int i = reg0 + blockIdx.x, il = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) {
        if (m == 1 && tid == 0) {
            w.loglik[b] = qnan();
            w.status[b] = ST_EINVAL;
        }
        return;
    }
    const int M = t.M, J = t.Jl[m];
    const bool direct = (m == M - 1);
    const int nsrc = direct ? 1 : J;
    const int np = npairs(m), npo = npairs(m - 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sL = (F *)smem_raw;                       // RP x (RP+1)
    double *sw = (double *)(sL + RP * (RP + 1)); // m RP
    F *sz = (F *)(sw + m * RP);                  // RP
    F *srs = sz + RP;                            // RP + 2
    double *red = (double *)(srs + RP + 2);      // 8
    F *sr2 = (F *)(red + 8);                     // RP + 1 (FP64 only)
    int *flag = (int *)((unsigned char *)sr2 + chol_scratch_bytes<T, RP>());
    T *sC = (T *)(flag + 16);                    // m blocks A^{k,m}, row-major (KB > 0: A^{m,m}, then KB staged)
    T *sZ = sC + (size_t)(KB > 0 ? KB + 1 : m) * B2; // RP x ((m-1) RP + 4)
    // subtree streaming: levels below sub_level keep only the chunk's regions
    const bool loc_out = w.sub_level > 0 && m > w.sub_level, loc_in = w.sub_level > 0 && m >= w.sub_level;
    const int64_t io = loc_out ? (int64_t)il : (int64_t)i, ic = loc_in ? (int64_t)il : (int64_t)i;
    const T *blk[4];
    const double *wv[4], *dus[4];
    for (int s = 0; s < nsrc; s++) {
        if (direct) {
            blk[s] = w.Ain + (size_t)b * w.Ain_stride + (size_t)il * np * B2;
            wv[s] = w.Ain_w + (size_t)b * w.Ainw_stride + (size_t)il * m * RP;
            dus[s] = w.Ain_du + (size_t)b * w.Aindu_stride + 2 * (size_t)il;
        } else {
            const int64_t ch = ic * J + s;
            blk[s] = w.Atil[m + 1] + (size_t)b * w.Atil_stride[m + 1] + (size_t)ch * np * B2;
            wv[s] = w.Atil_w[m + 1] + (size_t)b * w.Atilw_stride[m + 1] + (size_t)ch * m * RP;
            dus[s] = w.Atil_du[m + 1] + (size_t)b * w.Atildu_stride[m + 1] + 2 * (size_t)ch;
        }
    }
    if (tid == 0) flag[0] = 0;
    // column m: A^{k,m}, k = 1..m, contiguous blocks pidx(1,m) .. pidx(m,m)
    // (KB > 0: only A^{m,m} here, the others staged for the solve)
    const size_t c0off = (size_t)pidx(1, m) * B2;
    const int nfirst = KB > 0 ? 1 : m;
    const size_t f0off = c0off + (size_t)(m - nfirst) * B2;
    if (direct) {
        copy_g2s_async(sC, blk[0] + f0off, nfirst * B2);
        cp_async_commit();
    } else if (nsrc == 4) {
        sum_children<T, 4>(sC, blk, f0off, nfirst * B2);
    } else if (nsrc == 2) {
        sum_children<T, 2>(sC, blk, f0off, nfirst * B2);
    } else {
        sum_children<T, 1>(sC, blk, f0off, nfirst * B2);
    }
    for (int e = tid; e < m * RP; e += NT) {
        double v = wv[0][e];
        for (int s = 1; s < nsrc; s++) v += wv[s][e];
        sw[e] = v;
    }
    double dsum = 0.0, usum = 0.0;
    for (int s = 0; s < nsrc; s++) {
        dsum += dus[s][0];
        usum += dus[s][1];
    }
    if (direct) cp_async_wait<0>();
    __syncthreads();
    const T *Cm = sC + (size_t)(nfirst - 1) * B2;
    for (int e = tid; e < B2; e += NT) {
        const int a = e / RP, c = e % RP;
        if (c <= a) {
            F v = f_of_T(Cm[e]);
            if (a == c) v = f_add(v, f_of<F>(1.0));
            sL[a * (RP + 1) + c] = v;
        }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4)
        chol_blocked<RP>(sL, RP + 1, RP, srs, flag, MRA_SINGULAR, red);
    else
        chol_small<F, (tri_count(RP) + NT - 1) / NT>(sL, RP + 1, RP, srs, sr2, flag, MRA_SINGULAR);
    const double ld = logdet_small(sL, RP + 1, RP, red);
    // Z = Lt^{-1} [A^{m,1} .. A^{m,m-1}], stored row-major [a][(k-1) RP + bc] (ld ldz);
    // right-hand column (k, bc) is A^{m,k}[.][bc] = A^{k,m}[bc][.], contiguous in sC
    const int ncol = (m - 1) * RP, ldz = ncol + 4;
    for (int a = tid; a < RP; a += NT) sz[a] = f_of<F>(sw[(m - 1) * RP + a]);
    if constexpr (KB > 0) {
        T *stg = sC + B2;
        for (int k0 = 0; k0 < m - 1; k0 += KB) {
            const int nb = min(KB, m - 1 - k0);
            const size_t off = c0off + (size_t)k0 * B2;
            if (direct) {
                copy_g2s_async(stg, blk[0] + off, nb * B2);
                cp_async_commit();
                cp_async_wait<0>();
            } else if (nsrc == 4) {
                sum_children<T, 4>(stg, blk, off, nb * B2);
            } else if (nsrc == 2) {
                sum_children<T, 2>(stg, blk, off, nb * B2);
            } else {
                sum_children<T, 1>(stg, blk, off, nb * B2);
            }
            __syncthreads();
            fwd_solve_warp<T, RP>(sL, RP + 1, srs, stg, RP, 1, sZ + (size_t)k0 * RP, ldz, nb * RP);
        }
        fwd_solve_vec_lead<F, RP>(sL, RP + 1, srs, RP, sz);
    } else {
        // the vector solve (a 32-step chain) on warp 0 beside the columns of Z
        // on the other warps: the same operations on each column and on z
        __syncwarp();
        if (tid < 32)
            fwd_solve_vec_lead_warp<F, RP>(sL, RP + 1, srs, RP, sz);
        else
            fwd_solve_warps<T, RP>(sL, RP + 1, srs, sC, RP, 1, sZ, ldz, ncol, RP, 1, NT / 32 - 1);
        __syncthreads();
    }
    if (tid < 32) {
        F q = tid < RP ? f_sqr(sz[tid]) : f_of<F>(0.0);
        q = warp_sum_f(q);
        if (tid == 0) red[0] = f_dbl(q);
    }
    __syncthreads();
    const double q2 = red[0];
    const double dR = dsum + ld, uR = usum - q2;
    const int64_t g = t.lvl_off[m] + i;
    if (w.keep_up && b == 0) {
        // factors for prediction (layout: keep_up_doubles)
        double *kp = w.keep_up + (size_t)g * w.keep_up_stride;
        for (int e = tid; e < B2; e += NT) {
            const int a = e / RP, q = e % RP;
            kp[e] = q <= a ? f_dbl(sL[q * (RP + 1) + a]) : 0.0;
        }
        for (int a = tid; a < RP; a += NT) {
            kp[B2 + a] = f_dbl(srs[a]);
            kp[B2 + RP + a] = f_dbl(sz[a]);
        }
        const int ldk = (M - 2) * RP;
        for (int e = tid; e < RP * ncol; e += NT) {
            const int a = e / ncol, q = e % ncol;
            kp[B2 + 2 * RP + (size_t)a * ldk + q] = (double)sZ[a * ldz + q];
        }
    }
    if (m > 1) {
        T *out = w.Atil[m] + (size_t)b * w.Atil_stride[m] + (size_t)io * npo * B2;
        // pair p = pidx(k, l), l = 1..m-1, k = 1..l, in order
        if (nsrc == 4)
            up_parent_blocks<T, RP, 4>(out, blk, sZ, ldz, m);
        else if (nsrc == 2)
            up_parent_blocks<T, RP, 2>(out, blk, sZ, ldz, m);
        else
            up_parent_blocks<T, RP, 1>(out, blk, sZ, ldz, m);
        double *wo = w.Atil_w[m] + (size_t)b * w.Atilw_stride[m] + (size_t)io * (m - 1) * RP;
        for (int e = tid; e < (m - 1) * RP; e += NT) {
            F acc = f_of<F>(0.0);
            for (int q = 0; q < RP; q++) acc = f_add(acc, f_mul(f_of_T(sZ[q * ldz + e]), sz[q]));
            wo[e] = sw[e] - f_dbl(acc);
        }
        if (tid == 0) {
            double *du = w.Atil_du[m] + (size_t)b * w.Atildu_stride[m] + 2 * (size_t)io;
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
            w.loglik[b] = w.status[b] == ST_OK ? ll : qnan();
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
        w.loglik[b] = qnan();
        w.status[b] = ST_EINVAL;
        return;
    }
    const double *du = w.leaf_du + (size_t)b * w.leafdu_stride;
    const double ll = -0.5 * (du[0] + du[1] + (double)t.n_used * 1.8378770664093454836);
    w.loglik[b] = w.status[b] == ST_OK ? ll : qnan();
}

} // namespace mra

#include "mra_bigleaf.cuh"
#include "mra_predict.cuh"
