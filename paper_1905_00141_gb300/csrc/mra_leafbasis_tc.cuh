// mra_leafbasis_tc.cuh -- the leaf basis of the mixed mode with its remainder
// products on the tensor cores (tcgen05, kind::f16, BF16 slices on a fixed
// grid, sums exact in tensor memory).
//
// For observation rows x below a level-(M-1) region and its level-l ancestor
// A (Sec. 1.1 recursion in the whitened form), level by level:
//     W(x, j)  = C(x, q_j) - sum_{k<l} sum_t What^k(x, t) What^k_A(j, t)
//     What^l(x, c) = sum_j W(x, j) Linv_A(c, j),
// the remainder's product sum needing ~1e-11 sigma2 where W is small.
//
// Exact slices on a fixed grid.  Every entry of What^k at a point and of
// What^k_A at a knot is bounded by sigma (sum_k |What^k(x)|^2 <= C(x, x)), so
// one grid serves all of them: with 2^e > 2 sigma, a value v is split as
//     v = q0 + q1 + q2 + q3 + q4,   q_i = n_i 2^(e - 7 - 8 i),  |n_i| <= 128,
// exact for an FP32 v down to 2^(e - 40) (BF16 holds each q_i exactly).  The
// products q_i^a q_j^b are summed by order s = i + j (s <= 5; orders 6 to 8
// are below 2^(2e - 46) a product and dropped): D_s in tensor-memory column
// block s.  Within one order every product is an integer multiple of
// 2^(2e - 14 - 8 s) of at most 2^14 such steps, and an order has at most 5
// pairs, so sums over K <= 192 columns stay below 5 * 192 * 2^14 < 2^24 steps:
// the tensor cores add them exactly, whatever they do with lower bits.  The
// CUDA cores then form D_0 + ... + D_5 in float pairs, subtract it from the
// float-pair covariance and round W to FP32 once, as the CUDA-core kernel's
// remainder_ff does (there the product sum is accurate to ~1e-11 sigma2).
//
// A CTA of 256 threads takes 128 rows of one level-(M-1) region (the MMA's
// M = 128; rows past the region's end are zero) and one theta.  Per level
// and per ancestor block k it slices What^k of its rows (read back from U,
// which this CTA wrote at level k) and What^k_A (the prior) into one stage of
// shared memory (no-swizzle K-major core matrices, tc_sm100.cuh), thread 0
// issues the 19 MMAs of each K = 16 step and commits them to an mbarrier, and
// the threads wait (bounded) before the next block refills the stage.  Two
// threads share a row (TMEM lane): each reads half of the columns of the six
// accumulators, forms W, and computes half of What^l with FP32 FMAs in the
// order the CUDA-core kernel uses.
#pragma once
#include "tc_sm100.cuh"

namespace mra {

constexpr int kLbTcRows = 128;      // observation rows per CTA (the MMA's M)
constexpr int kLbTcThreads = 256;   // two threads per row
constexpr int kLbTcSlices = 5;
constexpr int kLbTcOrders = 6;      // slice orders 0..5 kept
constexpr int kLbTcMaxK = 192;      // ancestor columns one remainder sums over (exactness bound)
constexpr uint32_t kLbTcPolls = 1u << 24;

template <int RP>
__host__ __device__ constexpr uint32_t lbtc_tmem_cols()
{
    return RP == 32 ? 256u : 128u; // orders 0..5 at s * RP, rounded up to a power of two
}
template <int RP>
__host__ __device__ constexpr size_t lbtc_a_slice() { return (size_t)kLbTcRows * RP * 2; }
template <int RP>
__host__ __device__ constexpr size_t lbtc_b_slice() { return (size_t)RP * RP * 2; }
// dynamic shared memory: A and B stages, W (transposed), Linv, row and knot
// coordinates; at RP = 32 at least 80 KB so that at most two CTAs (2 x 256
// TMEM columns) share an SM
template <int RP>
__host__ __device__ constexpr size_t smem_leafbasis_tc_need()
{
    return 1024 + kLbTcSlices * (lbtc_a_slice<RP>() + lbtc_b_slice<RP>()) + (size_t)RP * kLbTcRows * 4 +
           (size_t)RP * RP * 4 + (size_t)2 * kLbTcRows * 4 + (size_t)2 * RP * 4;
}
template <int RP>
__host__ __device__ constexpr size_t smem_leafbasis_tc_bytes()
{
    return RP == 32 && smem_leafbasis_tc_need<RP>() < (size_t)80 * 1024 ? (size_t)80 * 1024
                                                                          : smem_leafbasis_tc_need<RP>();
}

// The five slices of v (|v| < 2^(e-1)) as BF16 bit patterns in absolute
// units; down = 2^-e, up = 2^e.
__device__ __forceinline__ void lbtc_slices(float v, float down, float up, uint32_t (&q)[kLbTcSlices])
{
    float r = __fmul_rn(v, down); // |r| < 1/2, exact
    float sc = 128.f, isc = 0.0078125f;
#pragma unroll
    for (int i = 0; i < kLbTcSlices; i++) {
        const float qi = __fmul_rn(rintf(__fmul_rn(r, sc)), isc); // a multiple of 2^(-7-8i), exact
        r = __fsub_rn(r, qi);                                      // exact: qi is r on a coarser grid
        q[i] = __float_as_uint(__fmul_rn(qi, up)) >> 16;           // <= 8 significant bits: BF16 exact
        sc = __fmul_rn(sc, 256.f);
        isc = __fmul_rn(isc, 0.00390625f);
    }
}

// 16 consecutive bytes of one core-matrix row: eight values of one row (or
// knot) at K positions 8g .. 8g + 7, sliced, into the five slice planes of a
// stage (plane stride `plane`, core matrix offset `off`).
__device__ __forceinline__ void lbtc_put8(unsigned char *stage, size_t plane, size_t off, const float (&v)[8],
                                          float down, float up)
{
    uint32_t w[kLbTcSlices][4];
#pragma unroll
    for (int p = 0; p < 4; p++) {
        uint32_t a[kLbTcSlices], b[kLbTcSlices];
        lbtc_slices(v[2 * p], down, up, a);
        lbtc_slices(v[2 * p + 1], down, up, b);
#pragma unroll
        for (int i = 0; i < kLbTcSlices; i++) w[i][p] = a[i] | (b[i] << 16);
    }
#pragma unroll
    for (int i = 0; i < kLbTcSlices; i++)
        *reinterpret_cast<uint4 *>(stage + (size_t)i * plane + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}


template <int RP>
__global__ void __launch_bounds__(kLbTcThreads) k_leafbasis_tc(DevTree t, Work<float> w, const Chunk *chunks)
{
    constexpr int H = RP / 2; // columns per thread (two threads per row)
    constexpr uint32_t LBO = 128u, SBO = (uint32_t)(RP / 8) * 128u;
    constexpr size_t ASL = lbtc_a_slice<RP>(), BSL = lbtc_b_slice<RP>();
    const Chunk ch = chunks[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x, warp = tid >> 5;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    __shared__ double s_ib;
    __shared__ ff s_par[2]; // sigma2 and 1/beta as float pairs
    __shared__ uint64_t mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    set_cov_params<float>(th, &s_ib, s_par);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *stA = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stB = stA + kLbTcSlices * ASL;
    float *sW = reinterpret_cast<float *>(stB + kLbTcSlices * BSL); // W(x_a, j) at j * 128 + a
    float *sLi = sW + RP * kLbTcRows;                                // Linv_A: (c, j) at j RP + c
    float *sp = sLi + RP * RP;                                       // rows: x at [a], y at [128 + a]
    float *sa = sp + 2 * kLbTcRows;                                  // knots: x at [j], y at [RP + j]
    const int M = t.M, P = ch.parent, nr = ch.n, UC = (M - 1) * RP;
    float *Ub = w.U + (size_t)b * w.U_stride;
    const float *pb = w.prior + (size_t)b * w.prior_stride;
    // the slicing grid: 2^e > 2 sigma >= 2 |v| for every sliced value
    const float sg = sqrtf((float)th[0]);
    const int e = (int)((__float_as_uint(sg) >> 23) & 0xffu) - 127 + 2;
    const float up = __int_as_float((127 + e) << 23), down = __int_as_float((127 - e) << 23);

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, lbtc_tmem_cols<RP>());
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_init_fence();
        s_bad = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc_bf16(kLbTcRows, RP);
    // this thread's row a (its TMEM lane) and its half of the columns
    const int a = tid & (kLbTcRows - 1), c0 = (tid >> 7) * H;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    int ncommit = 0;
    bool bad = false;
    for (int l = 1; l <= M - 1; l++) {
        const int64_t ia = anc_index(t, P, M - 1, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int R = t.Rl[l]; // the ancestor's knots
        // the ancestor's l blocks: What^1 .. What^{l-1}, then Linv (column-major)
        const float *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        const double ox = t.cx[ga], oy = t.cy[ga];
        if (tid < kLbTcRows) {
            sp[tid] = tid < nr ? (float)(t.sx[ch.row0 + tid] - ox) : 0.f;
            sp[kLbTcRows + tid] = tid < nr ? (float)(t.sy[ch.row0 + tid] - oy) : 0.f;
        }
        if (tid < RP) {
            sa[tid] = (float)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (float)(t.ky[ga * RP + tid] - oy);
        }
        for (int q = tid; q < RP * RP; q += kLbTcThreads) sLi[q] = anc[(size_t)(l - 1) * RP * RP + q];
        // sum_{k<l} What^k(x) What^k_A' on the tensor cores, one block k at a time
        for (int k = 1; k < l; k++) {
            // A: What^k of the rows (written to U by this CTA at level k)
            for (int it = tid; it < kLbTcRows * (RP / 8); it += kLbTcThreads) {
                const int r = it / (RP / 8), g = it % (RP / 8);
                float v[8];
                if (r < nr) {
                    const float4 *src =
                        reinterpret_cast<const float4 *>(Ub + (size_t)(ch.row0 + r) * UC + (size_t)(k - 1) * RP + 8 * g);
                    const float4 x0 = src[0], x1 = src[1];
                    v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
                    v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; q++) v[q] = 0.f;
                }
                lbtc_put8(stA, ASL, (size_t)(r / 8) * SBO + (size_t)g * LBO + (size_t)(r % 8) * 16, v, down, up);
            }
            // B: What^k of the ancestor's knots (element (j, t) at t RP + j)
            for (int it = tid; it < RP * (RP / 8); it += kLbTcThreads) {
                const int j = it / (RP / 8), g = it % (RP / 8);
                const float *src = anc + (size_t)(k - 1) * RP * RP + (size_t)(8 * g) * RP + j;
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = src[(size_t)q * RP];
                lbtc_put8(stB, BSL, (size_t)(j / 8) * SBO + (size_t)g * LBO + (size_t)(j % 8) * 16, v, down, up);
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_addr(stA), b0 = tc::smem_addr(stB);
                for (int kk = 0; kk < RP / 16; kk++) {
                    const uint32_t ko = (uint32_t)kk * 2u * LBO; // two core matrices along K per step
                    for (int i = 0; i < kLbTcSlices; i++)
#pragma unroll
                        for (int j = 0; j < kLbTcSlices; j++) {
                            const int s = i + j;
                            if (s >= kLbTcOrders) continue;
                            // the level's first product of order s overwrites D_s
                            const int ifirst = s > kLbTcSlices - 1 ? s - (kLbTcSlices - 1) : 0;
                            const uint32_t accum = (k == 1 && kk == 0 && i == ifirst) ? 0u : 1u;
                            tc::mma_bf16(tmem + (uint32_t)(s * RP), tc::smem_desc(a0 + (uint32_t)(i * ASL) + ko, LBO, SBO),
                                         tc::smem_desc(b0 + (uint32_t)(j * BSL) + ko, LBO, SBO), idesc, accum);
                        }
                }
                tc::mma_commit(&mbar);
            }
            // the stage is refilled next: every thread waits for the MMAs (bounded)
            if (!tc::mbar_wait(&mbar, (uint32_t)(ncommit & 1), kLbTcPolls)) bad = true;
            ncommit++;
            if (__syncthreads_or(bad)) break;
        }
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
        tc::fence_after_sync();
        // W = C(x, q) - sum_s D_s in float pairs, rounded to FP32 once
        {
            ff sum[H];
#pragma unroll
            for (int q = 0; q < H; q++) sum[q] = ff{0.f, 0.f};
            if (l > 1) {
#pragma unroll
                for (int s = 0; s < kLbTcOrders; s++) {
                    float d[H];
                    if constexpr (H == 16)
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)(s * RP + c0), d);
                    else
                        tc::tmem_ld8(tmem + lane_base + (uint32_t)(s * RP + c0), d);
#pragma unroll
                    for (int q = 0; q < H; q++) sum[q] = s == 0 ? ff{d[q], 0.f} : ff_add_f(sum[q], d[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < H; q++) {
                const int j = c0 + q;
                ff cv = ff{0.f, 0.f};
                if (a < nr && j < R) cv = ff_cov_exp(s_par[0], s_par[1], sp[a], sp[kLbTcRows + a], sa[j], sa[RP + j]);
                sW[j * kLbTcRows + a] = FADD(FSUB(cv.hi, sum[q].hi), FSUB(cv.lo, sum[q].lo));
            }
        }
        // every warp's TMEM reads are done before the next level's MMAs
        tc::fence_before_sync();
        __syncthreads();
        // What^l = W Linv' in FP32, the CUDA-core kernel's order of terms
        {
            float acc[H];
#pragma unroll
            for (int q = 0; q < H; q++) acc[q] = 0.f;
            for (int jj = 0; jj < RP; jj++) {
                const float wv = sW[jj * kLbTcRows + a];
                const float *li = sLi + jj * RP + c0;
#pragma unroll
                for (int q = 0; q < H; q++) acc[q] = fmaf(wv, li[q], acc[q]);
            }
            if (a < nr) {
                float4 *dst = reinterpret_cast<float4 *>(Ub + (size_t)(ch.row0 + a) * UC + (size_t)(l - 1) * RP + c0);
#pragma unroll
                for (int q = 0; q < H / 4; q++) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            }
        }
        // level l's rows of U are read back by the slicing of later levels;
        // sW, sLi, sp and sa are refilled
        __syncthreads();
    }
    if (__syncthreads_or(bad)) s_bad = 1;
    __syncthreads();
    if (s_bad && tid == 0) {
        // a wait gave up: report it and let the MMAs in flight drain (bounded)
        w.status[b] = ST_ETIMEDOUT;
        if (ncommit > 0) (void)tc::mbar_wait(&mbar, (uint32_t)((ncommit - 1) & 1), kLbTcPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, lbtc_tmem_cols<RP>());
}

} // namespace mra
