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
// Exact slices.  Both factors are bounded by sigma, so each is split on one
// fixed grid into five BF16 slices q_0..q_4 (tc_slices, mra_kernels.cuh:
// q_i a multiple of 2^(e - 7 - 8 i), at most 128 such steps).  Their products
// are summed by order s = i + j (s <= 5; orders 6 to 8 are below 2^(2e - 46)
// a product and dropped) into tensor-memory column block s.  Within one order
// every product is an integer multiple of 2^(2e - 14 - 8 s) of at most 2^14
// steps, and an order has at most 5 pairs, so sums over K <= 192 columns stay
// below 5 * 192 * 2^14 < 2^24 steps: the tensor cores add them exactly,
// whatever they do with lower bits.  The CUDA cores form the total in float
// pairs (the three smallest orders summed in FP32 first, below 2^-47 of the
// total), subtract it from the float-pair covariance and round W to FP32 once,
// as the CUDA-core kernel's remainder_ff does (whose product sum is accurate
// to ~1e-11 sigma2).
//
// Slices are made once per value, stored step-major (one K = 16 step of all
// five slices contiguous).  The prior writes each region's blocks What^k_A as
// slices (Work::lbB); this kernel slices its rows' What^l when it makes them,
// into the chunk's part of Work::lbA.  Per level, thread 0 streams the steps
// of every ancestor block through two shared-memory stages with bulk copies
// (two steps ahead), issues each step's 19 MMAs (no-swizzle K-major core
// matrices, tc_sm100.cuh) and commits them to the stage's mbarrier; the other
// threads meanwhile load the level's coordinates and Linv, then wait
// (bounded) for the level's last commit.  A CTA of 256 threads takes 128 rows
// of one level-(M-1) region (the MMA's M; rows past the region's end are zero)
// and one theta; two threads share a row (TMEM lane), each with half of the
// columns: it reads the six accumulators there, forms W, and computes half of
// What^l with FP32 FMAs in the order the CUDA-core kernel uses.
#pragma once
#include "tc_sm100.cuh"

namespace mra {

constexpr int kLbTcRows = 128;      // observation rows per CTA (the MMA's M)
constexpr int kLbTcThreads = 256;   // two threads per row
constexpr int kLbTcOrders = 6;      // slice orders 0..5 kept
constexpr int kLbTcMaxK = 192;      // ancestor columns one remainder sums over (exactness bound)
constexpr uint32_t kLbTcPolls = 1u << 24;

template <int RP>
__host__ __device__ constexpr uint32_t lbtc_tmem_cols()
{
    return RP == 32 ? 256u : 128u; // orders 0..5 at s * RP, rounded up to a power of two
}
// one K step of the rows' operand (128 rows) and of a knot block (RP rows),
// all five slices; a block of RP columns has RP / 16 steps
template <int RP>
__host__ __device__ constexpr size_t lbtc_a_step() { return kTcSlices * tc_step_plane<kLbTcRows>(); }
template <int RP>
__host__ __device__ constexpr size_t lbtc_b_step() { return kTcSlices * tc_step_plane<RP>(); }
// bytes of the rows' slices per level (one block of RP columns)
template <int RP>
__host__ __device__ constexpr size_t lbtc_a_level_bytes() { return (size_t)(RP / 16) * lbtc_a_step<RP>(); }
// dynamic shared memory: two stages of one K step (A and B), W (transposed),
// Linv, row and knot coordinates; at RP = 32 at least 80 KB so that at most
// two CTAs (2 x 256 TMEM columns) share an SM
template <int RP>
__host__ __device__ constexpr size_t smem_leafbasis_tc_need()
{
    return 1024 + 2 * (lbtc_a_step<RP>() + lbtc_b_step<RP>()) + (size_t)RP * kLbTcRows * 4 + (size_t)RP * RP * 4 +
           (size_t)2 * kLbTcRows * 4 + (size_t)2 * RP * 4;
}
template <int RP>
__host__ __device__ constexpr size_t smem_leafbasis_tc_bytes()
{
    return RP == 32 && smem_leafbasis_tc_need<RP>() < (size_t)80 * 1024 ? (size_t)80 * 1024
                                                                          : smem_leafbasis_tc_need<RP>();
}


template <int RP>
__global__ void __launch_bounds__(kLbTcThreads) k_leafbasis_tc(DevTree t, Work<float> w, const Chunk *chunks)
{
    constexpr int H = RP / 2;   // columns per thread (two threads per row)
    constexpr int KS = RP / 16; // K steps per block
    constexpr uint32_t LBO = 128u, SBO = 256u;
    constexpr uint32_t APL = (uint32_t)tc_step_plane<kLbTcRows>(), BPL = (uint32_t)tc_step_plane<RP>();
    constexpr uint32_t AST = (uint32_t)lbtc_a_step<RP>(), BST = (uint32_t)lbtc_b_step<RP>();
    constexpr size_t ABY = lbtc_a_level_bytes<RP>(), BBY = tc_block_bytes<RP>();
    const int cidx = blockIdx.x;
    const Chunk ch = chunks[cidx];
    const int b = blockIdx.y, tid = threadIdx.x, warp = tid >> 5;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    __shared__ double s_ib;
    __shared__ ff s_par[2];     // sigma2 and 1/beta as float pairs
    __shared__ uint64_t mcp[2]; // stage s filled (bulk copies)
    __shared__ uint64_t mmm[2]; // stage s read (MMAs committed)
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    set_cov_params<float>(th, &s_ib, s_par);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *stage = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023); // 2 x (A step, B step)
    float *sW = reinterpret_cast<float *>(stage + 2 * (AST + BST)); // W(x_a, j) at j * 128 + a
    float *sLi = sW + RP * kLbTcRows;                                // Linv_A: (c, j) at j RP + c
    float *sp = sLi + RP * RP;                                       // rows: x at [a], y at [128 + a]
    float *sa = sp + 2 * kLbTcRows;                                  // knots: x at [j], y at [RP + j]
    const int M = t.M, P = ch.parent, nr = ch.n, UC = (M - 1) * RP;
    float *Ub = w.U + (size_t)b * w.U_stride;
    const float *pb = w.prior + (size_t)b * w.prior_stride;
    unsigned char *myA = w.lbA + (size_t)b * w.lbA_stride + (size_t)cidx * (size_t)(M - 2) * ABY;
    const unsigned char *lB = w.lbB + (size_t)b * w.lbB_stride;
    const TcGrid gr = tc_grid(th[0]);

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, lbtc_tmem_cols<RP>());
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < 2; q++) {
            tc::mbar_init(&mcp[q], 1);
            tc::mbar_init(&mmm[q], 1);
        }
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
    // commits (and copies) made on each stage before this level: the same in
    // every thread, so that every wait knows the parity of its phase
    int ncs[2] = {0, 0};
    // the producer's copies issued and consumed, commits made, and commit
    // phases known complete, per stage (for a drain after a wait gave up:
    // phases are waited for one at a time)
    int issued[2] = {0, 0}, waited[2] = {0, 0}, made[2] = {0, 0}, conf[2] = {0, 0};
    bool bad = false;
    for (int l = 1; l <= M - 1; l++) {
        const int64_t ia = anc_index(t, P, M - 1, l);
        const int64_t ga = t.lvl_off[l] + ia;
        const int R = t.Rl[l]; // the ancestor's knots
        // the ancestor's prior: What^1 .. What^{l-1}, then Linv (column-major);
        // and the slices of its What blocks
        const float *anc = pb + w.prior_lvl[l] + (size_t)ia * l * RP * RP;
        const unsigned char *ancB = lB + w.lbB_lvl[l] + (size_t)ia * (size_t)(l - 1) * BBY;
        const int nsteps = (l - 1) * KS;
        // the producer: bulk copies two steps ahead, the MMAs of each step, commits
        if (tid == 0 && nsteps > 0) {
            auto issue = [&](int q) {
                const int s = q & 1, k = q / KS + 1, kk = q % KS;
                unsigned char *st = stage + (size_t)s * (AST + BST);
                tc::mbar_expect_tx(&mcp[s], AST + BST);
                tc::bulk_g2s(st, myA + (size_t)(k - 1) * ABY + (size_t)kk * AST, AST, &mcp[s]);
                tc::bulk_g2s(st + AST, ancB + (size_t)(k - 1) * BBY + (size_t)kk * BST, BST, &mcp[s]);
                issued[s]++;
            };
            issue(0);
            if (nsteps > 1) issue(1);
            for (int q = 0; q < nsteps; q++) {
                const int s = q & 1, idx = ncs[s] + q / 2;
                if (!tc::mbar_wait(&mcp[s], (uint32_t)(idx & 1), kLbTcPolls)) {
                    bad = true;
                    break;
                }
                waited[s]++;
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_addr(stage + (size_t)s * (AST + BST)), b0 = a0 + AST;
#pragma unroll
                for (int i = 0; i < kTcSlices; i++)
#pragma unroll
                    for (int j = 0; j < kTcSlices; j++) {
                        const int o = i + j;
                        if (o >= kLbTcOrders) continue;
                        // the level's first product of order o overwrites D_o
                        const int ifirst = o > kTcSlices - 1 ? o - (kTcSlices - 1) : 0;
                        const uint32_t accum = (q == 0 && i == ifirst) ? 0u : 1u;
                        tc::mma_bf16(tmem + (uint32_t)(o * RP), tc::smem_desc(a0 + (uint32_t)i * APL, LBO, SBO),
                                     tc::smem_desc(b0 + (uint32_t)j * BPL, LBO, SBO), idesc, accum);
                    }
                tc::mma_commit(&mmm[s]);
                made[s]++;
                if (q + 2 < nsteps) {
                    // the stage is refilled once its MMAs have read it
                    if (!tc::mbar_wait(&mmm[s], (uint32_t)(idx & 1), kLbTcPolls)) {
                        bad = true;
                        break;
                    }
                    conf[s] = idx + 1;
                    issue(q + 2);
                }
            }
        }
        // meanwhile: the coordinates, the knots and Linv of the ancestor
        if (tid < kLbTcRows) {
            const double ox = t.cx[ga], oy = t.cy[ga];
            sp[tid] = tid < nr ? (float)(t.sx[ch.row0 + tid] - ox) : 0.f;
            sp[kLbTcRows + tid] = tid < nr ? (float)(t.sy[ch.row0 + tid] - oy) : 0.f;
        }
        if (tid < RP) {
            const double ox = t.cx[ga], oy = t.cy[ga];
            sa[tid] = (float)(t.kx[ga * RP + tid] - ox);
            sa[RP + tid] = (float)(t.ky[ga * RP + tid] - oy);
        }
        for (int q = tid; q < RP * RP; q += kLbTcThreads) sLi[q] = anc[(size_t)(l - 1) * RP * RP + q];
        if (nsteps > 0) {
            // every thread: the level's last commit (all its MMAs are then done)
            const int sl = (nsteps - 1) & 1, idx = ncs[sl] + (nsteps - 1) / 2;
            if (!bad && !tc::mbar_wait(&mmm[sl], (uint32_t)(idx & 1), kLbTcPolls)) bad = true;
            ncs[0] += (nsteps + 1) / 2;
            ncs[1] += nsteps / 2;
            if (!bad) {
                // commits complete in order: every phase so far is done
                conf[0] = ncs[0];
                conf[1] = ncs[1];
            }
        }
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
        tc::fence_after_sync();
        // W = C(x, q) - sum_o D_o in float pairs, rounded to FP32 once
        {
            ff sum[H];
#pragma unroll
            for (int q = 0; q < H; q++) sum[q] = ff{0.f, 0.f};
            if (l > 1) {
                // ((D0 + D1) + D2) + ((D5 + D4) + D3), two accumulators read at a time
                auto ld = [&](int o, float (&d)[H]) {
                    if constexpr (H == 16)
                        tc::tmem_ld16(tmem + lane_base + (uint32_t)(o * RP + c0), d);
                    else
                        tc::tmem_ld8(tmem + lane_base + (uint32_t)(o * RP + c0), d);
                };
                float d0[H], d1[H];
                ld(0, d0);
                ld(1, d1);
#pragma unroll
                for (int q = 0; q < H; q++) sum[q] = two_sum(d0[q], d1[q]);
                ld(2, d0);
#pragma unroll
                for (int q = 0; q < H; q++) sum[q] = ff_add_f(sum[q], d0[q]);
                ld(5, d0);
                ld(4, d1);
#pragma unroll
                for (int q = 0; q < H; q++) d0[q] = FADD(d0[q], d1[q]);
                ld(3, d1);
#pragma unroll
                for (int q = 0; q < H; q++) sum[q] = ff_add_f(sum[q], FADD(d0[q], d1[q]));
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
            if (l <= M - 2) {
                // the slices of What^l for the later levels' bulk copies (rows
                // past nr are zero)
#pragma unroll
                for (int gq = 0; gq < H / 8; gq++) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) v[q] = acc[8 * gq + q];
                    tc_put8(myA + (size_t)(l - 1) * ABY, APL, tc_step_off<kLbTcRows>(a, c0 / 8 + gq), v, gr);
                }
                tc::fence_proxy_async_global();
            }
        }
        // level l's slices are read by later levels' bulk copies; sW, sLi, sp
        // and sa are refilled
        __syncthreads();
    }
    if (__syncthreads_or(bad)) s_bad = 1;
    __syncthreads();
    if (s_bad && tid == 0) {
        // a wait gave up: report it, then let the copies and MMAs in flight
        // drain (bounded) before the shared and tensor memory go away
        w.status[b] = ST_ETIMEDOUT;
        for (int s = 0; s < 2; s++)
            for (int c = waited[s]; c < issued[s]; c++) (void)tc::mbar_wait(&mcp[s], (uint32_t)(c & 1), kLbTcPolls);
        for (int s = 0; s < 2; s++)
            for (int c = conf[s]; c < made[s]; c++) (void)tc::mbar_wait(&mmm[s], (uint32_t)(c & 1), kLbTcPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, lbtc_tmem_cols<RP>());
}

} // namespace mra
