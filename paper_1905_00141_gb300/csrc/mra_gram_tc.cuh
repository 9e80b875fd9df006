// mra_gram_tc.cuh -- the leaf Gram blocks of the mixed mode on the tensor
// cores (tcgen05, kind::f16 with BF16 operands, accumulation in tensor
// memory), with sums that are exact in the tensor cores.
//
// For a region P of level M-1 the upward pass starts from
//     A = sum over the leaves c of P of Y_c' Y_c = Y_P' Y_P,
// Y_P the rows of Y = L^{-1} U of all observations below P (FP32, row-major,
// UC = (M-1) RP columns); the packed upper blocks (k <= l) of this UC x UC
// matrix are the ATilde blocks the leaves pass to their parent (App. B).
//
// Exact slices.  The tensor cores accumulate in FP32 and drop the bits below
// the running sum's last place (toward zero, about once per MMA), which biases
// a plain FP32 or 3xTF32 Gram: parity of the likelihood drifted to ~6e-6 per
// observation.  Here every value v of column x of a group of rows is split on
// a grid fixed per column, 2^e >= max |v| over the group:
//     v = 2^e (q0 + q1 + q2 + r),  q0 = i0 2^-7, q1 = i1 2^-15, q2 = i2 2^-23,
// integers |i_k| <= 128 (exact BF16 values) and |r| <= 2^-24, and the
// products are summed by slice order:
//     D0 = sum q0 q0,  D1 = sum (q0 q1 + q1 q0),  D2 = sum (q0 q2 + q1 q1 + q2 q0)
// (all in absolute units; the order-3 and -4 terms and the residual r are
// dropped: below 2^-23 of 2^(e_a + e_b) per product).  Within one order every
// product is an integer multiple of one grid step, at most 2^14 steps, so a
// group of up to 320 rows keeps every partial sum below 2^24 steps and the
// tensor cores add them exactly, whatever they do with lower bits.  D0 + D1 +
// D2 is then formed in float pairs and rounded to FP32 once per group; a
// region of more than 320 rows adds its groups' values in FP32 (one rounding per
// 320 rows, where the CUDA-core Gram rounds once per 32).
//
// Tiles.  A CTA of 128 threads computes a 128 x N tile of A, N <= 64: rows
// [xa0, xa0 + 128) and columns [xb0, xb0 + N), for one region (grid.x), one tile
// (grid.y) and one theta (grid.z).  Row chunk c of the output owns rows
// [128 c, 128 c + 128) (the MMA rows start at min(128 c, UC - 128) so every MMA
// has M = 128); its columns run from 128 c to UC (the upper triangle) in tiles
// of 64.  D0, D1, D2 sit at TMEM columns 0, 64, 128.
//
// Pipeline.  k_gram_colexp first finds each region's column exponents (one
// pass over Y).  Then per group of rows, in chunks of KC rows: all threads load
// (eight steps of loads in flight per thread), slice and store the three
// slices into one of two shared-memory stages in the no-swizzle K-major
// core-matrix layout (tc_sm100.cuh), thread 0 issues the six MMAs per K = 16
// step and commits them to the stage's mbarrier, which the threads wait on
// (bounded) before they refill the stage.  After a group the four warps read
// their 32 TMEM lanes (tile rows) and add the rounded D0 + D1 + D2 to FP32
// registers; at the end they write whole rows of the packed blocks.
#pragma once
#include "tc_sm100.cuh"

namespace mra {

constexpr int kGramTcThreads = 128;
constexpr int kGramTcN = 64;                 // columns per tile
constexpr uint32_t kGramTcCols = 256;        // TMEM columns per CTA: D0, D1, D2 at 0, 64, 128
constexpr uint32_t kGramTcPolls = 1u << 24;  // mbarrier polls before a wait gives up (~seconds)
constexpr int kGramTcGroup = 320;            // rows per exact group
constexpr int kGramTcMaxTiles = 48;
enum { ST_ETIMEDOUT = 5 };

// One output tile of the Gram (host-built list, the same for every region).
struct GramTile {
    int16_t xa0, xb0;  // first row (MMA rows: 128 of them) and first column
    int16_t n;         // columns (a multiple of 16, <= 64)
    int16_t rowlo;     // rows below this one are owned by an earlier chunk
    int16_t u0, w;     // staged columns of Y: [u0, u0 + w), w a multiple of 8
    int16_t kc, pad;   // rows per staged chunk (a multiple of 16)
};
struct GramTiles {
    int n;
    GramTile t[kGramTcMaxTiles];
};

// one stage: three slices of w x kc BF16 values
__host__ __device__ constexpr size_t gram_tc_slice_bytes(int w, int kc) { return (size_t)w * kc * 2; }
__host__ __device__ constexpr size_t smem_gram_tc_bytes(int w, int kc)
{
    return 2 * 3 * gram_tc_slice_bytes(w, kc) + (size_t)w * 4 + 1024 + 256;
}

// 2^-e as a float for the column exponent e (2^e >= max |v|)
__device__ __forceinline__ float gram_scale(int e) { return __int_as_float((127 - e) << 23); }

// The three slices of v on the grid of exponent e, as BF16 bit patterns (the
// slice values have at most 8 significant bits, so truncating the FP32 bits
// is exact).
__device__ __forceinline__ void gram_slices(float v, int e, uint32_t (&q)[3])
{
    const float y = __fmul_rn(v, gram_scale(e)); // |y| <= 1, exact
    const float q0 = __fmul_rn(rintf(__fmul_rn(y, 128.f)), 0.0078125f);
    const float r1 = __fsub_rn(y, q0);
    const float q1 = __fmul_rn(rintf(__fmul_rn(r1, 32768.f)), 3.0517578125e-05f);
    const float r2 = __fsub_rn(r1, q1);
    const float q2 = __fmul_rn(rintf(__fmul_rn(r2, 8388608.f)), 1.1920928955078125e-07f);
    const float up = __int_as_float((127 + e) << 23); // back to absolute units (exact)
    q[0] = __float_as_uint(__fmul_rn(q0, up)) >> 16;
    q[1] = __float_as_uint(__fmul_rn(q1, up)) >> 16;
    q[2] = __float_as_uint(__fmul_rn(q2, up)) >> 16;
}

// Column exponents of Y below each level-(M-1) region, 2^e > max |Y| over the
// region's rows (e = 0 for an all-zero column): one CTA per region, threads
// along the columns (coalesced rows), eight rows in flight per thread.  A grid
// from the region-wide maximum keeps every group of the Gram exact (the slices
// stay within +-128 steps).
template <int RP>
__global__ void __launch_bounds__(256) k_gram_colexp(DevTree t, Work<float> w, int reg0)
{
    const int P = reg0 + blockIdx.x, Pl = blockIdx.x, b = blockIdx.y;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const int M = t.M, J = t.Jl[M - 1], UC = (M - 1) * RP;
    const int64_t r0 = t.leaf_off[(int64_t)P * J], r1 = t.leaf_off[(int64_t)P * J + J];
    const float *Yb = w.U + (size_t)b * w.U_stride;
    int8_t *ge = w.gexp + (size_t)b * w.gexp_stride + (size_t)Pl * UC;
    for (int x = threadIdx.x; x < UC; x += blockDim.x) {
        float m = 0.f;
#pragma unroll 8
        for (int64_t r = r0; r < r1; r++) m = fmaxf(m, fabsf(Yb[(size_t)r * UC + x]));
        ge[x] = (int8_t)(m > 0.f ? (int)((__float_as_uint(m) >> 23) & 0xff) - 126 : 0);
    }
}

template <int RP>
__global__ void __launch_bounds__(kGramTcThreads) k_leafgram_tc(DevTree t, Work<float> w, int reg0, GramTiles tiles)
{
    const int P = reg0 + blockIdx.x, Pl = blockIdx.x, b = blockIdx.z, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const GramTile tl = tiles.t[blockIdx.y];
    const int M = t.M, J = t.Jl[M - 1], UC = (M - 1) * RP, np = npairs(M - 1);
    const int KC = tl.kc, W = tl.w, u0 = tl.u0, N = tl.n;
    const uint32_t SBO = (uint32_t)(KC / 8) * 128u, LBO = 128u;
    const int64_t r0 = t.leaf_off[(int64_t)P * J], r1 = t.leaf_off[(int64_t)P * J + J];
    const float *Yb = w.U + (size_t)b * w.U_stride;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *stg = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const size_t SL = gram_tc_slice_bytes(W, KC); // one slice; a stage is 3 SL
    int *cexp = reinterpret_cast<int *>(stg + 6 * SL); // [W] column exponents
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, kGramTcCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init_fence();
        s_bad = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc_bf16(128, N);
    // sums of this thread's tile row (x = xa0 + tid) over the groups
    float acc[kGramTcN];
#pragma unroll
    for (int q = 0; q < kGramTcN; q++) acc[q] = 0.f;

    // the column exponents of the staged columns (k_gram_colexp, region-wide)
    {
        const int8_t *ge = w.gexp + (size_t)b * w.gexp_stride + (size_t)Pl * UC;
        for (int xx = tid; xx < W; xx += kGramTcThreads) cexp[xx] = (u0 + xx < UC) ? (int)ge[u0 + xx] : 0;
    }
    __syncthreads();
    bool bad = false;
    int gc = 0;     // chunks committed so far (all groups)
    int last = -1;  // index of the last committed chunk
    for (int64_t g0 = r0; g0 < r1 && !bad; g0 += kGramTcGroup) {
        const int64_t g1 = min(r1, g0 + (int64_t)kGramTcGroup);
        // the group's chunks
        const int nch = (int)((g1 - g0 + KC - 1) / KC);
        for (int c = 0; c < nch; c++, gc++) {
            const int s = gc & 1;
            if (gc >= 2 && !tc::mbar_wait(&mbar[s], (uint32_t)((gc - 2) >> 1) & 1u, kGramTcPolls)) bad = true;
            unsigned char *st = stg + (size_t)s * 3 * SL;
            const int64_t rb = g0 + (int64_t)c * KC;
            // lane (x % 8, pair of rows): a warp fills one 128-byte core matrix of each
            // slice per step; the loads of CB steps are issued before any is used
            const int ncm = (W / 8) * (KC / 8);
            constexpr int CB = 8;
            if (!bad)
                for (int cm0 = warp; cm0 < ncm; cm0 += 4 * CB) {
                    float v0[CB], v1[CB];
#pragma unroll
                    for (int k = 0; k < CB; k++) {
                        const int cm = cm0 + 4 * k;
                        const int xg = cm / (KC / 8), rg = cm % (KC / 8);
                        const int x = u0 + xg * 8 + (lane >> 2);
                        const int64_t r = rb + rg * 8 + (lane & 3) * 2;
                        const bool ok = cm < ncm && x < UC;
                        v0[k] = (ok && r < g1) ? Yb[(size_t)r * UC + x] : 0.f;
                        v1[k] = (ok && r + 1 < g1) ? Yb[(size_t)(r + 1) * UC + x] : 0.f;
                    }
#pragma unroll
                    for (int k = 0; k < CB; k++) {
                        const int cm = cm0 + 4 * k;
                        if (cm >= ncm) continue;
                        const int xg = cm / (KC / 8), rg = cm % (KC / 8);
                        const int e = cexp[xg * 8 + (lane >> 2)];
                        uint32_t a[3], bq[3];
                        gram_slices(v0[k], e, a);
                        gram_slices(v1[k], e, bq);
                        const size_t off =
                            (size_t)xg * SBO + (size_t)rg * LBO + (size_t)(lane >> 2) * 16 + (size_t)(lane & 3) * 4;
#pragma unroll
                        for (int q = 0; q < 3; q++)
                            *reinterpret_cast<uint32_t *>(st + q * SL + off) = a[q] | (bq[q] << 16);
                    }
                }
            tc::fence_proxy_async();
            if (__syncthreads_or(bad)) {
                bad = true;
                break;
            }
            if (tid == 0) {
                tc::fence_after_sync();
                uint32_t as[3], bs[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    as[k] = tc::smem_addr(st + k * SL) + (uint32_t)((tl.xa0 - u0) / 8) * SBO;
                    bs[k] = tc::smem_addr(st + k * SL) + (uint32_t)((tl.xb0 - u0) / 8) * SBO;
                }
                for (int ks = 0; ks < KC / 16; ks++) {
                    const uint32_t ko = (uint32_t)ks * 2u * LBO; // two core matrices along K per step
                    const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u; // a new group overwrites D
                    auto mma = [&](int dk, int sa, int sb, uint32_t accum) {
                        tc::mma_bf16(tmem + 64u * dk, tc::smem_desc(as[sa] + ko, LBO, SBO),
                                     tc::smem_desc(bs[sb] + ko, LBO, SBO), idesc, accum);
                    };
                    mma(0, 0, 0, first);
                    mma(1, 0, 1, first);
                    mma(1, 1, 0, 1u);
                    mma(2, 0, 2, first);
                    mma(2, 1, 1, 1u);
                    mma(2, 2, 0, 1u);
                }
                tc::mma_commit(&mbar[s]);
            }
            last = gc;
        }
        if (bad) break;
        // the group's sums: wait for its last commit, then D0 + D1 + D2 (exact
        // FP32 values) in float pairs, rounded once, into the running sums
        bad = !tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u, kGramTcPolls);
        tc::fence_after_sync();
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
#pragma unroll
        for (int cc = 0; cc < kGramTcN; cc += 16) {
            float d0[16], d1[16], d2[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc;
            tc::tmem_ld16(ta, d0);
            tc::tmem_ld16(ta + 64u, d1);
            tc::tmem_ld16(ta + 128u, d2);
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const ff s = ff_add_f(two_sum(d0[q], d1[q]), d2[q]);
                acc[cc + q] = __fadd_rn(acc[cc + q], __fadd_rn(s.hi, s.lo));
            }
        }
        // the next group's first MMAs overwrite D only after every warp has read it
        tc::fence_before_sync();
        __syncthreads();
    }
    if (__syncthreads_or(bad)) s_bad = 1;
    __syncthreads();
    if (s_bad) {
        // a wait gave up: report it, let the MMAs in flight drain (bounded),
        // then free the tensor memory below
        if (tid == 0) {
            w.status[b] = ST_ETIMEDOUT;
            if (last >= 0) (void)tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u, kGramTcPolls);
        }
    } else {
        // tile row i = tid, output row x = xa0 + i: whole rows of the packed blocks
        float *out = w.Ain + (size_t)b * w.Ain_stride + (size_t)Pl * np * RP * RP;
        const int x = tl.xa0 + tid;
        if (x >= tl.rowlo && x < UC) {
            const int k = x / RP, ii = x % RP;
#pragma unroll
            for (int part = 0; part < kGramTcN / RP; part++) {
                const int xb = tl.xb0 + part * RP, l = xb / RP;
                if (part * RP >= N || xb >= UC || k > l) continue;
                float4 *dst = reinterpret_cast<float4 *>(out + (size_t)pidx(k + 1, l + 1) * RP * RP + (size_t)ii * RP);
#pragma unroll
                for (int q = 0; q < RP / 4; q++) {
                    const int c = part * RP + 4 * q;
                    dst[q] = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kGramTcCols);
    if (blockIdx.y == 0) {
        // the leaves' w and (d, u) summed into the region
        const double *lw = w.leaf_w + (size_t)b * w.leafw_stride;
        const double *ldu = w.leaf_du + (size_t)b * w.leafdu_stride;
        double *wo = w.Ain_w + (size_t)b * w.Ainw_stride + (size_t)Pl * UC;
        for (int col = tid; col < UC; col += kGramTcThreads) {
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

// The tile list of a Gram of UC columns (host side): row chunks of 128, each
// with its columns [128 c, UC) in tiles of 64; the staged range and the rows
// per chunk chosen so that the two stages stay under ~100 KB (two CTAs per SM).
__host__ inline int gram_tc_tiles(int UC, GramTile *out, int cap)
{
    int n = 0;
    for (int c = 0; 128 * c < UC; c++) {
        const int rowlo = 128 * c;
        const int xa0 = UC >= 128 ? (rowlo < UC - 128 ? rowlo : UC - 128) : 0;
        for (int xb0 = rowlo; xb0 < UC; xb0 += kGramTcN) {
            GramTile g;
            g.xa0 = (int16_t)xa0;
            g.xb0 = (int16_t)xb0;
            g.n = (int16_t)(UC - xb0 < kGramTcN ? UC - xb0 : kGramTcN);
            g.rowlo = (int16_t)rowlo;
            const int lo = xa0 < xb0 ? xa0 : xb0;
            const int hi = (xa0 + 128 > xb0 + g.n) ? xa0 + 128 : xb0 + g.n;
            g.u0 = (int16_t)lo;
            g.w = (int16_t)(hi - lo);
            int kc = 32;
            while (kc > 16 && smem_gram_tc_bytes(g.w, kc) > (size_t)100 * 1024) kc /= 2;
            g.kc = (int16_t)kc;
            g.pad = 0;
            if (n < cap) out[n] = g;
            n++;
        }
    }
    return n;
}

} // namespace mra
