// mra_gram_tc.cuh -- the leaf Gram blocks of the mixed mode on the tensor
// cores (tcgen05, kind::tf32, accumulation in tensor memory).
//
// For a region P of level M-1 the upward pass starts from
//     A = sum over the leaves c of P of Y_c' Y_c = Y_P' Y_P,
// Y_P the rows of Y = L^{-1} U of all observations below P (FP32, row-major,
// UC = (M-1) RP columns); the packed upper blocks (k <= l) of this UC x UC
// matrix are the ATilde blocks the leaves pass to their parent (App. B).
//
// Tensor-core form: D = T T' with T = Y_P' (UC rows, the region's observations
// along K).  A CTA of 128 threads computes a 128 x N tile of D: rows
// [xa0, xa0 + 128) and columns [xb0, xb0 + N), N <= 256, for one region
// (grid.x), one tile (grid.y) and one theta (grid.z).  Row chunk c of the
// output owns rows [128 c, 128 c + 128) (the MMA rows start at
// min(128 c, UC - 128) so that every MMA has M = 128); its columns run from
// 128 c to UC (the upper triangle), in pieces of at most 256.
//
// Precision: each FP32 value v is split into TF32 parts hi = tf32(v) and
// lo = tf32(v - hi) (22 significant bits together), and D accumulates
// hi hi' + hi lo' + lo hi' (the 3xTF32 product: every product exact in the
// tensor cores, the dropped lo lo' term below 2^-21 of |v1 v2|) in FP32 in
// tensor memory.
//
// Pipeline per CTA: the region's rows in groups of KC (32, 16 or 8) rows;
// all 128 threads load a group (plain coalesced loads), split it and store
// both parts into one of two shared-memory stages in the no-swizzle K-major
// core-matrix layout (tc_sm100.cuh), then thread 0 issues the MMAs of the
// group and commits them to the stage's mbarrier, which the threads wait on
// (bounded) before they refill that stage two groups later.  After the last
// group the four warps read their 32 TMEM lanes (tile rows) back, 32 columns
// at a time, and write whole rows of the packed 32 x 32 (or 16 x 16) blocks.
#pragma once
#include "tc_sm100.cuh"

namespace mra {

constexpr int kGramTcThreads = 128;
constexpr uint32_t kGramTcCols = 256; // TMEM columns per CTA (N <= 256)
constexpr uint32_t kGramTcPolls = 1u << 24; // mbarrier polls before a wait gives up (~seconds)
enum { ST_ETIMEDOUT = 5 };

// One output tile of the Gram (host-built list, the same for every region).
struct GramTile {
    int16_t xa0, xb0;  // first row (MMA rows: 128 of them) and first column
    int16_t n;         // columns (a multiple of 16, <= 256)
    int16_t rowlo;     // rows below this one are owned by an earlier chunk
    int16_t u0, w;     // staged columns of T: [u0, u0 + w)
    int16_t kc, pad;   // rows per staged group
};

constexpr int kGramTcMaxTiles = 12;
struct GramTiles {
    int n;
    GramTile t[kGramTcMaxTiles];
};

__host__ __device__ constexpr size_t gram_tc_stage_bytes(int w, int kc) { return (size_t)w * kc * 4; }
__host__ __device__ constexpr size_t smem_gram_tc_bytes(int w, int kc) { return 4 * gram_tc_stage_bytes(w, kc) + 1024; }

template <int RP>
__global__ void __launch_bounds__(kGramTcThreads) k_leafgram_tc(DevTree t, Work<float> w, int reg0, GramTiles tiles)
{
    const int P = reg0 + blockIdx.x, Pl = blockIdx.x, b = blockIdx.z, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const GramTile tl = tiles.t[blockIdx.y];
    const int M = t.M, J = t.J, UC = (M - 1) * RP, np = npairs(M - 1);
    const int KC = tl.kc, W = tl.w, u0 = tl.u0;
    const uint32_t SBO = (uint32_t)(KC / 4) * 128u, LBO = 128u;
    const int64_t r0 = t.leaf_off[(int64_t)P * J], r1 = t.leaf_off[(int64_t)P * J + J];
    const float *Yb = w.U + (size_t)b * w.U_stride;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stage s: hi part at 2 s, lo part at 2 s + 1
    unsigned char *stg = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const size_t SB = gram_tc_stage_bytes(W, KC);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    // (written only after the last pipeline barrier; read after the next one)

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
    const uint32_t idesc = tc::idesc_tf32(128, tl.n);
    const int ngroups = (int)((r1 - r0 + KC - 1) / KC);
    // every exit from the pipeline is uniform: a thread whose bounded wait
    // gave up says so at the next barrier (__syncthreads_or), and all stop
    bool bad = false;
    int last = -1; // the last group whose MMAs were committed
    for (int g = 0; g < ngroups; g++) {
        const int s = g & 1;
        if (g >= 2 && !tc::mbar_wait(&mbar[s], (uint32_t)((g - 2) >> 1) & 1u, kGramTcPolls)) bad = true;
        unsigned char *hi = stg + (size_t)(2 * s) * SB, *lo = hi + SB;
        const int64_t rb = r0 + (int64_t)g * KC;
        // lane (x % 8, r % 4): a warp fills one 128-byte core matrix per step
        const int ncm = (W / 8) * (KC / 4);
        if (!bad)
            for (int cm = warp; cm < ncm; cm += kGramTcThreads / 32) {
                const int xg = cm / (KC / 4), rg = cm % (KC / 4);
                const int xx = xg * 8 + (lane >> 2), rr = rg * 4 + (lane & 3);
                const int x = u0 + xx;
                const int64_t r = rb + rr;
                const float v = (r < r1 && x < UC) ? Yb[(size_t)r * UC + x] : 0.f;
                const float h = tc::to_tf32(v);
                const float l = tc::to_tf32(__fsub_rn(v, h));
                const size_t off =
                    (size_t)xg * SBO + (size_t)rg * LBO + (size_t)(lane >> 2) * 16 + (size_t)(lane & 3) * 4;
                *reinterpret_cast<float *>(hi + off) = h;
                *reinterpret_cast<float *>(lo + off) = l;
            }
        tc::fence_proxy_async();
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_addr(hi) + (uint32_t)((tl.xa0 - u0) / 8) * SBO;
            const uint32_t al = tc::smem_addr(lo) + (uint32_t)((tl.xa0 - u0) / 8) * SBO;
            const uint32_t bh = tc::smem_addr(hi) + (uint32_t)((tl.xb0 - u0) / 8) * SBO;
            const uint32_t bl = tc::smem_addr(lo) + (uint32_t)((tl.xb0 - u0) / 8) * SBO;
            for (int ks = 0; ks < KC / 8; ks++) {
                const uint32_t ko = (uint32_t)ks * 2u * LBO; // two core matrices along K per step
                tc::mma_tf32(tmem, tc::smem_desc(ah + ko, LBO, SBO), tc::smem_desc(bh + ko, LBO, SBO), idesc,
                             (g > 0 || ks > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, tc::smem_desc(ah + ko, LBO, SBO), tc::smem_desc(bl + ko, LBO, SBO), idesc, 1u);
                tc::mma_tf32(tmem, tc::smem_desc(al + ko, LBO, SBO), tc::smem_desc(bh + ko, LBO, SBO), idesc, 1u);
            }
            tc::mma_commit(&mbar[s]);
        }
        last = g;
    }
    // the last commit completes after every MMA of the CTA
    if (!bad && last >= 0) bad = !tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u, kGramTcPolls);
    tc::fence_after_sync();
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
        // tile row i = 32 warp + lane, output row x = xa0 + i
        float *out = w.Ain + (size_t)b * w.Ain_stride + (size_t)Pl * np * RP * RP;
        const int i = 32 * warp + lane, x = tl.xa0 + i;
        const bool mine = x >= tl.rowlo && x < UC;
        const int k = x / RP, ii = x % RP;
        for (int cc = 0; cc < tl.n; cc += 32) {
            float v[32];
            if (ngroups > 0) {
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
            } else {
#pragma unroll
                for (int q = 0; q < 32; q++) v[q] = 0.f;
            }
            if (!mine) continue;
#pragma unroll
            for (int part = 0; part < 32 / RP; part++) {
                const int xb = tl.xb0 + cc + part * RP, l = xb / RP;
                if (xb >= UC || k > l) continue;
                float4 *dst = reinterpret_cast<float4 *>(out + (size_t)pidx(k + 1, l + 1) * RP * RP + (size_t)ii * RP);
#pragma unroll
                for (int q = 0; q < RP / 4; q++)
                    dst[q] = make_float4(v[part * RP + 4 * q], v[part * RP + 4 * q + 1], v[part * RP + 4 * q + 2],
                                         v[part * RP + 4 * q + 3]);
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
// with its columns [128 c, UC) in pieces of at most 256; the staged range and
// the rows per group chosen so that two stages of both parts fit twice per SM.
__host__ inline int gram_tc_tiles(int UC, GramTile *out, int cap)
{
    int n = 0;
    for (int c = 0; 128 * c < UC; c++) {
        const int rowlo = 128 * c;
        const int xa0 = UC >= 128 ? (rowlo < UC - 128 ? rowlo : UC - 128) : 0;
        for (int xb0 = rowlo; xb0 < UC; xb0 += 256) {
            GramTile g;
            g.xa0 = (int16_t)xa0;
            g.xb0 = (int16_t)xb0;
            g.n = (int16_t)(UC - xb0 < 256 ? UC - xb0 : 256);
            g.rowlo = (int16_t)rowlo;
            const int lo = xa0 < xb0 ? xa0 : xb0;
            const int hi = (xa0 + 128 > xb0 + g.n) ? xa0 + 128 : xb0 + g.n;
            g.u0 = (int16_t)lo;
            g.w = (int16_t)(hi - lo);
            int kc = 32;
            while (kc > 8 && smem_gram_tc_bytes(g.w, kc) > (size_t)112 * 1024) kc /= 2;
            g.kc = (int16_t)kc;
            g.pad = 0;
            if (n < cap) out[n] = g;
            n++;
        }
    }
    return n;
}

} // namespace mra
