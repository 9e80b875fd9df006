// mra_launch.cuh -- host launchers of the MRA kernels, instantiated per
// precision in k_f64.cu and k_f32.cu.
#pragma once
#include <algorithm>
#include <cstring>

#include "mra_kernels.cuh"
#include "mra_gram_tc.cuh"
#include "mra_leafbasis_tc.cuh"

namespace mra {

// Raise the dynamic shared-memory limit of a kernel once per process.
template <typename K>
static int set_smem(K kernel, size_t bytes, size_t *done)
{
    if (bytes <= *done) return 0;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    *done = bytes;
    return 0;
}

// Deep levels run the streamed prior and upward pass (their footprints grow by
// one block per level instead of two)
template <typename T, int RP> bool prior_streams(int m) { return smem_prior_bytes<T, RP>(m, 1) > kSmemMax; }
template <typename T, int RP> bool up_streams(int m) { return smem_up_bytes<T, RP>(m) > kSmemMax; }
template <typename T, int RP> size_t smem_prior(int m)
{
    if (prior_streams<T, RP>(m)) return smem_prior_stream_bytes<T, RP, kPriorStreamBlocks>(m);
    return smem_prior_bytes<T, RP>(m, prior_stages<T, RP>(m));
}
template <typename T, int RP> size_t smem_leafbasis_cfg(int M, int rows, int stages)
{
    if (rows == kStreamRows) return smem_leafbasis_stream_bytes<T, RP, kStreamRows, kStreamBlocks>(M);
    return smem_leafbasis_bytes<T, RP>(M, stages, rows);
}
template <typename T, int RP> size_t smem_leafbasis(int M)
{
    return smem_leafbasis_bytes<T, RP>(M, leafbasis_stages<T, RP>(M));
}
template <typename T, int RP> size_t smem_leafpost_small(int M, int nmax) { return smem_leafpost_bytes<T, RP>(M, nmax); }
template <typename T, int RP> size_t smem_up(int m)
{
    return up_streams<T, RP>(m) ? smem_up_stream_bytes<T, RP, kUpStreamBlocks>(m) : smem_up_bytes<T, RP>(m);
}
// large-leaf assembly of deep trees (FP32 storage): U rows in column parts
template <typename T, int RP> bool big_assemble_parts(int M)
{
    return sizeof(T) == 4 && smem_big_assemble_bytes<T, RP>(M) > kSmemMax;
}
template <typename T, int RP> size_t smem_leafgram(int M) { return smem_leafgram_bytes<T, RP>(M); }
template <typename T, int RP> size_t smem_big(int M)
{
    size_t a = big_assemble_parts<T, RP>(M) ? smem_big_assemble_parts_bytes<T, RP, kBigAssembleParts>(M)
                                            : smem_big_assemble_bytes<T, RP>(M);
    size_t p = smem_big_potrf_bytes<T, RP>(M);
    return a > p ? a : p;
}

// How level m of the prior stages its ancestor blocks: 1 or 2 buffers of a
// whole level's blocks (the next level prefetched into the second), or 3: the
// streamed kernel, two blocks at a time (kPriorPairBlocks).  stages_req 1, 2
// or 3 forces that form (2 only where it fits); 0 decides by occupancy: the
// streamed kernel where it fits more CTAs per SM than one buffer and the
// level has more CTAs than one wave of the one-buffer kernel (its extra
// barriers cost less than the extra CTAs hide), else one buffer where that
// fits more CTAs per SM and saves a wave, else two where they fit.  All three
// sum the same terms in the same order.
constexpr int kPriorPairBlocks = 2;
template <typename T, int RP>
static int prior_mode_for(int m, long long ctas, int stages_req, size_t *done, size_t *done_p)
{
    const int fit = prior_stages<T, RP>(m);
    if (stages_req == 1 || stages_req == 3) return stages_req;
    if (stages_req == 2) return fit;
    // decided once per (level, CTA count): the first pass runs uncaptured, so
    // the queries below stay out of graph capture
    static long long seen_ctas[MRA_MAXM + 1] = {0};
    static int seen_mode[MRA_MAXM + 1] = {0};
    if (seen_ctas[m] == ctas && seen_mode[m] > 0) return seen_mode[m];
    const size_t b3 = smem_prior_stream_bytes<T, RP, kPriorPairBlocks>(m);
    if (set_smem(k_prior<T, RP>, smem_prior_bytes<T, RP>(m, fit), done) ||
        set_smem(k_prior<T, RP, kPriorPairBlocks>, b3, done_p))
        return fit;
    int dev = 0, sms = 0, o1 = 0, o2 = 0, o3 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_prior<T, RP>, NT, smem_prior_bytes<T, RP>(m, 1)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_prior<T, RP>, NT, smem_prior_bytes<T, RP>(m, fit)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o3, k_prior<T, RP, kPriorPairBlocks>, NT, b3) != cudaSuccess ||
        sms <= 0 || o1 <= 0 || o2 <= 0) {
        cudaGetLastError();
        return fit;
    }
    int mode;
    if (o3 > o1 && ctas > (long long)sms * o1) {
        mode = 3;
    } else {
        const long long w1 = (ctas + (long long)sms * o1 - 1) / ((long long)sms * o1);
        const long long w2 = (ctas + (long long)sms * o2 - 1) / ((long long)sms * o2);
        mode = (fit == 1 || w1 < w2) ? 1 : 2;
    }
    seen_ctas[m] = ctas;
    seen_mode[m] = mode;
    return mode;
}

template <typename T, int RP>
int launch_prior(const DevTree &t, const Work<T> &w, int m, int B, int stages_req, void *stream)
{
    static size_t done = 0, done_s = 0, done_p = 0;
    const long long nreg = (long long)(t.lvl_off[m + 1] - t.lvl_off[m]);
    if (prior_streams<T, RP>(m)) {
        const size_t sm = smem_prior_stream_bytes<T, RP, kPriorStreamBlocks>(m);
        if (int e = set_smem(k_prior<T, RP, kPriorStreamBlocks>, sm, &done_s)) return e;
        dim3 grid((unsigned)nreg, (unsigned)B);
        k_prior<T, RP, kPriorStreamBlocks><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, m, 1);
        return (int)cudaGetLastError();
    }
    const int mode = prior_mode_for<T, RP>(m, nreg * B, stages_req, &done, &done_p);
    dim3 grid((unsigned)nreg, (unsigned)B);
    if (mode == 3) {
        const size_t sm = smem_prior_stream_bytes<T, RP, kPriorPairBlocks>(m);
        if (int e = set_smem(k_prior<T, RP, kPriorPairBlocks>, sm, &done_p)) return e;
        k_prior<T, RP, kPriorPairBlocks><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, m, 1);
        return (int)cudaGetLastError();
    }
    const size_t sm = smem_prior_bytes<T, RP>(m, mode);
    if (int e = set_smem(k_prior<T, RP>, sm, &done)) return e;
    k_prior<T, RP><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, m, mode);
    return (int)cudaGetLastError();
}

template <typename T, int RP, int CH>
static int launch_leafbasis_ch(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int stages, int B,
                               void *stream)
{
    static size_t done = 0;
    if (stages <= 0) stages = leafbasis_stages<T, RP>(t.M, CH);
    const size_t sm = smem_leafbasis_bytes<T, RP>(t.M, stages, CH);
    if (int e = set_smem(k_leafbasis<T, RP, CH>, sm, &done)) return e;
    dim3 grid((unsigned)nchunks, (unsigned)B);
    k_leafbasis<T, RP, CH><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, chunks, stages);
    return (int)cudaGetLastError();
}

// rows: observation rows per chunk (32, or 64 in FP32; 16: the streaming
// kernel for deep trees, stages ignored); stages: 1 or 2 stages of ancestor
// blocks, 0 = two while two CTAs per SM still fit
template <typename T, int RP>
int launch_leafbasis(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int rows, int stages,
                     int B, void *stream)
{
    if (nchunks == 0) return 0;
    if (rows == kStreamRows) {
        static size_t done = 0;
        const size_t sm = smem_leafbasis_stream_bytes<T, RP, kStreamRows, kStreamBlocks>(t.M);
        if (int e = set_smem(k_leafbasis_stream<T, RP, kStreamRows, kStreamBlocks>, sm, &done)) return e;
        dim3 grid((unsigned)nchunks, (unsigned)B);
        k_leafbasis_stream<T, RP, kStreamRows, kStreamBlocks><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, chunks);
        return (int)cudaGetLastError();
    }
    if constexpr (sizeof(T) == 4)
        if (rows == 64) return launch_leafbasis_ch<T, RP, 64>(t, w, chunks, nchunks, stages, B, stream);
    return launch_leafbasis_ch<T, RP, 32>(t, w, chunks, nchunks, stages, B, stream);
}

// chunks of at most rows / 2 observation rows (the regions' tails of a 32- or
// 64-row chunk list) in the kernel of half the rows: each output sums the same
// terms in the same order, so U is the same bit for bit
template <typename T, int RP>
int launch_leafbasis_half(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int rows, int stages,
                          int B, void *stream)
{
    if (nchunks == 0) return 0;
    if constexpr (sizeof(T) == 4)
        if (rows == 64) return launch_leafbasis_ch<T, RP, 32>(t, w, chunks, nchunks, stages, B, stream);
    if (rows != 32) return (int)cudaErrorInvalidValue;
    return launch_leafbasis_ch<T, RP, 16>(t, w, chunks, nchunks, stages, B, stream);
}

// mixed mode: the leaf basis with the remainder products on the tensor cores
// (128-row chunks); EINVAL where the exactness bound does not hold
template <typename T, int RP>
int launch_leafbasis_tc(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int B, void *stream)
{
    if constexpr (sizeof(T) == 4) {
        if (nchunks == 0) return 0;
        if ((t.M - 2) * RP > kLbTcMaxK) return (int)cudaErrorInvalidValue;
        static size_t done = 0;
        const size_t sm = smem_leafbasis_tc_bytes<RP>();
        if (int e = set_smem(k_leafbasis_tc<RP>, sm, &done)) return e;
        dim3 grid((unsigned)nchunks, (unsigned)B);
        k_leafbasis_tc<RP><<<grid, kLbTcThreads, sm, (cudaStream_t)stream>>>(t, w, chunks);
        return (int)cudaGetLastError();
    } else {
        return (int)cudaErrorInvalidValue;
    }
}

template <typename T, int RP, int NMAX>
static int launch_leafpost_n(const DevTree &t, const Work<T> &w, const int64_t *leaves, int nleaves, int B,
                             unsigned *queue, void *stream)
{
    const size_t sm = smem_leafpost_bytes<T, RP>(t.M, NMAX);
    cudaStream_t s = (cudaStream_t)stream;
    if (!queue) {
        static size_t done = 0;
        if (int e = set_smem(k_leafpost_small<T, RP, NMAX>, sm, &done)) return e;
        dim3 grid((unsigned)nleaves, (unsigned)B);
        k_leafpost_small<T, RP, NMAX><<<grid, NT, sm, s>>>(t, w, leaves);
        return (int)cudaGetLastError();
    }
    // persistent grid: the CTAs that fit on the GPU at once (per theta), at
    // most one per leaf
    static size_t done_q = 0;
    static int per_sm = 0, sms = 0;
    if (int e = set_smem(k_leafpost_queue<T, RP, NMAX>, sm, &done_q)) return e;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leafpost_queue<T, RP, NMAX>, NT, sm);
        if (per_sm < 1) per_sm = 1;
    }
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned) * (size_t)B, s);
    if (e != cudaSuccess) return (int)e;
    const int per_theta = std::max(1, std::min(nleaves, sms * per_sm / std::max(B, 1)));
    dim3 grid((unsigned)per_theta, (unsigned)B);
    k_leafpost_queue<T, RP, NMAX><<<grid, NT, sm, s>>>(t, w, leaves, nleaves, queue);
    return (int)cudaGetLastError();
}

// nmax: a bucket cap (32, 40, 48 or 64); the leaves of the list have at most
// nmax observations.  queue: null for one CTA per leaf, else B zeroed counters
// for the persistent work-queue kernel.  The 40 cap has its own kernel at
// RP = 32 (its Y = L^{-1} U tile does not divide at RP = 16, where the 48
// kernel takes it).
template <typename T, int RP>
int launch_leafpost_small(const DevTree &t, const Work<T> &w, const int64_t *leaves, int nleaves, int nmax,
                          int B, unsigned *queue, void *stream)
{
    if (nleaves == 0) return 0;
    if (nmax <= 32) return launch_leafpost_n<T, RP, 32>(t, w, leaves, nleaves, B, queue, stream);
    if constexpr (RP == 32)
        if (nmax <= 40) return launch_leafpost_n<T, RP, 40>(t, w, leaves, nleaves, B, queue, stream);
    if (nmax <= 48) return launch_leafpost_n<T, RP, 48>(t, w, leaves, nleaves, B, queue, stream);
    return launch_leafpost_n<T, RP, 64>(t, w, leaves, nleaves, B, queue, stream);
}

template <typename T, int RP>
int launch_big(const DevTree &t, const Work<T> &w, int phase, const BigLeaf *leaves, const BigTile *items,
               int nitems, int k, int B, void *stream)
{
    static size_t done_a = 0, done_p = 0, done_t = 0, done_u = 0;
    if (nitems == 0) return 0;
    dim3 grid((unsigned)nitems, (unsigned)B);
    cudaStream_t s = (cudaStream_t)stream;
    size_t sm;
    switch (phase) {
    case BIG_ASSEMBLE:
        if constexpr (sizeof(T) == 4) {
            if (big_assemble_parts<T, RP>(t.M)) {
                static size_t done_ap = 0;
                sm = smem_big_assemble_parts_bytes<T, RP, kBigAssembleParts>(t.M);
                if (int e = set_smem(k_big_assemble<T, RP, kBigAssembleParts>, sm, &done_ap)) return e;
                k_big_assemble<T, RP, kBigAssembleParts><<<grid, NT, sm, s>>>(t, w, leaves, items);
                break;
            }
        }
        sm = smem_big_assemble_bytes<T, RP>(t.M);
        if (int e = set_smem(k_big_assemble<T, RP>, sm, &done_a)) return e;
        k_big_assemble<T, RP><<<grid, NT, sm, s>>>(t, w, leaves, items);
        break;
    case BIG_POTRF:
        sm = smem_big_potrf_bytes<T, RP>(t.M);
        if (int e = set_smem(k_big_potrf<T, RP>, sm, &done_p)) return e;
        k_big_potrf<T, RP><<<grid, NT, sm, s>>>(t, w, leaves, items, k);
        break;
    case BIG_TRSM:
        sm = smem_big_trsm_bytes<T, RP>();
        if (int e = set_smem(k_big_trsm<T, RP>, sm, &done_t)) return e;
        k_big_trsm<T, RP><<<grid, NT, sm, s>>>(t, w, leaves, items, k);
        break;
    case BIG_UPDATE:
        sm = smem_big_update_bytes<T, RP>();
        if (int e = set_smem(k_big_update<T, RP>, sm, &done_u)) return e;
        k_big_update<T, RP><<<grid, NT, sm, s>>>(t, w, leaves, items, k);
        break;
    default:
        k_big_finish<T, RP><<<grid, NT, 0, s>>>(t, w, leaves);
        break;
    }
    return (int)cudaGetLastError();
}

// tensor_cores (mixed modes): the exact tensor-core Gram (after launch_gram_colexp)
template <typename T, int RP>
int launch_leafgram(const DevTree &t, const Work<T> &w, int reg0, int nP, int B, bool tensor_cores, void *stream)
{
    if constexpr (sizeof(T) == 4) {
      if (tensor_cores) {
        // mixed mode: tensor cores, exact BF16-slice sums (mra_gram_tc.cuh)
        static size_t done_tc = 0;
        GramTiles tl;
        memset(&tl, 0, sizeof(tl));
        tl.n = gram_tc_tiles((t.M - 1) * RP, tl.t, kGramTcMaxTiles);
        if (tl.n > kGramTcMaxTiles) return (int)cudaErrorInvalidConfiguration;
        size_t sm = (size_t)80 * 1024; // at most two CTAs per SM: their TMEM (2 x 256 columns) always fits
        for (int k = 0; k < tl.n; k++) sm = std::max(sm, smem_gram_tc_bytes(tl.t[k].w, tl.t[k].kc));
        if (int e = set_smem(k_leafgram_tc<RP>, sm, &done_tc)) return e;
        dim3 grid((unsigned)nP, (unsigned)tl.n, (unsigned)B);
        k_leafgram_tc<RP><<<grid, kGramTcThreads, sm, (cudaStream_t)stream>>>(t, w, reg0, tl);
        return (int)cudaGetLastError();
      }
    }
    {
        static size_t done = 0;
        const size_t sm = smem_leafgram_bytes<T, RP>(t.M);
        if (int e = set_smem(k_leafgram<T, RP>, sm, &done)) return e;
        const int nt = ((t.M - 1) * RP + kGramTile - 1) / kGramTile;
        dim3 grid((unsigned)nP, (unsigned)(nt * (nt + 1) / 2), (unsigned)B);
        k_leafgram<T, RP><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, reg0);
        return (int)cudaGetLastError();
    }
}

// mixed mode: column exponents of Y per level-(M-1) region for the exact Gram
template <typename T, int RP>
int launch_gram_colexp(const DevTree &t, const Work<T> &w, int reg0, int nP, int B, void *stream)
{
    if constexpr (sizeof(T) == 4) {
        dim3 grid((unsigned)nP, (unsigned)B);
        k_gram_colexp<RP><<<grid, 256, 0, (cudaStream_t)stream>>>(t, w, reg0);
        return (int)cudaGetLastError();
    } else {
        return 0;
    }
}

// regions reg0 .. reg0 + nreg - 1 of level m (nreg < 0: the whole level)
template <typename T, int RP>
int launch_up(const DevTree &t, const Work<T> &w, int m, int reg0, int nreg, int B, void *stream)
{
    static size_t done = 0, done_s = 0;
    if (nreg < 0) nreg = (int)(t.lvl_off[m + 1] - t.lvl_off[m]);
    dim3 grid((unsigned)nreg, (unsigned)B);
    if (up_streams<T, RP>(m)) {
        const size_t sm = smem_up_stream_bytes<T, RP, kUpStreamBlocks>(m);
        if (int e = set_smem(k_up<T, RP, kUpStreamBlocks>, sm, &done_s)) return e;
        k_up<T, RP, kUpStreamBlocks><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, m, reg0);
        return (int)cudaGetLastError();
    }
    const size_t sm = smem_up_bytes<T, RP>(m);
    if (int e = set_smem(k_up<T, RP>, sm, &done)) return e;
    k_up<T, RP><<<grid, NT, sm, (cudaStream_t)stream>>>(t, w, m, reg0);
    return (int)cudaGetLastError();
}

template <typename T, int RP>
int launch_root_single(const DevTree &t, const Work<T> &w, int B, void *stream)
{
    k_root_single<T><<<(unsigned)B, 32, 0, (cudaStream_t)stream>>>(t, w);
    return (int)cudaGetLastError();
}

// Prediction: the downward pass (one level) and the per-point kernel.
template <int RP>
int launch_down(const DevTree &t, const double *keep, size_t stride, double *xi, int m, void *stream)
{
    const unsigned nreg = (unsigned)(t.lvl_off[m + 1] - t.lvl_off[m]);
    k_down<RP><<<nreg, 32, 0, (cudaStream_t)stream>>>(t, keep, stride, xi, m);
    return (int)cudaGetLastError();
}

template <typename T, int RP>
int launch_predict(const DevTree &t, const Work<T> &w, const PredArgs &q, void *stream)
{
    if (q.np <= 0) return 0;
    static size_t done = 0;
    const size_t sm = predict_warp_doubles(t.M, RP, q.nl) * sizeof(double) * (size_t)q.wpb;
    if (int e = set_smem(k_predict<T, RP>, sm, &done)) return e;
    const unsigned nb = (unsigned)((q.np + q.wpb - 1) / q.wpb);
    k_predict<T, RP><<<nb, 32 * q.wpb, sm, (cudaStream_t)stream>>>(t, w, q);
    return (int)cudaGetLastError();
}

#define MRA_INSTANTIATE_DOWN(RP) \
    template int launch_down<RP>(const DevTree &, const double *, size_t, double *, int, void *);

#define MRA_INSTANTIATE(T, RP)                                                                              \
    template size_t smem_prior<T, RP>(int);                                                                 \
    template size_t smem_leafbasis<T, RP>(int);                                                             \
    template size_t smem_leafbasis_cfg<T, RP>(int, int, int);                                               \
    template size_t smem_leafpost_small<T, RP>(int, int);                                                   \
    template size_t smem_up<T, RP>(int);                                                                    \
    template size_t smem_leafgram<T, RP>(int);                                                              \
    template int launch_prior<T, RP>(const DevTree &, const Work<T> &, int, int, int, void *);              \
    template int launch_leafbasis<T, RP>(const DevTree &, const Work<T> &, const Chunk *, int, int, int, int, \
                                         void *);                                                           \
    template int launch_leafbasis_tc<T, RP>(const DevTree &, const Work<T> &, const Chunk *, int, int, void *); \
    template int launch_leafbasis_half<T, RP>(const DevTree &, const Work<T> &, const Chunk *, int, int, int,  \
                                              int, void *);                                                 \
    template int launch_leafpost_small<T, RP>(const DevTree &, const Work<T> &, const int64_t *, int, int,   \
                                              int, unsigned *, void *);                                     \
    template size_t smem_big<T, RP>(int);                                                                   \
    template int launch_big<T, RP>(const DevTree &, const Work<T> &, int, const BigLeaf *, const BigTile *, \
                                   int, int, int, void *);                                                  \
    template int launch_leafgram<T, RP>(const DevTree &, const Work<T> &, int, int, int, bool, void *);     \
    template int launch_gram_colexp<T, RP>(const DevTree &, const Work<T> &, int, int, int, void *);        \
    template int launch_up<T, RP>(const DevTree &, const Work<T> &, int, int, int, int, void *);            \
    template int launch_root_single<T, RP>(const DevTree &, const Work<T> &, int, void *);                   \
    template int launch_predict<T, RP>(const DevTree &, const Work<T> &, const PredArgs &, void *);

} // namespace mra
