// mra_internal.h -- device-side data layout shared by the kernels and the host
// orchestration of libmra.  Not part of the public ABI (include/mra.h).
//
// Layout in HBM (one context):
//   knots      kx, ky [n_nonleaf][RP]        regions of levels 1..M-1, padded to RP
//   corners    cx, cy [n_nonleaf]            lower-left corner of each such region
//   obs        sx, sy, sz [n_used]           leaf order
//   leaf_off   [n_leaf + 1]
// Per theta (stride-separated copies for a batch of B theta), storage type T:
//   prior      level m, region i: m blocks of RP x RP, each stored column-major
//              (element (j, t) at t*RP + j): What^1..What^{m-1}, then
//              Linv = L^{-1}, L the Cholesky factor of W^m = C_m(Q, Q).
//   U          [n_used][(M-1) RP] row-major: the whitened leaf basis What^l of
//              every observation, overwritten in place by Y = L_V^{-1} U.
//   leaf_w     [n_leaf][(M-1) RP]  w_c = Y_c' y_c of each leaf (FP64)
//   leaf_du    [n_leaf][2]         (log|V_c|, y_c'y_c)
//   Ain        level M-1 regions: A = sum over the leaf children of Y'Y, packed
//              upper blocks (k <= l, pair index l(l-1)/2 + k-1), each RP x RP
//              row-major; Ain_w (FP64) the summed w, Ain_du the summed (d, u).
//              Holds one chunk of consecutive regions when the whole level
//              does not fit (the leaf Gram and the level M-1 upward step then
//              run chunk by chunk).
//   gexp       level M-1 regions (same chunking as Ain): int8 column exponents of
//              Y for the exact tensor-core Gram (mixed mode).
//   Atil[m]    level m regions (2 <= m <= M-1): ATilde after the region's
//              step, blocks (k <= l <= m-1), same packing, plus w (FP64) and (d, u).
#pragma once
#include <cstddef>
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

#define MRA_MAXM 36
#define MRA_NT 256

namespace mra {

// The tree the kernels run on.  Its levels are the partition's levels, except
// that a region with more knots than one warp holds (33..64) enters its knots
// in two successive levels of the same region: the first ceil(r/2) knots,
// then the rest, with a single child between the two (Sec. 1.1 recursion: the
// remainder after projecting on Q1 and then on Q2 is the remainder after
// projecting on Q1 u Q2, so Sigma_MRA is unchanged).  Rl[m] is the number of
// knots of a level-m region (the rest of the RP slots is inert padding), Jl[m]
// the children of a level-m region, and region i of level m has the ancestor
// i >> (sh[m] - sh[l]) at level l.
struct DevTree {
    int M, RP;
    int64_t n_used;
    const double *kx, *ky;
    const double *cx, *cy;
    const double *sx, *sy, *sz;
    const int64_t *leaf_off;
    int64_t lvl_off[MRA_MAXM + 2]; // first global region id of level m (1-based)
    int Rl[MRA_MAXM + 1];
    int Jl[MRA_MAXM + 1];
    int sh[MRA_MAXM + 2];
};

// Index of the level-l ancestor of region i (index within its level) of level m.
__host__ __device__ inline int64_t anc_index(const DevTree &t, int64_t i, int m, int l)
{
    return i >> (t.sh[m] - t.sh[l]);
}

template <typename T>
struct Work {
    const double *theta; // [B][3]
    int *status;         // [B]
    double *loglik;      // [B]
    T *prior;
    size_t prior_stride;
    size_t prior_lvl[MRA_MAXM + 1]; // element offset of level m inside one theta's prior
    T *U;
    size_t U_stride;
    double *leaf_w; // FP64 in both modes (see gram_vec)
    size_t leafw_stride;
    double *leaf_du; // [nleaf][2]
    size_t leafdu_stride;
    double *Vbig; // big-leaf scratch
    size_t V_stride;
    T *Ain;         // [nP][npairs(M-1)][RP*RP]
    double *Ain_w;  // [nP][(M-1) RP]
    double *Ain_du; // [nP][2]
    size_t Ain_stride, Ainw_stride, Aindu_stride;
    int8_t *gexp;   // [nP][(M-1) RP]: per column of Y below each region, e with 2^e > max |Y| (mixed mode)
    size_t gexp_stride;
    // tensor-core leaf basis (null otherwise): fixed-grid BF16 slices of What,
    // stored step-major (mra_kernels.cuh, tc_step_off).  lbB: each region of
    // levels 2..M-1, its m - 1 blocks of RP x RP (at byte offset lbB_lvl[m] +
    // i (m - 1) 5 RP^2 2); lbA: each 128-row chunk, its rows' What^1..What^{M-2}
    // (chunk c, level k at (c (M - 2) + k - 1) 5 128 RP 2)
    unsigned char *lbA, *lbB;
    size_t lbA_stride, lbB_stride;
    size_t lbB_lvl[MRA_MAXM + 1];
    T *Atil[MRA_MAXM + 1];
    double *Atil_w[MRA_MAXM + 1];
    double *Atil_du[MRA_MAXM + 1];
    size_t Atil_stride[MRA_MAXM + 1], Atilw_stride[MRA_MAXM + 1], Atildu_stride[MRA_MAXM + 1];
    int exact_rem;  // FP32 storage: remainder recursions with float-pair covariance and exact products
    // subtree streaming (0: off): levels m > sub_level run chunk by chunk of
    // level-sub_level subtrees, and their Atil arrays (and Ain) hold only the
    // current chunk's regions, indexed from the chunk's first region
    int sub_level;
    double *reg_du; // [nreg][2] or null
    double *reg_lw; // [n_nonleaf] or null
    size_t regdu_stride, reglw_stride;
    // prediction (null otherwise; batch slot 0 only): the upward pass keeps
    // its factors per non-leaf region (keep_up, FP64, keep_up_stride doubles
    // each), the shared-memory leaf posterior its L^{-1} (keep_li, k-major,
    // kKeepLd x kKeepLd per leaf) and y = L^{-1} z (keep_y, kKeepLd per leaf)
    double *keep_up;
    size_t keep_up_stride;
    T *keep_li;
    double *keep_y;
};

// Dynamic shared memory one CTA may ask for on this GPU (227 KB).
constexpr size_t kSmemMax = (size_t)227 * 1024;

// Leading dimension of a kept leaf factor: the largest shared-memory bucket.
constexpr int kKeepLd = 64;

// Doubles kept per non-leaf region (Work::keep_up):
//   [0, RP^2)              L~, the factor of I + A^{m,m}: lower, row-major
//   [RP^2, RP^2 + RP)      1 / L~_ii
//   [RP^2 + RP, RP^2 + 2RP) v = L~^{-1} omega^m
//   then Z = L~^{-1} [A^{m,1} .. A^{m,m-1}] as RP rows of (M-2) RP doubles
//   (level m uses the first (m-1) RP)
__host__ __device__ inline size_t keep_up_doubles(int M, int RP)
{
    return (size_t)RP * RP + 2 * (size_t)RP + (size_t)RP * (size_t)(M > 2 ? (M - 2) * RP : 0);
}

struct BigLeaf;
struct PredArgs {
    int64_t np;
    const double *px, *py; // prediction points, grouped by leaf
    const int64_t *leaf;   // leaf of each point, -1 outside the domain
    const void *Ua;        // per point: (M-1) RP basis values a* (storage type)
    const double *xi;      // per non-leaf region: RP posterior means
    const double *keep_up;
    size_t keep_stride;
    const int32_t *bigidx; // per leaf: index into big, -1 for a shared-memory leaf
    const BigLeaf *big;
    double *mean, *var;
    int nl;  // per-warp scratch rows (largest leaf, at least 1)
    int wpb; // warps per block
};

// Doubles of per-warp scratch.
__host__ __device__ inline size_t predict_warp_doubles(int M, int RP, int nl)
{
    return 3 * (size_t)(M - 1) * RP + 2 * (size_t)nl + (size_t)RP;
}


// Leaf-posterior buckets: a leaf with n observations runs in the kernel of the
// smallest cap >= n (shared-memory footprint grows as cap^2, so a cap close
// above the common leaf sizes keeps more CTAs per SM: a 40-observation bucket
// runs four CTAs per SM where the 48 one runs three at r = 32).
constexpr int kLeafBuckets = 4;
constexpr int kLeafCap[kLeafBuckets] = {32, 40, 48, 64};

struct Chunk {
    int32_t parent; // level M-1 region index
    int32_t n;      // rows in this chunk (<= chunk rows of the precision)
    int64_t row0;   // first observation row
};

struct BigLeaf {
    int64_t leaf;
    int64_t voff; // element offset (doubles) of its scratch in Vbig
};

// Large leaves are factored in square tiles of kBigTile rows.
constexpr int kBigTile = 32;

// One work item of the tiled large-leaf kernels: leaf bl (index into the
// BigLeaf list), tile row i, tile column j.
struct BigTile {
    int32_t bl, i, j, pad;
};

// Scratch of one large leaf in Vbig, in 8-byte slots: V and its factor
// (n^2), z then y (n), reciprocal pivots (n), (log-det, quadratic form) (2).
inline int64_t big_leaf_scratch(int64_t n) { return n * n + 2 * n + 2; }

// The streaming leaf basis of deep trees: rows per chunk and ancestor blocks
// staged at a time (mra_tune_t.leafbasis_rows = 16 selects it).
constexpr int kStreamRows = 16, kStreamBlocks = 2;

// Deep levels whose shared-memory footprint exceeds one CTA's: the prior
// stages its ancestor's blocks kPriorStreamBlocks at a time, the upward pass
// the right-hand blocks of its solve kUpStreamBlocks at a time, and the
// large-leaf assembly reads its U rows in kBigAssembleParts column parts.
// Each sums the same terms in the same order as the whole-staged kernel.
constexpr int kPriorStreamBlocks = 4, kUpStreamBlocks = 4, kBigAssembleParts = 2;

// Observation rows per leaf-basis chunk: 64 in FP32, 32 in FP64 (shared memory).
template <typename T> __host__ __device__ constexpr int chunk_rows() { return sizeof(T) == 4 ? 64 : 32; }

// Launchers (one instantiation per precision T and padding RP).
template <typename T, int RP>
int launch_prior(const DevTree &t, const Work<T> &w, int m, int B, int stages_req, void *stream);
template <int RP>
int launch_down(const DevTree &t, const double *keep, size_t stride, double *xi, int m, void *stream);
template <typename T, int RP>
int launch_predict(const DevTree &t, const Work<T> &w, const PredArgs &q, void *stream);
template <typename T, int RP>
int launch_leafbasis(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int rows, int stages,
                     int B, void *stream);
template <typename T, int RP>
int launch_leafbasis_half(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int rows, int stages,
                          int B, void *stream);
template <typename T, int RP>
int launch_leafbasis_tc(const DevTree &t, const Work<T> &w, const Chunk *chunks, int nchunks, int B, void *stream);
// Rows per chunk of the tensor-core leaf basis, and the largest (M - 2) RP
// its exact sums allow.
constexpr int kLeafBasisTcRows = 128;
constexpr int kLeafBasisTcMaxK = 192;
template <typename T, int RP>
int launch_leafpost_small(const DevTree &t, const Work<T> &w, const int64_t *leaves, int nleaves,
                          int nmax, int B, unsigned *queue, void *stream);
// Tiled large-leaf posterior: one launch per phase; items of that phase.
enum BigPhase { BIG_ASSEMBLE = 0, BIG_POTRF = 1, BIG_TRSM = 2, BIG_UPDATE = 3, BIG_FINISH = 4 };
template <typename T, int RP>
int launch_big(const DevTree &t, const Work<T> &w, int phase, const BigLeaf *leaves, const BigTile *items,
               int nitems, int k, int B, void *stream);
template <typename T, int RP>
int launch_leafgram(const DevTree &t, const Work<T> &w, int reg0, int nP, int B, bool tensor_cores, void *stream);
template <typename T, int RP>
int launch_gram_colexp(const DevTree &t, const Work<T> &w, int reg0, int nP, int B, void *stream);
template <typename T, int RP>
int launch_up(const DevTree &t, const Work<T> &w, int m, int reg0, int nreg, int B, void *stream);
template <typename T, int RP>
int launch_root_single(const DevTree &t, const Work<T> &w, int B, void *stream);

// Dynamic shared memory (bytes) each kernel needs.
template <typename T, int RP> size_t smem_prior(int m);
template <typename T, int RP> size_t smem_leafbasis(int M);
template <typename T, int RP> size_t smem_leafbasis_cfg(int M, int rows, int stages);
template <typename T, int RP> size_t smem_leafpost_small(int M, int nmax);
template <typename T, int RP> size_t smem_up(int m);
template <typename T, int RP> size_t smem_leafgram(int M);
template <typename T, int RP> size_t smem_big(int M);

} // namespace mra
