// mra_api.cu -- the C ABI of libmra (include/mra.h): partition build on the
// host, device layout, and the per-level launch sequence of one likelihood
// evaluation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

#include "../../include/mra.h"
#include "mra_internal.h"

using namespace mra;

namespace {

const double kDefaultOffset = 2.718281828459045235360287 / 100.0; // e/100 (Sec. 1.2)

// ------------------------------------------------------------ partition --
// Sec. 1.2: bounding box pushed out by 1% at the top and right, half-open
// regions, J = 4 quadrants or J = 2 halves of the longer side (decided per
// level from the nominal side lengths, which halve exactly; ties cut x),
// ceil(sqrt r) x floor(r / ceil(sqrt r)) knots at x0 + L (f + p (1-2f)/(n-1)).
struct Partition {
    int M = 0, J = 0, r = 0, nx = 0, ny = 0, R = 0;
    double f = 0.0;
    std::vector<int64_t> lvl_off; // [M+2], index m = first global id of level m
    std::vector<double> bx0, bx1, by0, by1;
    std::vector<char> cut_x;      // per level m < M (J = 2)
    std::vector<double> kx, ky;   // [n_nonleaf * R]
    std::vector<int64_t> leaf_off;
    std::vector<double> sx, sy, sz;
    std::vector<int64_t> perm;
    int64_t n_in = 0, n_used = 0, n_nan = 0, n_dup = 0, n_knot = 0;
    int64_t nreg() const { return lvl_off[M + 1]; }
    int64_t nleaf() const { return lvl_off[M + 1] - lvl_off[M]; }
    int64_t nnonleaf() const { return lvl_off[M]; }
};

int side_bars(int r)
{
    int a = 1;
    while (a * a < r) a++;
    return a;
}

void knot_grid(double x0, double x1, double y0, double y1, int nx, int ny, double f, double *kx, double *ky)
{
    const double Lx = x1 - x0, Ly = y1 - y0;
    for (int q = 0; q < ny; q++) {
        const double yq = ny > 1 ? y0 + Ly * (f + (double)q * (1.0 - 2.0 * f) / (double)(ny - 1)) : y0 + 0.5 * Ly;
        for (int p = 0; p < nx; p++) {
            kx[q * nx + p] = nx > 1 ? x0 + Lx * (f + (double)p * (1.0 - 2.0 * f) / (double)(nx - 1)) : x0 + 0.5 * Lx;
            ky[q * nx + p] = yq;
        }
    }
}

mra_status build_partition(const double *x, const double *y, const double *z, int64_t n, int M, int J, int r,
                           double f, int dedup, Partition &P, std::string &err)
{
    if (n < 0 || M < 1 || M > MRA_MAXM - 1 || (J != 2 && J != 4) || r < 1) {
        err = "invalid n, M, J or r";
        return MRA_EINVAL;
    }
    if (!(f >= 0.0 && f < 0.5)) {
        err = "offset must lie in [0, 0.5)";
        return MRA_EINVAL;
    }
    double total = 0.0, pw = 1.0;
    for (int m = 1; m <= M; m++) {
        total += pw;
        pw *= J;
    }
    if (total > 268435456.0) {
        err = "too many regions (J^M)";
        return MRA_EINVAL;
    }
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(x[i]) || !std::isfinite(y[i])) {
            err = "non-finite location";
            return MRA_EINVAL;
        }
    P.M = M;
    P.J = J;
    P.r = r;
    P.f = f;
    P.nx = side_bars(r);
    P.ny = r / P.nx;
    P.R = P.nx * P.ny;
    P.n_in = n;

    std::vector<int64_t> idx;
    idx.reserve((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        if (std::isnan(z[i]))
            P.n_nan++;
        else
            idx.push_back(i);
    }
    if (dedup && !idx.empty()) {
        std::vector<int64_t> s(idx);
        std::sort(s.begin(), s.end(), [&](int64_t a, int64_t b) {
            if (x[a] != x[b]) return x[a] < x[b];
            if (y[a] != y[b]) return y[a] < y[b];
            return a < b;
        });
        std::vector<char> gone((size_t)n, 0);
        for (size_t k = 1; k < s.size(); k++)
            if (x[s[k]] == x[s[k - 1]] && y[s[k]] == y[s[k - 1]]) {
                gone[(size_t)s[k]] = 1;
                P.n_dup++;
            }
        std::vector<int64_t> kept;
        kept.reserve(idx.size());
        for (int64_t i : idx)
            if (!gone[(size_t)i]) kept.push_back(i);
        idx.swap(kept);
    }
    if (idx.empty()) {
        err = "no observation left";
        return MRA_EEMPTY;
    }
    double xmin = x[idx[0]], xmax = xmin, ymin = y[idx[0]], ymax = ymin;
    for (int64_t i : idx) {
        xmin = std::min(xmin, x[i]);
        xmax = std::max(xmax, x[i]);
        ymin = std::min(ymin, y[i]);
        ymax = std::max(ymax, y[i]);
    }
    if (!(xmax > xmin) || !(ymax > ymin)) {
        err = "degenerate domain (zero extent)";
        return MRA_EINVAL;
    }
    P.lvl_off.assign((size_t)M + 2, 0);
    int64_t cnt = 1;
    for (int m = 1; m <= M; m++) {
        P.lvl_off[(size_t)m + 1] = P.lvl_off[(size_t)m] + cnt;
        cnt *= J;
    }
    const int64_t NR = P.nreg();
    P.bx0.resize((size_t)NR);
    P.bx1.resize((size_t)NR);
    P.by0.resize((size_t)NR);
    P.by1.resize((size_t)NR);
    P.bx0[0] = xmin;
    P.bx1[0] = xmax + 0.01 * (xmax - xmin);
    P.by0[0] = ymin;
    P.by1[0] = ymax + 0.01 * (ymax - ymin);
    P.cut_x.assign((size_t)M + 1, 1);
    double lx = P.bx1[0] - P.bx0[0], ly = P.by1[0] - P.by0[0];
    for (int m = 1; m < M; m++) {
        const bool cx = lx >= ly;
        P.cut_x[(size_t)m] = cx;
        if (J == 4) {
            lx *= 0.5;
            ly *= 0.5;
        } else if (cx) {
            lx *= 0.5;
        } else {
            ly *= 0.5;
        }
        for (int64_t g = P.lvl_off[(size_t)m]; g < P.lvl_off[(size_t)m + 1]; g++) {
            const int64_t i = g - P.lvl_off[(size_t)m];
            const int64_t c0 = P.lvl_off[(size_t)m + 1] + i * J;
            const double X0 = P.bx0[(size_t)g], X1 = P.bx1[(size_t)g], Y0 = P.by0[(size_t)g], Y1 = P.by1[(size_t)g];
            const double mx = 0.5 * (X0 + X1), my = 0.5 * (Y0 + Y1);
            for (int j = 0; j < J; j++) {
                double a0 = X0, a1 = X1, b0 = Y0, b1 = Y1;
                if (J == 4) {
                    (j & 1 ? a0 : a1) = mx;
                    (j & 2 ? b0 : b1) = my;
                } else if (cx) {
                    (j ? a0 : a1) = mx;
                } else {
                    (j ? b0 : b1) = my;
                }
                P.bx0[(size_t)(c0 + j)] = a0;
                P.bx1[(size_t)(c0 + j)] = a1;
                P.by0[(size_t)(c0 + j)] = b0;
                P.by1[(size_t)(c0 + j)] = b1;
            }
        }
    }
    const int64_t NK = P.nnonleaf();
    P.kx.resize((size_t)(NK * P.R));
    P.ky.resize((size_t)(NK * P.R));
    for (int64_t g = 0; g < NK; g++)
        knot_grid(P.bx0[(size_t)g], P.bx1[(size_t)g], P.by0[(size_t)g], P.by1[(size_t)g], P.nx, P.ny, f,
                  &P.kx[(size_t)(g * P.R)], &P.ky[(size_t)(g * P.R)]);
    if (NK > 0) {
        std::vector<std::pair<double, double>> ks((size_t)(NK * P.R));
        for (size_t k = 0; k < ks.size(); k++) ks[k] = {P.kx[k], P.ky[k]};
        std::sort(ks.begin(), ks.end());
        std::vector<int64_t> kept;
        kept.reserve(idx.size());
        for (int64_t i : idx) {
            if (std::binary_search(ks.begin(), ks.end(), std::make_pair(x[i], y[i])))
                P.n_knot++;
            else
                kept.push_back(i);
        }
        idx.swap(kept);
    }
    const int64_t NL = P.nleaf();
    std::vector<int64_t> leaf(idx.size());
    for (size_t k = 0; k < idx.size(); k++) {
        const double a = x[idx[k]], b = y[idx[k]];
        int64_t i = 0;
        for (int m = 1; m < M; m++) {
            const int64_t g = P.lvl_off[(size_t)m] + i;
            const double mx = 0.5 * (P.bx0[(size_t)g] + P.bx1[(size_t)g]);
            const double my = 0.5 * (P.by0[(size_t)g] + P.by1[(size_t)g]);
            int j;
            if (J == 4)
                j = (a >= mx) | ((b >= my) << 1);
            else
                j = P.cut_x[(size_t)m] ? (a >= mx) : (b >= my);
            i = i * J + j;
        }
        leaf[k] = i;
    }
    P.leaf_off.assign((size_t)NL + 1, 0);
    for (int64_t l : leaf) P.leaf_off[(size_t)l + 1]++;
    for (int64_t i = 0; i < NL; i++) P.leaf_off[(size_t)i + 1] += P.leaf_off[(size_t)i];
    std::vector<int64_t> pos(P.leaf_off.begin(), P.leaf_off.end() - 1);
    P.n_used = (int64_t)idx.size();
    P.sx.resize(idx.size());
    P.sy.resize(idx.size());
    P.sz.resize(idx.size());
    P.perm.resize(idx.size());
    for (size_t k = 0; k < idx.size(); k++) {
        const int64_t p = pos[(size_t)leaf[k]]++;
        P.sx[(size_t)p] = x[idx[k]];
        P.sy[(size_t)p] = y[idx[k]];
        P.sz[(size_t)p] = z[idx[k]];
        P.perm[(size_t)p] = idx[k];
    }
    if (P.n_used == 0) {
        err = "no observation left";
        return MRA_EEMPTY;
    }
    return MRA_OK;
}

// The levels the kernels run on (DevTree).  With r_hat <= 32 they are the
// partition's levels.  With 32 < r_hat <= 64 every non-leaf level l enters its
// knots in two device levels of the same regions: 2l - 1 holds the first
// ceil(r_hat/2) knots and has one child (itself at 2l), 2l holds the rest and
// has the J children of level l.  The remainder recursion of Sec. 1.1 after
// projecting on Q1 and then on Q2 equals the one after projecting on
// Q1 u Q2 (the Schur complement of the knot covariance), so Sigma_MRA, the
// likelihood and the predictive distribution are unchanged, and every region
// still fits one warp's lanes.
struct Levels {
    int M = 0, split = 1, RP = 0;
    std::vector<int64_t> lvl_off; // [M+2]
    std::vector<int> Rl, Jl;      // [M+1]: knots and children of a level-m region
    std::vector<int> real;        // [M+1]: partition level of device level m
    std::vector<double> kx, ky;   // [nnonleaf * RP], padded with zeros
    std::vector<double> cx, cy;   // [nnonleaf] lower-left corner of the region
    int64_t nreg() const { return lvl_off[(size_t)M + 1]; }
    int64_t nnonleaf() const { return lvl_off[(size_t)M]; }
    int64_t nleaf() const { return nreg() - nnonleaf(); }
    int lgJ(int m) const { return Jl[(size_t)m] == 4 ? 2 : (Jl[(size_t)m] == 2 ? 1 : 0); }
};

// Largest r_hat the two-level split serves.
constexpr int kMaxRhat = 64;

mra_status make_levels(const Partition &P, Levels &G, std::string &err)
{
    if (P.R > kMaxRhat) {
        err = "r_hat > 64 is not supported";
        return MRA_EINVAL;
    }
    G.split = P.R > 32 ? 2 : 1;
    const int Mr = P.M;
    G.M = G.split == 1 ? Mr : 2 * (Mr - 1) + 1;
    if (G.M > MRA_MAXM - 1) {
        err = "M too large for r_hat > 32 (device levels 2 (M - 1) + 1 exceed the limit)";
        return MRA_EINVAL;
    }
    const int R1 = G.split == 1 ? P.R : (P.R + 1) / 2;
    G.lvl_off.assign((size_t)G.M + 2, 0);
    G.Rl.assign((size_t)G.M + 1, 0);
    G.Jl.assign((size_t)G.M + 1, 0);
    G.real.assign((size_t)G.M + 1, 0);
    for (int m = 1; m <= G.M; m++) {
        const int l = G.split == 1 ? m : (m + 1) / 2; // partition level
        const int h = G.split == 1 ? 0 : (m - 1) % 2; // which half of its knots
        G.real[(size_t)m] = l;
        const int64_t cnt = P.lvl_off[(size_t)l + 1] - P.lvl_off[(size_t)l];
        G.lvl_off[(size_t)m + 1] = G.lvl_off[(size_t)m] + cnt;
        if (m < G.M) {
            G.Rl[(size_t)m] = h == 0 ? R1 : P.R - R1;
            G.Jl[(size_t)m] = (G.split == 2 && h == 0) ? 1 : P.J;
        }
    }
    int rmax = 0;
    for (int m = 1; m < G.M; m++) rmax = std::max(rmax, G.Rl[(size_t)m]);
    G.RP = rmax <= 16 ? 16 : 32;
    const int64_t NK = G.nnonleaf();
    G.kx.assign((size_t)(NK * G.RP), 0.0);
    G.ky.assign((size_t)(NK * G.RP), 0.0);
    G.cx.assign((size_t)std::max<int64_t>(NK, 1), 0.0);
    G.cy.assign(G.cx.size(), 0.0);
    for (int m = 1; m < G.M; m++) {
        const int l = G.real[(size_t)m];
        const int first = (G.split == 2 && (m - 1) % 2 == 1) ? R1 : 0;
        for (int64_t i = 0; i < G.lvl_off[(size_t)m + 1] - G.lvl_off[(size_t)m]; i++) {
            const int64_t g = G.lvl_off[(size_t)m] + i, pg = P.lvl_off[(size_t)l] + i;
            for (int j = 0; j < G.Rl[(size_t)m]; j++) {
                G.kx[(size_t)(g * G.RP + j)] = P.kx[(size_t)(pg * P.R + first + j)];
                G.ky[(size_t)(g * G.RP + j)] = P.ky[(size_t)(pg * P.R + first + j)];
            }
            G.cx[(size_t)g] = P.bx0[(size_t)pg];
            G.cy[(size_t)g] = P.by0[(size_t)pg];
        }
    }
    return MRA_OK;
}

} // namespace

// --------------------------------------------------------------- context --
struct mra_ctx {
    Partition P; // the partition of Sec. 1.2 (what the user sees)
    Levels G;    // the levels the kernels run on
    int RP = 0, lgJ = 0, precision = MRA_FP64, device = 0;
    std::string err;
    // device tree
    double *d_kx = nullptr, *d_ky = nullptr, *d_sx = nullptr, *d_sy = nullptr, *d_sz = nullptr;
    double *d_cx = nullptr, *d_cy = nullptr;
    int64_t *d_leaf_off = nullptr;
    Chunk *d_chunks32 = nullptr, *d_chunks64 = nullptr; // leaf-basis chunks of 32 / 64 rows
    int nchunks32 = 0, nchunks64 = 0;
    // the last ntail32 (ntail64) chunks of each list are the regions' tails
    // of at most half a chunk, which run as chunks of half the rows
    int ntail32 = 0, ntail64 = 0;
    Chunk *d_chunks128 = nullptr; // 128-row chunks of the tensor-core leaf basis
    int nchunks128 = 0;
    Chunk *d_chunks16 = nullptr; // 16-row chunks of the streaming leaf basis (deep trees)
    int nchunks16 = 0;
    // leaves with 1..kLeafCap[k] observations (and more than the previous cap),
    // one CTA each; larger leaves take the global-memory path
    int64_t *d_leaves[kLeafBuckets] = {};
    int nl[kLeafBuckets] = {};
    int nmax_small = 64; // largest bucket cap whose shared memory fits
    bool lb64_fits = true; // mixed modes: 64-row leaf-basis chunks fit in shared memory
    bool fp64_fits = true; // the FP64 kernels fit in shared memory on this tree
    // the buckets above the first as one list (bucket set 1)
    int64_t *d_leaves_m = nullptr;
    int nl_m = 0;
    // launch configuration (mra_autotune): leaf-basis rows per chunk (0 = the
    // precision's default) and prefetch stages (0 = automatic), bucket set
    // (0: 32/40/48/64, 1: 32/64), side streams for the leaf posterior
    int lb_rows = 0, lb_stages = 0, bucket_set = 0;
    bool concurrent = true;
    bool gram_tc = false; // mixed modes: leaf Gram on the tensor cores (exact slices)
    bool lb_tc = false;   // MRA_MIXED: leaf basis with its remainder products on the tensor cores
    bool leaf_queue = false; // shared-memory leaf buckets as persistent work-queue kernels
    bool lb_whole = false;   // leaf basis: tails of 32/64-row chunks kept in full-size chunks
    int prior_st = 0;        // prior: 0 by occupancy, 1 one stage, 2 two where they fit, 3 two blocks at a time
    unsigned *d_qcnt = nullptr; // their counters: kLeafBuckets x status_cap
    BigLeaf *d_big = nullptr;
    int nbig = 0;
    // work items of the tiled large-leaf kernels: [0, n_assemble) assembly
    // tiles, then per step k the potrf, trsm and update items at big_off[k]
    BigTile *d_bigitems = nullptr;
    int big_nassemble = 0;
    std::vector<std::array<int, 6>> big_steps; // (potrf off, cnt, trsm off, cnt, update off, cnt)
    int64_t vbig_elems = 0;
    // per-theta scratch: one allocation for `cap` theta, sized for FP64
    int cap = 0;     // theta the scratch currently holds
    int max_cap = 1; // theta per device pass allowed by the memory budget
    int user_max_batch = 0;
    size_t hbm_budget = 0;   // from the options (0 = 60% of free HBM)
    int ain_chunk = 0;       // level M-1 regions per Ain chunk (0 = the whole level)
    // subtree streaming: levels below device level sub_level run chunk by
    // chunk of sub_chunk level-sub_level subtrees (0 = off); sub_req_* force
    // it (mra_set_launch), 0 = chosen by the memory plan
    int sub_level = 0, sub_chunk = 0, sub_req_level = 0, sub_req_chunk = 0;
    int status_cap = 0;      // theta the status array holds
    // captured device passes, replayed when the same pass comes again
    struct GraphEntry {
        const double *theta;
        double *loglik;
        int *status;
        int B, precision, regions;
        uint64_t gen, last_use;
        cudaGraphExec_t exec;
    };
    bool graphs = true;
    uint64_t scratch_gen = 0, use_clock = 0;
    std::vector<GraphEntry> graph_cache;
    std::vector<GraphEntry> graph_seen; // passes run once, captured on their next call
    cudaStream_t cap_stream = nullptr;
    // independent leaf-posterior launches (size buckets, the large-leaf
    // pipeline) run side by side on these streams, forked from and joined to
    // the pass's stream by events
    cudaStream_t aux[kLeafBuckets] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kLeafBuckets] = {};
    cudaEvent_t lbt_fork = nullptr, lbt_join = nullptr; // the leaf basis's tail chunks on aux[0]
    unsigned char *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    size_t per_theta_bytes = 0;
    int *d_status = nullptr;
    double *d_theta_stage = nullptr, *d_ll_stage = nullptr;
    int stage_cap = 0;
    double *d_reg_du = nullptr, *d_reg_lw = nullptr;
    size_t bytes_held = 0;
    // optional per-kernel device timing (events around every launch)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    int launches_last = 0;
    int64_t max_leaf = 0, empty_leaves = 0;
    double flops = 0.0, covs = 0.0;
    // set only while mra_predict runs its pass: where the kernels keep the
    // factors prediction needs (Work::keep_*)
    double *keep_up = nullptr, *keep_y = nullptr;
    void *keep_li = nullptr;
    size_t keep_stride = 0;
    // every device pass counts itself; mra_predict reuses the factors of its
    // last pass while theta, the precision and the scratch are unchanged and
    // no other pass has run since
    uint64_t pass_count = 0;
    struct PredState {
        unsigned char *pt = nullptr, *tree = nullptr; // per-point and per-tree buffers (grow-only)
        size_t pt_bytes = 0, tree_bytes = 0;
        double theta[3] = {0.0, 0.0, 0.0};
        int precision = -1;
        uint64_t pass_id = 0, gen = 0;
        bool valid = false;
    } pred;
    double flops_k[8] = {0};
};

namespace {

mra_status cuda_fail(mra_ctx *c, cudaError_t e, const char *what)
{
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return MRA_ECUDA;
}

template <typename T>
mra_status dev_upload(mra_ctx *c, T **dst, const T *src, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)dst, count * sizeof(T));
    if (e != cudaSuccess) {
        c->err = "cudaMalloc failed for the tree";
        return MRA_ENOMEM;
    }
    c->bytes_held += count * sizeof(T);
    if (src) {
        e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    }
    return MRA_OK;
}

// Element counts of one theta's scratch (in units of the storage type for the
// T-typed parts, doubles for the rest).
struct Plan {
    size_t prior = 0, prior_lvl[MRA_MAXM + 1] = {0};
    size_t U = 0, leafw = 0, leafdu = 0, V = 0;
    size_t Ain = 0, Ainw = 0, Aindu = 0, Gexp = 0;
    size_t lbA = 0, lbB = 0, lbB_lvl[MRA_MAXM + 1] = {0}; // bytes (tensor-core leaf basis)
    size_t Atil[MRA_MAXM + 1] = {0}, Atilw[MRA_MAXM + 1] = {0}, Atildu[MRA_MAXM + 1] = {0};
    size_t t_elems = 0, d_elems = 0; // totals
};

Plan make_plan(const mra_ctx *c)
{
    const Levels &P = c->G;
    const int M = P.M, RP = c->RP;
    const size_t B2 = (size_t)RP * RP;
    Plan p;
    size_t acc = 0;
    for (int m = 1; m < M; m++) {
        p.prior_lvl[m] = acc;
        acc += (size_t)(P.lvl_off[(size_t)m + 1] - P.lvl_off[(size_t)m]) * m * B2;
    }
    p.prior = acc;
    p.U = (size_t)c->P.n_used * (size_t)(M - 1) * RP;
    p.leafw = (size_t)P.nleaf() * (size_t)(M - 1) * RP;
    p.leafdu = 2 * (size_t)P.nleaf();
    p.V = (size_t)c->vbig_elems;
    // regions of level m the per-theta arrays hold: the whole level, or under
    // subtree streaming the descendants of sub_chunk level-S regions below S
    const int S = c->sub_level;
    auto held = [&](int m) {
        const size_t nr = (size_t)(P.lvl_off[(size_t)m + 1] - P.lvl_off[(size_t)m]);
        if (S <= 0 || m <= S) return nr;
        const size_t nS = (size_t)(P.lvl_off[(size_t)S + 1] - P.lvl_off[(size_t)S]);
        return std::min(nS, (size_t)c->sub_chunk) * (nr / nS);
    };
    if (M >= 2) {
        size_t nP = held(M - 1);
        if (c->ain_chunk > 0) nP = std::min(nP, (size_t)c->ain_chunk);
        p.Ain = nP * (size_t)(M - 1) * M / 2 * B2;
        p.Ainw = nP * (size_t)(M - 1) * RP;
        p.Aindu = 2 * nP;
        p.Gexp = nP * (size_t)(M - 1) * RP;
        if (c->lb_tc && M >= 3) {
            // fixed-grid slices: 5 planes of BF16 per block
            const size_t bblk = (size_t)5 * RP * RP * 2, arow = (size_t)5 * kLeafBasisTcRows * RP * 2;
            p.lbA = (size_t)c->nchunks128 * (size_t)(M - 2) * arow;
            size_t acc_b = 0;
            for (int m = 2; m <= M - 1; m++) {
                p.lbB_lvl[m] = acc_b;
                acc_b += (size_t)(P.lvl_off[(size_t)m + 1] - P.lvl_off[(size_t)m]) * (size_t)(m - 1) * bblk;
            }
            p.lbB = acc_b;
        }
        for (int m = 2; m <= M - 1; m++) {
            const size_t nr = held(m);
            p.Atil[m] = nr * (size_t)(m - 1) * m / 2 * B2;
            p.Atilw[m] = nr * (size_t)(m - 1) * RP;
            p.Atildu[m] = 2 * nr;
        }
    }
    p.t_elems = p.prior + p.U + p.leafw + p.Ain;
    for (int m = 2; m <= M - 1; m++) p.t_elems += p.Atil[m];
    p.d_elems = p.leafdu + p.V + p.Ainw + p.Aindu;
    for (int m = 2; m <= M - 1; m++) p.d_elems += p.Atilw[m] + p.Atildu[m];
    return p;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve one theta-batch view of the scratch for storage type T.
template <typename T>
Work<T> make_work(const mra_ctx *c, const Plan &p, int B)
{
    Work<T> w;
    memset(&w, 0, sizeof(w));
    unsigned char *base = c->d_scratch;
    size_t off = 0;
    auto takeT = [&](size_t elems) {
        T *q = (T *)(base + off);
        off = align256(off + elems * (size_t)B * sizeof(T));
        return q;
    };
    auto takeD = [&](size_t elems) {
        double *q = (double *)(base + off);
        off = align256(off + elems * (size_t)B * sizeof(double));
        return q;
    };
    // T arrays in sizeof(T): the allocation is sized for the precision in use
    auto takeT8 = takeT;
    w.prior = takeT8(p.prior);
    w.prior_stride = p.prior;
    for (int m = 0; m <= MRA_MAXM; m++) w.prior_lvl[m] = p.prior_lvl[m];
    w.U = takeT8(p.U);
    w.U_stride = p.U;
    w.leaf_w = takeD(p.leafw);
    w.leafw_stride = p.leafw;
    w.leaf_du = takeD(p.leafdu);
    w.leafdu_stride = p.leafdu;
    w.Vbig = takeD(p.V);
    w.V_stride = p.V;
    w.Ain = takeT8(p.Ain);
    w.Ain_stride = p.Ain;
    w.Ain_w = takeD(p.Ainw);
    w.Ainw_stride = p.Ainw;
    w.Ain_du = takeD(p.Aindu);
    w.Aindu_stride = p.Aindu;
    {
        w.gexp = (int8_t *)(base + off);
        off = align256(off + p.Gexp * (size_t)B);
        w.gexp_stride = p.Gexp;
    }
    if (p.lbA > 0) {
        w.lbA = base + off;
        off = align256(off + p.lbA * (size_t)B);
        w.lbA_stride = p.lbA;
        w.lbB = base + off;
        off = align256(off + p.lbB * (size_t)B);
        w.lbB_stride = p.lbB;
        for (int m = 0; m <= MRA_MAXM; m++) w.lbB_lvl[m] = p.lbB_lvl[m];
    }
    for (int m = 2; m <= c->G.M - 1; m++) {
        w.Atil[m] = takeT8(p.Atil[m]);
        w.Atil_stride[m] = p.Atil[m];
        w.Atil_w[m] = takeD(p.Atilw[m]);
        w.Atilw_stride[m] = p.Atilw[m];
        w.Atil_du[m] = takeD(p.Atildu[m]);
        w.Atildu_stride[m] = p.Atildu[m];
    }
    w.status = c->d_status;
    w.sub_level = c->sub_level;
    return w;
}

// Bytes of the per-theta scratch for B theta; arrays of the storage type
// take 4 bytes per element in the mixed mode and 8 in the FP64 mode (the
// layout make_work<T> lays out).
size_t scratch_bytes_for(const Plan &p, const mra_ctx *c, int B)
{
    const size_t ts = c->precision != MRA_FP64 ? sizeof(float) : sizeof(double);
    size_t s = 0;
    auto addT = [&](size_t elems) { s = align256(s + elems * (size_t)B * ts); };
    auto addD = [&](size_t elems) { s = align256(s + elems * (size_t)B * sizeof(double)); };
    addT(p.prior);
    addT(p.U);
    addD(p.leafw);
    addD(p.leafdu);
    addD(p.V);
    addT(p.Ain);
    addD(p.Ainw);
    addD(p.Aindu);
    s = align256(s + p.Gexp * (size_t)B);
    if (p.lbA > 0) {
        s = align256(s + p.lbA * (size_t)B);
        s = align256(s + p.lbB * (size_t)B);
    }
    for (int m = 2; m <= c->G.M - 1; m++) {
        addT(p.Atil[m]);
        addD(p.Atilw[m]);
        addD(p.Atildu[m]);
    }
    return s;
}

DevTree dev_tree(const mra_ctx *c)
{
    DevTree t;
    memset(&t, 0, sizeof(t));
    const Levels &G = c->G;
    t.M = G.M;
    t.RP = c->RP;
    t.n_used = c->P.n_used;
    t.kx = c->d_kx;
    t.ky = c->d_ky;
    t.cx = c->d_cx;
    t.cy = c->d_cy;
    t.sx = c->d_sx;
    t.sy = c->d_sy;
    t.sz = c->d_sz;
    t.leaf_off = c->d_leaf_off;
    for (int m = 0; m <= G.M + 1; m++) t.lvl_off[m] = G.lvl_off[(size_t)m];
    t.sh[1] = 0;
    for (int m = 1; m <= G.M; m++) {
        if (m < G.M) {
            t.Rl[m] = G.Rl[(size_t)m];
            t.Jl[m] = G.Jl[(size_t)m];
        }
        t.sh[m + 1] = t.sh[m] + (m < G.M ? G.lgJ(m) : 0);
    }
    return t;
}

enum { K_PRIOR, K_LEAFBASIS, K_LEAFPOST, K_LEAFPOST_BIG, K_LEAFGRAM, K_UP, K_ROOT, K_COUNT };
const char *kKernelNames[K_COUNT] = {"prior", "leafbasis", "leafpost", "leafpost_big", "leafgram", "up", "root"};

// Launch one kernel, bracketed by CUDA events when profiling is on.
template <typename F>
int timed_launch(mra_ctx *c, int kind, cudaStream_t s, F &&launch)
{
    if (!c->prof_on) {
        c->launches_last++;
        return launch();
    }
    if (c->ev_used + 2 > c->ev.size()) {
        for (int k = 0; k < 64; k++) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return (int)cudaErrorMemoryAllocation;
            c->ev.push_back(e);
        }
        c->ev_kind.resize(c->ev.size() / 2);
    }
    cudaEventRecord(c->ev[c->ev_used], s);
    const int rc = launch();
    cudaEventRecord(c->ev[c->ev_used + 1], s);
    c->ev_kind[c->ev_used / 2] = kind;
    c->ev_used += 2;
    c->launches_last++;
    return rc;
}

// The default leaf-basis kernel of a tree: the streaming one (16-row chunks,
// ancestor blocks staged two at a time) where 32-row chunks in one stage
// leave room for a single CTA per SM.
template <typename T, int RP>
bool leafbasis_streams(int M)
{
    return smem_leafbasis_cfg<T, RP>(M, 32, 1) > (size_t)112 * 1024;
}

template <typename T, int RP>
int run_pass(mra_ctx *c, const Work<T> &w, int B, cudaStream_t s)
{
    const DevTree t = dev_tree(c);
    const int M = c->G.M;
    int e;
    c->launches_last = 0;
    for (int m = 1; m < M; m++)
        if ((e = timed_launch(c, K_PRIOR, s, [&] { return launch_prior<T, RP>(t, w, m, B, c->prior_st, s); })))
            return e;
    int rows;
    if (c->lb_rows == kStreamRows || (c->lb_rows == 0 && leafbasis_streams<T, RP>(M))) {
        rows = kStreamRows; // the streaming kernel (deep trees)
    } else {
        rows = (sizeof(T) == 4 && c->lb_rows == 32) ? 32 : chunk_rows<T>();
        if (rows == 64 && !c->lb64_fits) rows = 32; // deep trees: 64-row chunks exceed shared memory
    }
    const Chunk *chunks = rows == 64 ? c->d_chunks64 : (rows == kStreamRows ? c->d_chunks16 : c->d_chunks32);
    const int nchunks = rows == 64 ? c->nchunks64 : (rows == kStreamRows ? c->nchunks16 : c->nchunks32);
    const bool lbtc = sizeof(T) == 4 && c->lb_tc && c->precision == MRA_MIXED;
    // the regions' short tails (at most half a chunk, listed last) run as
    // chunks of half the rows beside the full chunks, on a side stream
    const int ntail = (lbtc || c->lb_whole) ? 0 : (rows == 64 ? c->ntail64 : (rows == 32 ? c->ntail32 : 0));
    const int nmain = nchunks - ntail;
    // (a profiled pass runs them one after another, so that each kernel's
    // events time that kernel alone)
    const bool tail_side = ntail > 0 && nmain > 0 && c->concurrent && !c->prof_on;
    if (tail_side) {
        if (!c->lbt_fork && cudaEventCreateWithFlags(&c->lbt_fork, cudaEventDisableTiming) != cudaSuccess)
            return (int)cudaErrorLaunchFailure;
        if (!c->lbt_join && cudaEventCreateWithFlags(&c->lbt_join, cudaEventDisableTiming) != cudaSuccess)
            return (int)cudaErrorLaunchFailure;
        if (!c->aux[0] && cudaStreamCreateWithFlags(&c->aux[0], cudaStreamNonBlocking) != cudaSuccess)
            return (int)cudaErrorLaunchFailure;
        cudaEventRecord(c->lbt_fork, s);
    }
    if (M > 1 && nmain > 0)
        if ((e = timed_launch(c, K_LEAFBASIS, s, [&] {
                 return lbtc ? launch_leafbasis_tc<T, RP>(t, w, c->d_chunks128, c->nchunks128, B, s)
                             : launch_leafbasis<T, RP>(t, w, chunks, nmain, rows, c->lb_stages, B, s);
             })))
            return e;
    if (M > 1 && ntail > 0) {
        cudaStream_t q = tail_side ? c->aux[0] : s;
        if (tail_side) cudaStreamWaitEvent(q, c->lbt_fork, 0);
        if ((e = timed_launch(c, K_LEAFBASIS, q, [&] {
                 return launch_leafbasis_half<T, RP>(t, w, chunks + nmain, ntail, rows, c->lb_stages, B, q);
             })))
            return e;
        if (tail_side) {
            cudaEventRecord(c->lbt_join, q);
            cudaStreamWaitEvent(s, c->lbt_join, 0);
        }
    }
    // leaf posterior: the size buckets and the large-leaf pipeline touch
    // disjoint leaves, so they run concurrently: the large leaves (or the first
    // bucket) on s, every other bucket on a side stream forked from s
    int naux = 0;
    {
        // the launch list of this bucket set: (leaves, count, cap)
        const int64_t *lists[kLeafBuckets];
        int counts[kLeafBuckets], caps[kLeafBuckets];
        int nlist = 0;
        const bool merged = c->bucket_set == 1 && c->nmax_small >= 64;
        for (int k = 0; k < kLeafBuckets; k++) {
            if (merged && kLeafCap[k] > kLeafCap[0] && kLeafCap[k] < 64) continue;
            lists[nlist] = (merged && kLeafCap[k] == 64) ? c->d_leaves_m : c->d_leaves[k];
            counts[nlist] = (merged && kLeafCap[k] == 64) ? c->nl_m : c->nl[k];
            caps[nlist] = kLeafCap[k];
            nlist++;
        }
        int jobs = c->nbig > 0 ? 1 : 0;
        for (int k = 0; k < nlist; k++) jobs += counts[k] > 0;
        const bool fork = jobs > 1 && c->concurrent && !c->prof_on;
        if (fork) {
            if (!c->fork_ev && cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess)
                return (int)cudaErrorLaunchFailure;
            cudaEventRecord(c->fork_ev, s);
        }
        bool s_taken = c->nbig > 0;
        for (int k = 0; k < nlist; k++) {
            if (counts[k] == 0) continue;
            cudaStream_t q = s;
            if (fork && s_taken) {
                const int a = naux++;
                if (!c->aux[a] && cudaStreamCreateWithFlags(&c->aux[a], cudaStreamNonBlocking) != cudaSuccess)
                    return (int)cudaErrorLaunchFailure;
                if (!c->join_ev[a] && cudaEventCreateWithFlags(&c->join_ev[a], cudaEventDisableTiming) != cudaSuccess)
                    return (int)cudaErrorLaunchFailure;
                q = c->aux[a];
                cudaStreamWaitEvent(q, c->fork_ev, 0);
            }
            s_taken = true;
            unsigned *qc = c->leaf_queue ? c->d_qcnt + (size_t)k * c->status_cap : nullptr;
            if ((e = timed_launch(c, K_LEAFPOST, q, [&] {
                     return launch_leafpost_small<T, RP>(t, w, lists[k], counts[k], caps[k], B, qc, q);
                 })))
                return e;
        }
    }
    if (c->nbig > 0) {
        auto big = [&](int phase, int off, int cnt, int k) {
            return timed_launch(c, K_LEAFPOST_BIG, s, [&] {
                return launch_big<T, RP>(t, w, phase, c->d_big, c->d_bigitems + off, cnt, k, B, s);
            });
        };
        if ((e = big(BIG_ASSEMBLE, 0, c->big_nassemble, 0))) return e;
        for (int k = 0; k < (int)c->big_steps.size(); k++) {
            const auto &st = c->big_steps[(size_t)k];
            if ((e = big(BIG_POTRF, st[0], st[1], k))) return e;
            if (st[3] > 0 && (e = big(BIG_TRSM, st[2], st[3], k))) return e;
            if (st[5] > 0 && (e = big(BIG_UPDATE, st[4], st[5], k))) return e;
        }
        if ((e = timed_launch(c, K_LEAFPOST_BIG, s, [&] {
                 return launch_big<T, RP>(t, w, BIG_FINISH, c->d_big, nullptr, c->nbig, 0, B, s);
             })))
            return e;
    }
    // join the side streams back into s
    for (int a = 0; a < naux; a++) {
        cudaEventRecord(c->join_ev[a], c->aux[a]);
        cudaStreamWaitEvent(s, c->join_ev[a], 0);
    }
    if (M > 1 && c->sub_level > 0) {
        // subtree streaming: the Gram and the upward pass of levels M-1 .. S
        // chunk by chunk of level-S subtrees (contiguous at every level), into
        // arrays that hold one chunk; then levels S-1 .. 1 whole
        const int S = c->sub_level;
        auto nreg = [&](int m) { return c->G.lvl_off[(size_t)m + 1] - c->G.lvl_off[(size_t)m]; };
        const int64_t nS = nreg(S);
        const bool tc = sizeof(T) == 4 && c->gram_tc;
        for (int64_t q0 = 0; q0 < nS; q0 += c->sub_chunk) {
            const int64_t q = std::min<int64_t>(c->sub_chunk, nS - q0);
            const int64_t dP = nreg(M - 1) / nS;
            const int p0 = (int)(q0 * dP), cnt = (int)(q * dP);
            if (tc && (e = timed_launch(c, K_LEAFGRAM, s, [&] { return launch_gram_colexp<T, RP>(t, w, p0, cnt, B, s); })))
                return e;
            if ((e = timed_launch(c, K_LEAFGRAM, s, [&] { return launch_leafgram<T, RP>(t, w, p0, cnt, B, tc, s); })))
                return e;
            for (int m = M - 1; m >= S; m--) {
                const int64_t d = nreg(m) / nS;
                if ((e = timed_launch(c, K_UP, s,
                                      [&] { return launch_up<T, RP>(t, w, m, (int)(q0 * d), (int)(q * d), B, s); })))
                    return e;
            }
        }
        for (int m = S - 1; m >= 1; m--)
            if ((e = timed_launch(c, K_UP, s, [&] { return launch_up<T, RP>(t, w, m, 0, -1, B, s); }))) return e;
    } else if (M > 1) {
        const int nP = (int)(c->G.lvl_off[(size_t)M] - c->G.lvl_off[(size_t)M - 1]);
        const int chunk = c->ain_chunk > 0 ? c->ain_chunk : nP;
        for (int p0 = 0; p0 < nP; p0 += chunk) {
            const int cnt = std::min(chunk, nP - p0);
            const bool tc = sizeof(T) == 4 && c->gram_tc;
            if (tc && (e = timed_launch(c, K_LEAFGRAM, s, [&] { return launch_gram_colexp<T, RP>(t, w, p0, cnt, B, s); })))
                return e;
            if ((e = timed_launch(c, K_LEAFGRAM, s, [&] { return launch_leafgram<T, RP>(t, w, p0, cnt, B, tc, s); })))
                return e;
            if ((e = timed_launch(c, K_UP, s, [&] { return launch_up<T, RP>(t, w, M - 1, p0, cnt, B, s); })))
                return e;
        }
        for (int m = M - 1; m >= 1; m--)
            if (m < M - 1 && (e = timed_launch(c, K_UP, s, [&] { return launch_up<T, RP>(t, w, m, 0, -1, B, s); })))
                return e;
    } else {
        if ((e = timed_launch(c, K_ROOT, s, [&] { return launch_root_single<T, RP>(t, w, B, s); }))) return e;
    }
    return 0;
}

template <typename T>
int dispatch_rp(mra_ctx *c, const Work<T> &w, int B, cudaStream_t s)
{
    if (c->RP == 16) return run_pass<T, 16>(c, w, B, s);
    return run_pass<T, 32>(c, w, B, s);
}

// The largest dynamic shared memory one pass's kernels ask for with storage
// type T: leaf-basis chunks of 32 rows in one stage (the smallest
// configuration), the prior in two stages where they fit, leaf buckets up to
// nmax observations.
template <typename T, int RP>
size_t smem_need(int M, int nmax)
{
    size_t mx = 0;
    auto upd = [&](size_t v) { mx = std::max(mx, v); };
    for (int m = 1; m < M; m++) {
        upd(smem_prior<T, RP>(m));
        upd(smem_up<T, RP>(m));
    }
    upd(smem_big<T, RP>(M));
    upd(smem_leafgram<T, RP>(M));
    upd(std::min(smem_leafbasis_cfg<T, RP>(M, 32, 1), smem_leafbasis_cfg<T, RP>(M, kStreamRows, 1)));
    upd(smem_leafpost_small<T, RP>(M, 32));
    if (nmax > 0) upd(smem_leafpost_small<T, RP>(M, nmax));
    return mx;
}

size_t max_smem_needed(const mra_ctx *c, int nmax, bool fp64)
{
    const int M = c->G.M;
    if (fp64) return c->RP == 16 ? smem_need<double, 16>(M, nmax) : smem_need<double, 32>(M, nmax);
    return c->RP == 16 ? smem_need<float, 16>(M, nmax) : smem_need<float, 32>(M, nmax);
}

// Algorithmic FP operations of one evaluation per kernel family (r_hat, not
// the padding; symmetric products counted once; FMA = 2), and covariance
// evaluations.
void count_work(mra_ctx *c)
{
    // on the device levels: Rk[m] knots of a level-m region, S[m] the knots of
    // its ancestors (levels 1..m-1)
    const Levels &G = c->G;
    const Partition &P = c->P;
    const int M = G.M, J = P.J;
    std::vector<double> Rk((size_t)M + 1, 0.0), S((size_t)M + 1, 0.0);
    for (int m = 1; m <= M; m++) {
        if (m < M) Rk[(size_t)m] = G.Rl[(size_t)m];
        S[(size_t)m] = m > 1 ? S[(size_t)m - 1] + Rk[(size_t)m - 1] : 0.0;
    }
    double f[K_COUNT] = {0};
    double cv = 0.0;
    for (int m = 1; m < M; m++) {
        const double nr = (double)(G.lvl_off[(size_t)m + 1] - G.lvl_off[(size_t)m]);
        const double R = Rk[(size_t)m], Sm = S[(size_t)m];
        double per = 0.0;
        for (int l = 1; l < m; l++) {
            const double Rl = Rk[(size_t)l];
            per += 2.0 * S[(size_t)l] * R * Rl + R * Rl * Rl; // W^l and W^l Linv'
            cv += nr * R * Rl;
        }
        per += Sm * R * (R + 1) + 2.0 * R * R * R / 3.0; // self block, chol, inverse
        f[K_PRIOR] += nr * per;
        cv += nr * R * (R + 1) / 2;
        double upd = 0.0; // ATilde^{k,l} = A^{k,l} - Z_k' Z_l, k <= l < m
        for (int l = 1; l < m; l++) {
            upd += Rk[(size_t)l] * (Rk[(size_t)l] + 1) * R;
            for (int k = 1; k < l; k++) upd += 2.0 * Rk[(size_t)k] * Rk[(size_t)l] * R;
        }
        f[K_UP] += nr * (R * R * R / 3.0 + Sm * R * R + R * R + upd + 2.0 * Sm * R);
    }
    if (M > 1) {
        double perrow = 0.0, gram = 0.0;
        for (int l = 1; l < M; l++) {
            const double Rl = Rk[(size_t)l];
            perrow += 2.0 * S[(size_t)l] * Rl + Rl * Rl;
            gram += Rl * (Rl + 1);
            for (int k = 1; k < l; k++) gram += 2.0 * Rk[(size_t)k] * Rl;
        }
        const double SM = S[(size_t)M];
        f[K_LEAFBASIS] += (double)P.n_used * perrow;
        cv += (double)P.n_used * SM;
        const int64_t nP = G.lvl_off[(size_t)M] - G.lvl_off[(size_t)M - 1];
        for (int64_t p = 0; p < nP; p++) {
            const double N = (double)(P.leaf_off[(size_t)((p + 1) * J)] - P.leaf_off[(size_t)(p * J)]);
            f[K_LEAFGRAM] += N * gram + 2.0 * N * SM;
        }
    }
    const double SM = S[(size_t)M];
    for (int64_t l = 0; l < P.nleaf(); l++) {
        const double n = (double)(P.leaf_off[(size_t)l + 1] - P.leaf_off[(size_t)l]);
        const double fl = SM * n * (n + 1) + n * n * n / 3.0 + SM * n * n + n * n;
        if (n <= c->nmax_small || c->d_sx == nullptr)
            f[K_LEAFPOST] += fl;
        else
            f[K_LEAFPOST_BIG] += fl;
        cv += n * (n + 1) / 2;
    }
    double tot = 0.0;
    for (int k = 0; k < K_COUNT; k++) {
        c->flops_k[k] = f[k];
        tot += f[k];
    }
    c->flops = tot;
    c->covs = cv;
}

mra_status ensure_capacity(mra_ctx *c, int B)
{
    Plan p = make_plan(c);
    const size_t bytes = scratch_bytes_for(p, c, B);
    if (c->d_scratch && bytes <= c->scratch_bytes && B <= c->status_cap) {
        c->cap = B;
        return MRA_OK;
    }
    if (c->d_scratch) {
        cudaFree(c->d_scratch);
        c->bytes_held -= c->scratch_bytes;
        c->d_scratch = nullptr;
    }
    if (c->d_status) {
        cudaFree(c->d_status);
        c->d_status = nullptr;
    }
    cudaError_t e = cudaMalloc((void **)&c->d_scratch, bytes);
    if (e != cudaSuccess) {
        c->cap = 0;
        c->err = "cannot allocate per-theta scratch";
        return MRA_ENOMEM;
    }
    e = cudaMalloc((void **)&c->d_status, sizeof(int) * (size_t)B);
    if (e == cudaSuccess) {
        if (c->d_qcnt) cudaFree(c->d_qcnt);
        c->d_qcnt = nullptr;
        e = cudaMalloc((void **)&c->d_qcnt, sizeof(unsigned) * (size_t)kLeafBuckets * (size_t)B);
    }
    if (e != cudaSuccess) {
        cudaFree(c->d_scratch);
        c->d_scratch = nullptr;
        c->cap = 0;
        c->err = "cannot allocate status";
        return MRA_ENOMEM;
    }
    c->scratch_bytes = bytes;
    c->bytes_held += bytes;
    c->cap = B;
    c->status_cap = B;
    c->scratch_gen++;
    return MRA_OK;
}

// Theta per device pass for the current precision, and the Ain chunking:
// the level M-1 Gram blocks (the largest per-theta array on deep trees) are
// produced and consumed chunk by chunk only when one theta would not fit
// otherwise.
int max_batch_for(mra_ctx *c, size_t budget)
{
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)8 << 30;
        budget = (size_t)(0.6 * (double)(fr + c->scratch_bytes));
    }
    c->ain_chunk = 0;
    c->sub_level = 0;
    c->sub_chunk = 0;
    const int M = c->G.M;
    auto nreg = [&](int m) { return c->G.lvl_off[(size_t)m + 1] - c->G.lvl_off[(size_t)m]; };
    // bytes of one theta's scratch with subtree streaming below level S in
    // chunks of q level-S subtrees
    auto sub_bytes = [&](int S, int64_t q) {
        c->sub_level = S;
        c->sub_chunk = (int)q;
        const size_t v = scratch_bytes_for(make_plan(c), c, 1) + 4096;
        c->sub_level = 0;
        c->sub_chunk = 0;
        return v;
    };
    if (c->sub_req_level > 0 && M >= 3) {
        // forced (mra_set_launch): the requested level, the requested chunk or
        // the largest that fits the budget
        const int S = std::min(c->sub_req_level, M - 2);
        int64_t q = c->sub_req_chunk;
        if (q <= 0) {
            const size_t b1 = sub_bytes(S, 1), b2 = sub_bytes(S, 2);
            const size_t per_sub = b2 > b1 ? b2 - b1 : 1;
            q = budget > b1 ? 1 + (int64_t)((budget - b1) / per_sub) : 1;
        }
        c->sub_level = S;
        c->sub_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(q, nreg(S)));
    }
    Plan p = make_plan(c);
    size_t per = scratch_bytes_for(p, c, 1) + 4096;
    if (per > budget && M >= 3 && c->sub_level == 0) {
        // Where even one region's Ain leaves the scratch over the budget (the
        // ATilde arrays of deep trees grow with the tree, not with n), stream
        // subtrees: the level S whose chunks of the largest fitting size are
        // fewest, the deepest of those (fewer levels run chunked).
        c->ain_chunk = 1;
        const size_t ain1 = scratch_bytes_for(make_plan(c), c, 1) + 4096;
        c->ain_chunk = 0;
        if (ain1 > budget) {
            int bestS = 0;
            int64_t bestq = 0, bestn = 0;
            for (int S = M - 2; S >= 1; S--) {
                const size_t b1 = sub_bytes(S, 1);
                if (b1 > budget) continue;
                const size_t b2 = nreg(S) > 1 ? sub_bytes(S, 2) : b1 + 1;
                const size_t per_sub = b2 > b1 ? b2 - b1 : 1;
                const int64_t q = std::min<int64_t>(nreg(S), 1 + (int64_t)((budget - b1) / per_sub));
                const int64_t nch = (nreg(S) + q - 1) / q;
                if (bestS == 0 || nch < bestn) {
                    bestS = S;
                    bestq = q;
                    bestn = nch;
                }
            }
            if (bestS > 0) {
                c->sub_level = bestS;
                c->sub_chunk = (int)bestq;
                p = make_plan(c);
                per = scratch_bytes_for(p, c, 1) + 4096;
            }
        }
    }
    if (per > budget && M >= 2 && p.Ain > 0 && c->sub_level == 0) {
        const int64_t nP = c->G.lvl_off[(size_t)M] - c->G.lvl_off[(size_t)M - 1];
        const size_t full_ain = scratch_bytes_for(p, c, 1);
        c->ain_chunk = 1;
        const size_t base = scratch_bytes_for(make_plan(c), c, 1);
        const double per_region = (double)(full_ain - base) / (double)std::max<int64_t>(nP - 1, 1);
        const double room = (double)budget - (double)base - 4096.0;
        int64_t chunk = room > 0 ? (int64_t)(room / std::max(per_region, 1.0)) : 1;
        chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, nP));
        c->ain_chunk = (int)chunk;
        per = scratch_bytes_for(make_plan(c), c, 1) + 4096;
    }
    c->per_theta_bytes = per;
    size_t b = budget / per;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

// One device pass of B theta (theta_dev, loglik_dev, status_dev already
// offset to the pass) on stream s: clear the status, run the kernels, copy the
// status out.
mra_status pass_ops(mra_ctx *c, const double *theta_dev, int B, double *loglik_dev, int *status_dev, cudaStream_t s,
                    bool with_regions)
{
    c->pass_count++;
    Plan p = make_plan(c);
    cudaError_t e = cudaMemsetAsync(c->d_status, 0, sizeof(int) * (size_t)B, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    int rc;
    if (c->precision != MRA_FP64) {
        Work<float> w = make_work<float>(c, p, B);
        w.exact_rem = c->precision == MRA_MIXED;
        w.theta = theta_dev;
        w.loglik = loglik_dev;
        w.keep_up = c->keep_up;
        w.keep_up_stride = c->keep_stride;
        w.keep_li = (float *)c->keep_li;
        w.keep_y = c->keep_y;
        if (with_regions) {
            w.reg_du = c->d_reg_du;
            w.reg_lw = c->d_reg_lw;
        }
        rc = dispatch_rp<float>(c, w, B, s);
    } else {
        Work<double> w = make_work<double>(c, p, B);
        w.theta = theta_dev;
        w.loglik = loglik_dev;
        w.keep_up = c->keep_up;
        w.keep_up_stride = c->keep_stride;
        w.keep_li = (double *)c->keep_li;
        w.keep_y = c->keep_y;
        if (with_regions) {
            w.reg_du = c->d_reg_du;
            w.reg_lw = c->d_reg_lw;
        }
        rc = dispatch_rp<double>(c, w, B, s);
    }
    if (rc) return cuda_fail(c, (cudaError_t)rc, "kernel launch");
    if (status_dev) {
        e = cudaMemcpyAsync(status_dev, c->d_status, sizeof(int) * (size_t)B, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync");
    }
    return MRA_OK;
}

void drop_graphs(mra_ctx *c)
{
    for (auto &g : c->graph_cache) cudaGraphExecDestroy(g.exec);
    c->graph_cache.clear();
    c->graph_seen.clear();
}

// Replay a captured pass, or capture it when it comes for the second time (the
// first run also sets the kernels' shared-memory limits, which are not stream
// work); a pass seen for the first time runs without a graph.
mra_status graph_pass(mra_ctx *c, const double *theta_dev, int B, double *loglik_dev, int *status_dev,
                      cudaStream_t s, bool with_regions)
{
    c->pass_count++;
    const int regions = with_regions ? 1 : 0;
    auto same = [&](const mra_ctx::GraphEntry &g) {
        return g.theta == theta_dev && g.loglik == loglik_dev && g.status == status_dev && g.B == B &&
               g.precision == c->precision && g.regions == regions && g.gen == c->scratch_gen;
    };
    c->use_clock++;
    for (auto &g : c->graph_cache)
        if (same(g)) {
            g.last_use = c->use_clock;
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
            return MRA_OK;
        }
    bool seen = false;
    for (auto &g : c->graph_seen)
        if (same(g)) seen = true;
    if (!seen) {
        if (c->graph_seen.size() >= 64) c->graph_seen.erase(c->graph_seen.begin());
        c->graph_seen.push_back(mra_ctx::GraphEntry{theta_dev, loglik_dev, status_dev, B, c->precision, regions,
                                                    c->scratch_gen, 0, nullptr});
        return pass_ops(c, theta_dev, B, loglik_dev, status_dev, s, with_regions);
    }
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreate");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    mra_status st = pass_ops(c, theta_dev, B, loglik_dev, status_dev, c->cap_stream, with_regions);
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != MRA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    if (c->graph_cache.size() >= 16) {
        size_t old = 0;
        for (size_t k = 1; k < c->graph_cache.size(); k++)
            if (c->graph_cache[k].last_use < c->graph_cache[old].last_use) old = k;
        cudaGraphExecDestroy(c->graph_cache[old].exec);
        c->graph_cache.erase(c->graph_cache.begin() + (long)old);
    }
    c->graph_cache.push_back(mra_ctx::GraphEntry{theta_dev, loglik_dev, status_dev, B, c->precision, regions,
                                                 c->scratch_gen, c->use_clock, exec});
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    return MRA_OK;
}

mra_status enqueue(mra_ctx *c, const double *theta_dev, int batch, double *loglik_dev, int *status_dev,
                   cudaStream_t s, bool with_regions)
{
    int done = 0;
    while (done < batch) {
        const int B = std::min(batch - done, std::max(c->max_cap, 1));
        if (mra_status st = ensure_capacity(c, B)) return st;
        const double *th = theta_dev + 3 * (size_t)done;
        double *ll = loglik_dev + done;
        int *sd = status_dev ? status_dev + done : nullptr;
        mra_status st = (c->graphs && !c->prof_on && !with_regions) ? graph_pass(c, th, B, ll, sd, s, false)
                                                                    : pass_ops(c, th, B, ll, sd, s, with_regions);
        if (st != MRA_OK) return st;
        done += B;
    }
    return MRA_OK;
}

mra_status ensure_stage(mra_ctx *c, int batch)
{
    if (batch <= c->stage_cap) return MRA_OK;
    cudaFree(c->d_theta_stage);
    cudaFree(c->d_ll_stage);
    c->d_theta_stage = nullptr;
    c->d_ll_stage = nullptr;
    if (cudaMalloc((void **)&c->d_theta_stage, sizeof(double) * 3 * (size_t)batch) != cudaSuccess ||
        cudaMalloc((void **)&c->d_ll_stage, sizeof(double) * (size_t)batch + sizeof(int) * (size_t)batch) !=
            cudaSuccess) {
        c->stage_cap = 0;
        c->err = "cannot allocate theta staging";
        return MRA_ENOMEM;
    }
    c->stage_cap = batch;
    return MRA_OK;
}

// Leaf of a location by the descent build_partition bins observations with;
// -1 outside the root box.
int64_t leaf_of(const Partition &P, double a, double b)
{
    if (!(a >= P.bx0[0] && a < P.bx1[0] && b >= P.by0[0] && b < P.by1[0])) return -1;
    int64_t i = 0;
    for (int m = 1; m < P.M; m++) {
        const int64_t g = P.lvl_off[(size_t)m] + i;
        const double mx = 0.5 * (P.bx0[(size_t)g] + P.bx1[(size_t)g]);
        const double my = 0.5 * (P.by0[(size_t)g] + P.by1[(size_t)g]);
        int j;
        if (P.J == 4)
            j = (a >= mx) | ((b >= my) << 1);
        else
            j = P.cut_x[(size_t)m] ? (a >= mx) : (b >= my);
        i = i * P.J + j;
    }
    return i;
}

// Grow-only device buffer of the prediction state.
bool pred_reserve(unsigned char **buf, size_t *have, size_t need)
{
    if (need <= *have) return true;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc((void **)buf, need) != cudaSuccess) {
        *buf = nullptr;
        return false;
    }
    *have = need;
    return true;
}

// Clears the pointers the kernels keep factors through, on every exit.
struct KeepGuard {
    mra_ctx *c;
    ~KeepGuard()
    {
        c->keep_up = c->keep_y = nullptr;
        c->keep_li = nullptr;
        c->keep_stride = 0;
    }
};

// Prediction for storage type T: the likelihood pass at theta keeping the
// factors and the downward pass (both skipped while the factors of the last
// call still hold), the basis at the points (the leaf-basis kernel on a tree
// view whose observation rows are the points) and one warp per point.
// Points come grouped by leaf (sx, sy, sl sorted the same way).
template <typename T, int RP>
mra_status predict_impl(mra_ctx *c, const double *theta, const std::vector<double> &sx,
                        const std::vector<double> &sy, const std::vector<int64_t> &sl, double *mean_out,
                        double *var_out)
{
    const Levels &G = c->G;
    const int M = G.M;
    const int64_t np = (int64_t)sx.size(), NK = G.nnonleaf(), NL = G.nleaf();
    const int UC = (M - 1) * RP;
    const size_t stride = keep_up_doubles(M, RP);
    KeepGuard guard{c};
    // per-tree buffers: keep_up, L^{-1} and y of the leaves, xi, leaf -> large-leaf index
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_keep = carve(sizeof(double) * (size_t)std::max<int64_t>(NK, 1) * stride);
    const size_t o_li = carve(sizeof(T) * (size_t)NL * kKeepLd * kKeepLd);
    const size_t o_ky = carve(sizeof(double) * (size_t)NL * kKeepLd);
    const size_t o_xi = carve(sizeof(double) * (size_t)std::max<int64_t>(NK, 1) * RP);
    const size_t o_bi = carve(sizeof(int32_t) * (size_t)NL);
    const size_t tree_need = off;
    if (tree_need > c->pred.tree_bytes) c->pred.valid = false;
    if (!pred_reserve(&c->pred.tree, &c->pred.tree_bytes, tree_need)) {
        c->err = "cannot allocate the prediction buffers";
        return MRA_ENOMEM;
    }
    double *d_keep = (double *)(c->pred.tree + o_keep);
    T *d_li = (T *)(c->pred.tree + o_li);
    double *d_ky = (double *)(c->pred.tree + o_ky);
    double *d_xi = (double *)(c->pred.tree + o_xi);
    int32_t *d_bigidx = (int32_t *)(c->pred.tree + o_bi);
    // per-point buffers
    const int rows = (chunk_rows<T>() == 64 && !c->lb64_fits) ? 32 : chunk_rows<T>();
    std::vector<Chunk> chunks;
    if (M > 1)
        for (int64_t k = 0; k < np; k++) {
            if (sl[(size_t)k] < 0) continue;
            const int32_t parent = (int32_t)(sl[(size_t)k] >> c->lgJ);
            if (chunks.empty() || chunks.back().parent != parent || chunks.back().n == rows)
                chunks.push_back(Chunk{parent, 0, k});
            chunks.back().n++;
        }
    off = 0;
    const size_t o_px = carve(sizeof(double) * (size_t)np), o_py = carve(sizeof(double) * (size_t)np);
    const size_t o_lf = carve(sizeof(int64_t) * (size_t)np);
    const size_t o_mn = carve(sizeof(double) * (size_t)np), o_vr = carve(sizeof(double) * (size_t)np);
    const size_t o_ua = carve(sizeof(T) * (size_t)np * (size_t)std::max(UC, 1));
    const size_t o_ch = carve(sizeof(Chunk) * chunks.size());
    if (!pred_reserve(&c->pred.pt, &c->pred.pt_bytes, off)) {
        c->err = "cannot allocate the prediction buffers";
        return MRA_ENOMEM;
    }
    double *d_px = (double *)(c->pred.pt + o_px), *d_py = (double *)(c->pred.pt + o_py);
    int64_t *d_leaf = (int64_t *)(c->pred.pt + o_lf);
    double *d_mean = (double *)(c->pred.pt + o_mn), *d_var = (double *)(c->pred.pt + o_vr);
    T *d_ua = (T *)(c->pred.pt + o_ua);
    Chunk *d_chunks = (Chunk *)(c->pred.pt + o_ch);
    cudaError_t e = cudaMemcpy(d_px, sx.data(), sizeof(double) * (size_t)np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_py, sy.data(), sizeof(double) * (size_t)np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_leaf, sl.data(), sizeof(int64_t) * (size_t)np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !chunks.empty())
        e = cudaMemcpy(d_chunks, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_theta_stage, theta, sizeof(double) * 3, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "prediction upload");
    const DevTree t = dev_tree(c);
    int *d_st = (int *)(c->d_ll_stage + 1);
    const bool reuse = c->pred.valid && c->pred.precision == c->precision && c->pred.gen == c->scratch_gen &&
                       c->pred.pass_id == c->pass_count && memcmp(c->pred.theta, theta, sizeof(c->pred.theta)) == 0;
    int rc = 0;
    if (!reuse) {
        c->pred.valid = false;
        // leaf -> large-leaf index
        std::vector<int32_t> bigidx((size_t)NL, -1);
        if (c->nbig > 0) {
            std::vector<BigLeaf> hb((size_t)c->nbig);
            if (cudaMemcpy(hb.data(), c->d_big, sizeof(BigLeaf) * hb.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
                c->err = "cannot read the large-leaf list";
                return MRA_ECUDA;
            }
            for (int k = 0; k < c->nbig; k++) bigidx[(size_t)hb[(size_t)k].leaf] = k;
        }
        e = cudaMemcpy(d_bigidx, bigidx.data(), sizeof(int32_t) * (size_t)NL, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "prediction upload");
        // the likelihood pass, keeping the factors
        c->keep_up = d_keep;
        c->keep_stride = stride;
        c->keep_li = d_li;
        c->keep_y = d_ky;
        if (mra_status st = pass_ops(c, c->d_theta_stage, 1, c->d_ll_stage, d_st, (cudaStream_t)0, false)) return st;
        c->keep_up = c->keep_y = nullptr;
        c->keep_li = nullptr;
        for (int m = 1; m < M && !rc; m++) rc = launch_down<RP>(t, d_keep, stride, d_xi, m, nullptr);
    }
    const Plan plan = make_plan(c);
    Work<T> w = make_work<T>(c, plan, 1);
    w.theta = c->d_theta_stage;
    w.loglik = c->d_ll_stage;
    w.exact_rem = c->precision == MRA_MIXED;
    w.keep_li = d_li;
    w.keep_y = d_ky;
    if (!rc && !chunks.empty()) {
        DevTree tp = t;
        tp.sx = d_px;
        tp.sy = d_py;
        Work<T> wp = w;
        wp.U = d_ua;
        wp.U_stride = 0;
        rc = launch_leafbasis<T, RP>(tp, wp, d_chunks, (int)chunks.size(), rows, c->lb_stages, 1, nullptr);
    }
    if (!rc) {
        PredArgs q;
        memset(&q, 0, sizeof(q));
        q.np = np;
        q.px = d_px;
        q.py = d_py;
        q.leaf = d_leaf;
        q.Ua = d_ua;
        q.xi = d_xi;
        q.keep_up = d_keep;
        q.keep_stride = stride;
        q.bigidx = d_bigidx;
        q.big = c->d_big;
        q.mean = d_mean;
        q.var = d_var;
        q.nl = (int)std::max<int64_t>(c->max_leaf, 1);
        const size_t per_warp = predict_warp_doubles(M, RP, q.nl) * sizeof(double);
        if (per_warp > 200 * 1024) {
            c->err = "largest leaf too large for the prediction kernel";
            return MRA_EINVAL;
        }
        q.wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (160 * 1024) / per_warp));
        rc = launch_predict<T, RP>(t, w, q, nullptr);
    }
    if (rc) return cuda_fail(c, (cudaError_t)rc, "prediction launch");
    int hs = 0;
    e = cudaMemcpy(&hs, d_st, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mean_out, d_mean, sizeof(double) * (size_t)np, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(var_out, d_var, sizeof(double) * (size_t)np, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "prediction readback");
    if (hs != MRA_OK) {
        c->err = "Cholesky factor not positive definite";
        return (mra_status)hs;
    }
    if (!reuse) {
        memcpy(c->pred.theta, theta, sizeof(c->pred.theta));
        c->pred.precision = c->precision;
        c->pred.gen = c->scratch_gen;
        c->pred.pass_id = c->pass_count;
        c->pred.valid = true;
    }
    return MRA_OK;
}

} // namespace

// Reason of the calling thread's last failure that has no context to hold it
// (mra_build, mra_dense_loglik_noalloc); read through mra_last_error(NULL).
static thread_local std::string g_build_err = "no context";

namespace mra {
void set_thread_error(const std::string &msg) { g_build_err = msg; }
} // namespace mra

// ---------------------------------------------------------------- C ABI --
extern "C" {

void mra_default_opts(mra_opts *opt)
{
    if (!opt) return;
    opt->offset = -1.0;
    opt->dedup = 0;
    opt->precision = MRA_FP64;
    opt->device = 0;
    opt->max_batch = 0;
    opt->hbm_budget = 0;
    opt->graphs = 1;
}


static mra_status build_ctx(const double *lon, const double *lat, const double *z, int64_t n, int M, int J, int r,
                            const mra_opts *opt_in, mra_ctx **out);

mra_status mra_build(const double *lon, const double *lat, const double *z, int64_t n, int M, int J, int r,
                     const mra_opts *opt_in, mra_ctx **out)
{
    if (!out) return MRA_EINVAL;
    *out = nullptr;
    mra_ctx *c = nullptr;
    mra_status st = build_ctx(lon, lat, z, n, M, J, r, opt_in, &c);
    if (st != MRA_OK) {
        g_build_err = c ? c->err : std::string("out of host memory");
        mra_free(c);
        return st;
    }
    *out = c;
    return MRA_OK;
}

static mra_status build_ctx(const double *lon, const double *lat, const double *z, int64_t n, int M, int J, int r,
                            const mra_opts *opt_in, mra_ctx **out)
{
    if (n > 0 && (!lon || !lat || !z)) return MRA_EINVAL;
    mra_opts opt;
    mra_default_opts(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.precision != MRA_FP64 && opt.precision != MRA_MIXED && opt.precision != MRA_MIXED_FAST) return MRA_EINVAL;
    mra_ctx *c = new (std::nothrow) mra_ctx();
    if (!c) return MRA_ENOMEM;
    *out = c;
    c->precision = opt.precision;
    c->device = opt.device;
    const double f = opt.offset < 0.0 ? kDefaultOffset : opt.offset;
    mra_status st = build_partition(lon, lat, z, n, M, J, r, f, opt.dedup, c->P, c->err);
    if (st != MRA_OK) return st;
    const Partition &P = c->P;
    st = make_levels(P, c->G, c->err);
    if (st != MRA_OK) {
        *out = c;
        return st;
    }
    c->RP = c->G.RP;
    c->lgJ = J == 4 ? 2 : 1;
    if (opt.device < 0) { // host-only partition: stats and tree queries, no likelihood
        for (int64_t l = 0; l < P.nleaf(); l++) {
            const int64_t nl = P.leaf_off[(size_t)l + 1] - P.leaf_off[(size_t)l];
            c->max_leaf = std::max(c->max_leaf, nl);
            c->empty_leaves += nl == 0;
        }
        count_work(c);
        return MRA_OK;
    }
    cudaError_t e = cudaSetDevice(opt.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    // work lists
    std::vector<Chunk> chunks32, chunks64, chunks128, chunks16;
    if (M > 1) {
        const int64_t nP = P.lvl_off[(size_t)M] - P.lvl_off[(size_t)M - 1];
        for (int64_t p = 0; p < nP; p++) {
            const int64_t r0 = P.leaf_off[(size_t)(p * J)], r1 = P.leaf_off[(size_t)((p + 1) * J)];
            for (int rows : {32, 64, kLeafBasisTcRows, kStreamRows}) {
                std::vector<Chunk> &dst =
                    rows == 32 ? chunks32 : (rows == 64 ? chunks64 : (rows == kStreamRows ? chunks16 : chunks128));
                for (int64_t rb = r0; rb < r1; rb += rows) {
                    Chunk ch;
                    ch.parent = (int32_t)p;
                    ch.n = (int32_t)std::min<int64_t>(rows, r1 - rb);
                    ch.row0 = rb;
                    dst.push_back(ch);
                }
            }
        }
    }
    // a region's last chunk of at most half the rows (the padding of a 32- or
    // 64-row chunk otherwise) goes to the end of its list, where the launcher
    // runs it as a chunk of half the rows
    auto tails_last = [](std::vector<Chunk> &v, int rows) {
        std::stable_partition(v.begin(), v.end(), [rows](const Chunk &ch) { return 2 * ch.n > rows; });
        return (int)std::count_if(v.begin(), v.end(), [rows](const Chunk &ch) { return 2 * ch.n <= rows; });
    };
    c->ntail32 = tails_last(chunks32, 32);
    c->ntail64 = tails_last(chunks64, 64);
    // The leaf buckets are sized where the FP64 kernels fit (they take twice
    // the bytes); on trees too deep for them only the mixed modes run.
    c->fp64_fits = max_smem_needed(c, kLeafCap[0], true) <= kSmemMax;
    const bool f64 = c->fp64_fits;
    int kcap = kLeafBuckets - 1;
    while (kcap > 0 && max_smem_needed(c, kLeafCap[kcap], f64) > kSmemMax) kcap--;
    const int nmax_small = kLeafCap[kcap];
    if (max_smem_needed(c, nmax_small, f64) > kSmemMax) {
        c->err = "M too large for the shared-memory kernels at this r";
        *out = c;
        return MRA_EINVAL;
    }
    if (!f64 && c->precision == MRA_FP64) {
        c->err = "tree too deep for the FP64 shared-memory kernels at this r; build in a mixed precision";
        *out = c;
        return MRA_EINVAL;
    }
    c->nmax_small = nmax_small;
    c->lb64_fits = (c->RP == 16 ? smem_leafbasis_cfg<float, 16>(c->G.M, 64, 1)
                                : smem_leafbasis_cfg<float, 32>(c->G.M, 64, 1)) <= kSmemMax;
    std::vector<int64_t> lb[kLeafBuckets];
    std::vector<BigLeaf> big;
    int64_t voff = 0;
    for (int64_t l = 0; l < P.nleaf(); l++) {
        const int64_t nl = P.leaf_off[(size_t)l + 1] - P.leaf_off[(size_t)l];
        c->max_leaf = std::max(c->max_leaf, nl);
        if (nl == 0) {
            c->empty_leaves++;
        } else if (nl <= nmax_small) {
            int k = 0;
            while (nl > kLeafCap[k]) k++;
            lb[k].push_back(l);
        } else {
            big.push_back(BigLeaf{l, voff});
            voff += big_leaf_scratch(nl);
        }
    }
    c->vbig_elems = voff;
    // bucket set 1: the leaves of every bucket above the first as one list
    std::vector<int64_t> lbm;
    for (int64_t l = 0; l < P.nleaf(); l++) {
        const int64_t nl = P.leaf_off[(size_t)l + 1] - P.leaf_off[(size_t)l];
        if (nl > kLeafCap[0] && nl <= nmax_small) lbm.push_back(l);
    }
    // largest leaves first within each list (the block scheduler starts CTAs
    // in index order, so the longest leaves do not form the tail; the
    // dynamic-scheduling idea of Sec. 4.1, cost ~ n^2 and up, inside one GPU)
    auto by_size = [&](std::vector<int64_t> &v) {
        std::stable_sort(v.begin(), v.end(), [&](int64_t a, int64_t b) {
            return P.leaf_off[(size_t)a + 1] - P.leaf_off[(size_t)a] > P.leaf_off[(size_t)b + 1] - P.leaf_off[(size_t)b];
        });
    };
    for (int k = 0; k < kLeafBuckets; k++) by_size(lb[k]);
    by_size(lbm);
    // tiled large-leaf work lists
    std::vector<BigTile> items;
    {
        int ntmax = 0;
        for (const BigLeaf &bl : big) {
            const int64_t nl = P.leaf_off[(size_t)bl.leaf + 1] - P.leaf_off[(size_t)bl.leaf];
            ntmax = std::max(ntmax, (int)((nl + kBigTile - 1) / kBigTile));
        }
        auto ntiles = [&](size_t q) {
            const int64_t nl = P.leaf_off[(size_t)big[q].leaf + 1] - P.leaf_off[(size_t)big[q].leaf];
            return (int)((nl + kBigTile - 1) / kBigTile);
        };
        for (size_t q = 0; q < big.size(); q++)
            for (int i = 0; i < ntiles(q); i++)
                for (int j = 0; j <= i; j++) items.push_back(BigTile{(int32_t)q, i, j, 0});
        c->big_nassemble = (int)items.size();
        c->big_steps.clear();
        for (int k = 0; k < ntmax; k++) {
            std::array<int, 6> st{};
            st[0] = (int)items.size();
            for (size_t q = 0; q < big.size(); q++)
                if (ntiles(q) > k) items.push_back(BigTile{(int32_t)q, k, k, 0});
            st[1] = (int)items.size() - st[0];
            st[2] = (int)items.size();
            for (size_t q = 0; q < big.size(); q++)
                for (int i = k + 1; i < ntiles(q); i++) items.push_back(BigTile{(int32_t)q, i, k, 0});
            st[3] = (int)items.size() - st[2];
            st[4] = (int)items.size();
            for (size_t q = 0; q < big.size(); q++)
                for (int i = k + 1; i < ntiles(q); i++)
                    for (int j = k + 1; j <= i; j++) items.push_back(BigTile{(int32_t)q, i, j, 0});
            st[5] = (int)items.size() - st[4];
            c->big_steps.push_back(st);
        }
    }
    // device levels: knots padded to RP, region corners
    const Levels &G = c->G;
    if ((st = dev_upload(c, &c->d_kx, G.kx.data(), G.kx.size())) || (st = dev_upload(c, &c->d_ky, G.ky.data(), G.ky.size())) ||
        (st = dev_upload(c, &c->d_cx, G.cx.data(), G.cx.size())) || (st = dev_upload(c, &c->d_cy, G.cy.data(), G.cy.size())) ||
        (st = dev_upload(c, &c->d_sx, P.sx.data(), P.sx.size())) || (st = dev_upload(c, &c->d_sy, P.sy.data(), P.sy.size())) ||
        (st = dev_upload(c, &c->d_sz, P.sz.data(), P.sz.size())) ||
        (st = dev_upload(c, &c->d_leaf_off, P.leaf_off.data(), P.leaf_off.size())) ||
        (st = dev_upload(c, &c->d_chunks32, chunks32.data(), chunks32.size())) ||
        (st = dev_upload(c, &c->d_chunks64, chunks64.data(), chunks64.size())) ||
        (st = dev_upload(c, &c->d_chunks128, chunks128.data(), chunks128.size())) ||
        (st = dev_upload(c, &c->d_chunks16, chunks16.data(), chunks16.size())) ||
        (st = dev_upload(c, &c->d_leaves[0], lb[0].data(), lb[0].size())) ||
        (st = dev_upload(c, &c->d_leaves[1], lb[1].data(), lb[1].size())) ||
        (st = dev_upload(c, &c->d_leaves[2], lb[2].data(), lb[2].size())) ||
        (st = dev_upload(c, &c->d_leaves[3], lb[3].data(), lb[3].size())) ||
        (st = dev_upload(c, &c->d_leaves_m, lbm.data(), lbm.size())) ||
        (st = dev_upload(c, &c->d_big, big.data(), big.size())) ||
        (st = dev_upload(c, &c->d_bigitems, items.data(), items.size()))) {
        *out = c;
        return st;
    }
    c->nchunks32 = (int)chunks32.size();
    c->nchunks64 = (int)chunks64.size();
    c->nchunks128 = (int)chunks128.size();
    c->nchunks16 = (int)chunks16.size();
    for (int k = 0; k < kLeafBuckets; k++) c->nl[k] = (int)lb[k].size();
    c->nl_m = (int)lbm.size();
    c->nbig = (int)big.size();
    count_work(c);
    c->hbm_budget = opt.hbm_budget;
    c->graphs = opt.graphs != 0;
    c->user_max_batch = opt.max_batch;
    const int mb = max_batch_for(c, opt.hbm_budget);
    c->max_cap = opt.max_batch > 0 ? std::min(opt.max_batch, 1024) : mb;
    st = ensure_capacity(c, 1);
    if (st != MRA_OK) {
        *out = c;
        return st;
    }
    *out = c;
    return MRA_OK;
}

mra_status mra_autotune(mra_ctx *c, const double *theta, int reps, mra_tune_t *out)
{
    if (!c || !theta || reps < 1) return MRA_EINVAL;
    if (!c->d_sx) {
        c->err = "context was built without a device";
        return MRA_EINVAL;
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (mra_status st = ensure_stage(c, 1)) return st;
    e = cudaMemcpy(c->d_theta_stage, theta, 3 * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy theta");
    struct Cfg {
        int rows, stages, set;
        bool conc, queue;
        int prior;
    };
    const bool mixed = c->precision != MRA_FP64;
    const int RP = c->RP, M = c->G.M;
    auto smem_ok = [&](int rows, int stages) {
        size_t b;
        if (mixed)
            b = RP == 16 ? smem_leafbasis_cfg<float, 16>(M, rows, stages) : smem_leafbasis_cfg<float, 32>(M, rows, stages);
        else
            b = RP == 16 ? smem_leafbasis_cfg<double, 16>(M, rows, stages) : smem_leafbasis_cfg<double, 32>(M, rows, stages);
        return b <= kSmemMax;
    };
    std::vector<Cfg> cand;
    const Cfg start{c->lb_rows, c->lb_stages, c->bucket_set, c->concurrent, c->leaf_queue, c->prior_st};
    cand.push_back(start);
    for (int rows : {64, 32, kStreamRows}) {
        if (rows == 64 && !mixed) continue;
        for (int stages : {1, 2}) {
            if (rows == kStreamRows && stages == 2) continue; // stages do not apply to the streaming kernel
            if (!smem_ok(rows, stages)) continue;
            for (int set : {0, 1}) {
                if (set == 1 && c->nmax_small < 64) continue;
                for (bool conc : {true, false})
                    for (bool queue : {false, true}) cand.push_back(Cfg{rows, stages, set, conc, queue, start.prior});
            }
        }
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        if (st) cudaStreamDestroy(st);
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaErrorMemoryAllocation, "autotune stream");
    }
    auto apply = [&](const Cfg &g) {
        c->lb_rows = g.rows;
        c->lb_stages = g.stages;
        c->bucket_set = g.set;
        c->concurrent = g.conc;
        c->leaf_queue = g.queue;
        c->prior_st = g.prior;
        drop_graphs(c); // the pass changes
    };
    double best = 1e300, first = 0.0;
    Cfg bestc = start;
    mra_status rs = MRA_OK;
    int tried = 0;
    // mean pass time of one candidate (2 untimed passes, then reps timed)
    auto time_one = [&](const Cfg &g, double &per) {
        apply(g);
        for (int w = 0; w < 2 && rs == MRA_OK; w++)
            rs = enqueue(c, c->d_theta_stage, 1, c->d_ll_stage, nullptr, st, false);
        if (rs != MRA_OK) return false;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rs == MRA_OK; r++)
            rs = enqueue(c, c->d_theta_stage, 1, c->d_ll_stage, nullptr, st, false);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rs = cuda_fail(c, cudaGetLastError(), "autotune timing");
        if (rs != MRA_OK) return false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        per = (double)ms / reps;
        tried++;
        return true;
    };
    // the leaf-side candidates, then the prior's staging (a kernel of its
    // own) on the best of them
    for (size_t q = 0; q < cand.size(); q++) {
        double per = 0.0;
        if (!time_one(cand[q], per)) break;
        if (q == 0) first = per;
        if (per < best) {
            best = per;
            bestc = cand[q];
        }
    }
    const Cfg lead = bestc;
    for (int ps : {0, 1, 2, 3}) {
        if (rs != MRA_OK || ps == lead.prior) continue;
        Cfg g = lead;
        g.prior = ps;
        double per = 0.0;
        if (!time_one(g, per)) break;
        if (per < best) {
            best = per;
            bestc = g;
        }
    }
    apply(rs == MRA_OK ? bestc : start);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rs != MRA_OK) return rs;
    if (out) {
        const bool streams = mixed ? (RP == 16 ? leafbasis_streams<float, 16>(M) : leafbasis_streams<float, 32>(M))
                                   : (RP == 16 ? leafbasis_streams<double, 16>(M) : leafbasis_streams<double, 32>(M));
        out->leafbasis_rows = bestc.rows > 0 ? bestc.rows : (streams ? kStreamRows : ((mixed && c->lb64_fits) ? 64 : 32));
        int stages = bestc.stages;
        if (out->leafbasis_rows == kStreamRows) stages = 1;
        if (stages == 0) { // the automatic rule of the launcher
            const int r = out->leafbasis_rows;
            const size_t b2 = mixed ? (RP == 16 ? smem_leafbasis_cfg<float, 16>(M, r, 2) : smem_leafbasis_cfg<float, 32>(M, r, 2))
                                    : (RP == 16 ? smem_leafbasis_cfg<double, 16>(M, r, 2) : smem_leafbasis_cfg<double, 32>(M, r, 2));
            stages = b2 <= (size_t)110 * 1024 ? 2 : 1;
        }
        out->leafbasis_stages = stages;
        out->bucket_set = bestc.set;
        out->concurrent = bestc.conc ? 1 : 0;
        out->gram_tensor_cores = c->gram_tc ? 1 : 0;
        out->leafbasis_tensor_cores = c->lb_tc ? 1 : 0;
        out->leaf_queue = bestc.queue ? 1 : 0;
        out->leafbasis_whole_chunks = c->lb_whole ? 1 : 0;
        out->prior_stages = bestc.prior;
        out->subtree_level = c->sub_req_level;
        out->subtree_chunk = c->sub_req_chunk;
        out->ms_default = first;
        out->ms_best = best;
        out->tried = tried;
    }
    return MRA_OK;
}

mra_status mra_set_launch(mra_ctx *c, const mra_tune_t *g)
{
    if (!c || !g) return MRA_EINVAL;
    const bool mixed = c->precision != MRA_FP64;
    const int rows = g->leafbasis_rows, stages = g->leafbasis_stages;
    if (!(rows == 0 || rows == 32 || rows == kStreamRows || (rows == 64 && mixed)) || stages < 0 || stages > 2 ||
        g->bucket_set < 0 ||
        g->bucket_set > 1 || (g->bucket_set == 1 && c->nmax_small < 64) || g->prior_stages < 0 ||
        g->prior_stages > 3) {
        c->err = "launch configuration outside the candidates";
        return MRA_EINVAL;
    }
    if (g->subtree_level < 0 || g->subtree_chunk < 0 || (g->subtree_level > 0 && g->subtree_level > c->G.M - 2)) {
        c->err = "subtree_level must be 0 (chosen by the memory plan) or a device level in 1 .. device levels - 2";
        return MRA_EINVAL;
    }
    if (g->leafbasis_tensor_cores && (c->G.M - 2) * c->RP > kLeafBasisTcMaxK) {
        c->err = "tensor-core leaf basis: (M - 2) x padded r_hat must not exceed 192 (exact sums)";
        return MRA_EINVAL;
    }
    if (stages > 0) {
        const int r = rows > 0 ? rows : (mixed ? 64 : 32), RP = c->RP, M = c->G.M;
        size_t b;
        if (mixed)
            b = RP == 16 ? smem_leafbasis_cfg<float, 16>(M, r, stages) : smem_leafbasis_cfg<float, 32>(M, r, stages);
        else
            b = RP == 16 ? smem_leafbasis_cfg<double, 16>(M, r, stages) : smem_leafbasis_cfg<double, 32>(M, r, stages);
        if (b > kSmemMax) {
            c->err = "leaf-basis stages do not fit in shared memory";
            return MRA_EINVAL;
        }
    }
    c->lb_rows = rows;
    c->lb_stages = stages;
    c->bucket_set = g->bucket_set;
    c->concurrent = g->concurrent != 0;
    c->gram_tc = g->gram_tensor_cores != 0;
    const bool sub_change = g->subtree_level != c->sub_req_level || g->subtree_chunk != c->sub_req_chunk;
    c->sub_req_level = g->subtree_level;
    c->sub_req_chunk = g->subtree_level > 0 ? g->subtree_chunk : 0;
    if ((g->leafbasis_tensor_cores != 0) != c->lb_tc || sub_change) {
        c->lb_tc = g->leafbasis_tensor_cores != 0;
        if (c->d_sx) {
            // the slice buffers join or leave the per-theta scratch, or its
            // chunk-local arrays change size
            const int mb = max_batch_for(c, c->hbm_budget);
            c->max_cap = c->user_max_batch > 0 ? std::min(c->user_max_batch, 1024) : mb;
            c->cap = 0;
        }
    }
    c->leaf_queue = g->leaf_queue != 0;
    c->lb_whole = g->leafbasis_whole_chunks != 0;
    c->prior_st = g->prior_stages;
    drop_graphs(c);
    return MRA_OK;
}

mra_status mra_set_precision(mra_ctx *c, int precision)
{
    if (!c) return MRA_EINVAL;
    if (precision != MRA_FP64 && precision != MRA_MIXED && precision != MRA_MIXED_FAST) {
        c->err = "precision must be MRA_FP64, MRA_MIXED or MRA_MIXED_FAST";
        return MRA_EINVAL;
    }
    if (precision == c->precision) return MRA_OK;
    if (precision == MRA_FP64 && !c->fp64_fits) {
        c->err = "tree too deep for the FP64 shared-memory kernels at this r";
        return MRA_EINVAL;
    }
    c->precision = precision;
    c->lb_rows = c->lb_stages = c->bucket_set = 0; // tuned for the other precision
    c->concurrent = true;
    c->leaf_queue = false;
    c->prior_st = 0;
    if (c->d_sx) {
        // the scratch layout and the theta per pass depend on the storage type
        const int mb = max_batch_for(c, c->hbm_budget);
        c->max_cap = c->user_max_batch > 0 ? std::min(c->user_max_batch, 1024) : mb;
        c->cap = 0;
    }
    return MRA_OK;
}

mra_status mra_loglik_device(mra_ctx *c, const double *theta_dev, int batch, double *loglik_dev, int *status_dev,
                             void *stream)
{
    if (!c) return MRA_EINVAL;
    if (!c->d_sx) {
        c->err = "context was built without a device";
        return MRA_EINVAL;
    }
    if (batch < 0 || (batch > 0 && (!theta_dev || !loglik_dev))) {
        c->err = "bad batch or null pointer";
        return MRA_EINVAL;
    }
    if (batch == 0) return MRA_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return enqueue(c, theta_dev, batch, loglik_dev, status_dev, (cudaStream_t)stream, false);
}

mra_status mra_loglik(mra_ctx *c, const double *theta, int batch, double *loglik)
{
    if (!c) return MRA_EINVAL;
    if (!c->d_sx) {
        c->err = "context was built without a device";
        return MRA_EINVAL;
    }
    if (batch < 0 || (batch > 0 && (!theta || !loglik))) {
        c->err = "bad batch or null pointer";
        return MRA_EINVAL;
    }
    if (batch == 0) return MRA_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (mra_status st = ensure_stage(c, batch)) return st;
    int *d_st = (int *)(c->d_ll_stage + batch);
    e = cudaMemcpy(c->d_theta_stage, theta, sizeof(double) * 3 * (size_t)batch, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy theta");
    mra_status st = enqueue(c, c->d_theta_stage, batch, c->d_ll_stage, d_st, (cudaStream_t)0, false);
    if (st != MRA_OK) return st;
    // loglik and status are adjacent in the staging buffer: one copy back
    std::vector<unsigned char> back(sizeof(double) * (size_t)batch + sizeof(int) * (size_t)batch);
    e = cudaMemcpy(back.data(), c->d_ll_stage, back.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy loglik");
    std::vector<int> hs((size_t)batch);
    memcpy(loglik, back.data(), sizeof(double) * (size_t)batch);
    memcpy(hs.data(), back.data() + sizeof(double) * (size_t)batch, sizeof(int) * (size_t)batch);
    for (int b = 0; b < batch; b++)
        if (hs[(size_t)b] != MRA_OK) {
            c->err = hs[(size_t)b] == MRA_EINVAL       ? "theta must be finite and positive"
                     : hs[(size_t)b] == MRA_ETIMEDOUT ? "a bounded device wait ran out (tensor-core pipeline)"
                                                      : "Cholesky factor not positive definite";
            return (mra_status)hs[(size_t)b];
        }
    return MRA_OK;
}

mra_status mra_region_terms(mra_ctx *c, const double *theta, double *d, double *u, double *logdetW, double *loglik)
{
    if (!c || !theta) return MRA_EINVAL;
    if (!c->d_sx) {
        c->err = "context was built without a device";
        return MRA_EINVAL;
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    // the kernels record per device region; the output is per partition region
    const int64_t NR = c->G.nreg(), NK = c->G.nnonleaf();
    if (!c->d_reg_du) {
        if (cudaMalloc((void **)&c->d_reg_du, sizeof(double) * 2 * (size_t)NR) != cudaSuccess ||
            cudaMalloc((void **)&c->d_reg_lw, sizeof(double) * (size_t)std::max<int64_t>(NK, 1)) != cudaSuccess) {
            c->err = "cannot allocate region records";
            return MRA_ENOMEM;
        }
        c->bytes_held += sizeof(double) * (2 * (size_t)NR + (size_t)std::max<int64_t>(NK, 1));
    }
    if (mra_status st = ensure_stage(c, 1)) return st;
    std::vector<double> nanv((size_t)std::max<int64_t>(NK, 1), std::nan(""));
    e = cudaMemset(c->d_reg_du, 0, sizeof(double) * 2 * (size_t)NR);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_reg_lw, nanv.data(), sizeof(double) * nanv.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_theta_stage, theta, sizeof(double) * 3, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "region setup");
    int *d_st = (int *)(c->d_ll_stage + 1);
    mra_status st = enqueue(c, c->d_theta_stage, 1, c->d_ll_stage, d_st, (cudaStream_t)0, true);
    if (st != MRA_OK) return st;
    std::vector<double> du((size_t)(2 * NR)), lw((size_t)std::max<int64_t>(NK, 1));
    int hs = 0;
    double ll = 0.0;
    e = cudaMemcpy(du.data(), c->d_reg_du, sizeof(double) * du.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lw.data(), c->d_reg_lw, sizeof(double) * lw.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ll, c->d_ll_stage, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hs, d_st, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "region readback");
    // Partition region (level l, index i): d and u of its first device level
    // (the terms of levels l..M, both halves of level l included); log|W| of
    // its knots = log|W of the first half| + log|W of the second half given
    // the first| (Schur complement).
    const Partition &P = c->P;
    const Levels &G = c->G;
    for (int l = 1; l <= P.M; l++) {
        const int m1 = l == P.M ? G.M : (G.split == 1 ? l : 2 * l - 1);
        for (int64_t i = 0; i < P.lvl_off[(size_t)l + 1] - P.lvl_off[(size_t)l]; i++) {
            const int64_t gr = P.lvl_off[(size_t)l] + i, gd = G.lvl_off[(size_t)m1] + i;
            if (d) d[gr] = du[(size_t)(2 * gd)];
            if (u) u[gr] = du[(size_t)(2 * gd + 1)];
            if (logdetW) {
                double v = std::nan("");
                if (l < P.M) {
                    v = lw[(size_t)gd];
                    if (G.split == 2) v += lw[(size_t)(G.lvl_off[(size_t)m1 + 1] + i)];
                }
                logdetW[gr] = v;
            }
        }
    }
    if (loglik) *loglik = ll;
    return (mra_status)hs;
}

mra_status mra_predict(mra_ctx *c, const double *theta, const double *px, const double *py, int64_t np,
                       double *mean, double *var)
{
    if (!c) return MRA_EINVAL;
    if (!c->d_sx) {
        c->err = "context was built without a device";
        return MRA_EINVAL;
    }
    if (!theta || np < 0 || (np > 0 && (!px || !py || !mean || !var))) {
        c->err = "bad count or null pointer";
        return MRA_EINVAL;
    }
    for (int k = 0; k < 3; k++)
        if (!(std::isfinite(theta[k]) && theta[k] > 0.0)) {
            c->err = "theta must be finite and positive";
            return MRA_EINVAL;
        }
    if (np == 0) return MRA_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (mra_status st = ensure_stage(c, 1)) return st;
    if (mra_status st = ensure_capacity(c, 1)) return st;
    // group the points by leaf (a stable counting sort), outside points first
    const int64_t NL = c->P.nleaf();
    std::vector<int64_t> leaf((size_t)np), order((size_t)np), pos((size_t)NL + 2, 0);
    for (int64_t k = 0; k < np; k++) {
        leaf[(size_t)k] = std::isfinite(px[k]) && std::isfinite(py[k]) ? leaf_of(c->P, px[k], py[k]) : -1;
        pos[(size_t)(leaf[(size_t)k] + 2)]++;
    }
    for (int64_t l = 1; l < NL + 2; l++) pos[(size_t)l] += pos[(size_t)(l - 1)];
    for (int64_t k = 0; k < np; k++) order[(size_t)pos[(size_t)(leaf[(size_t)k] + 1)]++] = k;
    std::vector<double> sx((size_t)np), sy((size_t)np), m((size_t)np), v((size_t)np);
    std::vector<int64_t> sl((size_t)np);
    for (int64_t k = 0; k < np; k++) {
        const int64_t o = order[(size_t)k];
        sx[(size_t)k] = leaf[(size_t)o] >= 0 ? px[o] : 0.0;
        sy[(size_t)k] = leaf[(size_t)o] >= 0 ? py[o] : 0.0;
        sl[(size_t)k] = leaf[(size_t)o];
    }
    mra_status st;
    if (c->precision != MRA_FP64)
        st = c->RP == 16 ? predict_impl<float, 16>(c, theta, sx, sy, sl, m.data(), v.data())
                         : predict_impl<float, 32>(c, theta, sx, sy, sl, m.data(), v.data());
    else
        st = c->RP == 16 ? predict_impl<double, 16>(c, theta, sx, sy, sl, m.data(), v.data())
                         : predict_impl<double, 32>(c, theta, sx, sy, sl, m.data(), v.data());
    if (st != MRA_OK) return st;
    for (int64_t k = 0; k < np; k++) {
        mean[order[(size_t)k]] = m[(size_t)k];
        var[order[(size_t)k]] = v[(size_t)k];
    }
    return MRA_OK;
}

mra_status mra_stats(const mra_ctx *c, mra_stats_t *o)
{
    if (!c || !o) return MRA_EINVAL;
    memset(o, 0, sizeof(*o));
    const Partition &P = c->P;
    o->n_in = P.n_in;
    o->n_used = P.n_used;
    o->n_nan = P.n_nan;
    o->n_dup = P.n_dup;
    o->n_knot = P.n_knot;
    if (!P.lvl_off.empty()) {
        o->n_regions = P.nreg();
        o->n_leaves = P.nleaf();
    }
    o->M = P.M;
    o->J = P.J;
    o->r = P.r;
    o->r_hat = P.R;
    o->max_leaf = c->max_leaf;
    o->empty_leaves = c->empty_leaves;
    o->max_batch = c->cap;
    o->flops_per_theta = c->flops;
    o->cov_evals_per_theta = c->covs;
    o->device_bytes = c->bytes_held;
    o->launches_per_pass = c->launches_last;
    for (int k = 0; k < 8; k++) o->flops_by_kernel[k] = c->flops_k[k];
    o->device_levels = c->G.M;
    o->subtree_level = c->sub_level;
    o->subtree_chunks = 0;
    if (c->sub_level > 0 && c->sub_chunk > 0) {
        const int64_t nS = c->G.lvl_off[(size_t)c->sub_level + 1] - c->G.lvl_off[(size_t)c->sub_level];
        o->subtree_chunks = (int)((nS + c->sub_chunk - 1) / c->sub_chunk);
    }
    return MRA_OK;
}

mra_status mra_tree_export(const mra_ctx *c, double *kx, double *ky, int64_t *leaf_off, int64_t *perm, double *bounds)
{
    if (!c || c->P.lvl_off.empty()) return MRA_EINVAL;
    const Partition &P = c->P;
    if (kx) std::copy(P.kx.begin(), P.kx.end(), kx);
    if (ky) std::copy(P.ky.begin(), P.ky.end(), ky);
    if (leaf_off) std::copy(P.leaf_off.begin(), P.leaf_off.end(), leaf_off);
    if (perm) std::copy(P.perm.begin(), P.perm.end(), perm);
    if (bounds)
        for (int64_t g = 0; g < P.nreg(); g++) {
            bounds[4 * g + 0] = P.bx0[(size_t)g];
            bounds[4 * g + 1] = P.bx1[(size_t)g];
            bounds[4 * g + 2] = P.by0[(size_t)g];
            bounds[4 * g + 3] = P.by1[(size_t)g];
        }
    return MRA_OK;
}

mra_status mra_profile(mra_ctx *c, int enable)
{
    if (!c) return MRA_EINVAL;
    c->prof_on = enable != 0;
    c->ev_used = 0;
    return MRA_OK;
}

int mra_profile_read(mra_ctx *c, mra_kernel_time *out, int cap)
{
    if (!c || (cap > 0 && !out)) return -1;
    double ms[K_COUNT] = {0};
    int64_t cnt[K_COUNT] = {0};
    for (size_t k = 0; k + 1 < c->ev_used + 1 && k < c->ev_used; k += 2) {
        float t = 0.f;
        if (cudaEventSynchronize(c->ev[k + 1]) != cudaSuccess) return -1;
        if (cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]) != cudaSuccess) return -1;
        ms[c->ev_kind[k / 2]] += t;
        cnt[c->ev_kind[k / 2]]++;
    }
    c->ev_used = 0;
    int n = 0;
    for (int k = 0; k < K_COUNT; k++) {
        if (cnt[k] == 0) continue;
        if (n < cap) {
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
            out[n].launches = cnt[k];
            out[n].ms = ms[k];
        }
        n++;
    }
    return n;
}

const char *mra_last_error(const mra_ctx *c)
{
    if (!c) return g_build_err.c_str();
    return c->err.c_str();
}

void mra_free(mra_ctx *c)
{
    if (!c) return;
    if (c->device >= 0 && c->d_sx) cudaSetDevice(c->device);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int k = 0; k < kLeafBuckets; k++) {
        if (c->aux[k]) cudaStreamDestroy(c->aux[k]);
        if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->lbt_fork) cudaEventDestroy(c->lbt_fork);
    if (c->lbt_join) cudaEventDestroy(c->lbt_join);
    void *ptrs[] = {c->d_kx, c->d_ky, c->d_cx, c->d_cy, c->d_sx, c->d_sy, c->d_sz, c->d_leaf_off, c->d_chunks32,
                    c->d_chunks64, c->d_chunks128, c->d_chunks16, c->d_leaves[0], c->d_leaves[1], c->d_leaves[2], c->d_leaves[3], c->d_leaves_m, c->d_big, c->d_bigitems, c->d_scratch, c->d_status, c->d_theta_stage, c->d_ll_stage,
                    c->d_reg_du, c->d_reg_lw, c->pred.pt, c->pred.tree, c->d_qcnt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
}

} // extern "C"
