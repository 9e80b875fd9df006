/*
 * mra.h -- C ABI of the GB300 (sm_103a) multi-resolution approximation (MRA)
 * Gaussian-process log-likelihood library (libmra.so).
 *
 * The method (Huang, Blake & Hammerling, "Pushing the Limit: A Hybrid
 * Parallel Implementation of the Multi-resolution Approximation for Massive
 * Data", Sec. 1.1-1.2): the domain is split recursively into J (2 or 4)
 * sub-regions for M levels; every region above the finest level carries
 * r_hat = ceil(sqrt r) * floor(r / ceil(sqrt r)) knots on a regular grid; the
 * knots of a finest-level region are the observations inside it.  The process
 * is a sum of predictive processes on the remainder covariances C_1 .. C_M of
 * Sec. 1.1.  mra_loglik evaluates log N(z; 0, Sigma_MRA + tau2 I) at
 * theta = (sigma2, beta, tau2) for the exponential covariance
 * sigma2 * exp(-|s1 - s2| / beta) ("likelihood" mode, Sec. 2.2.5; sill ALPHA,
 * range BETA, nugget TAU of the user-parameter table, Sec. 2.2.3, with TAU read
 * as the nugget variance tau2).
 *
 * Conventions for every entry point:
 *   - Host pointers are plain CPU memory and are only read during the call
 *     (the library copies what it keeps).  "Device" pointers are CUDA global
 *     memory on the context's device.
 *   - A mra_ctx owns all the device memory it allocates; mra_free releases it.
 *   - A context is not reentrant: calls on one context must not overlap.
 *     Several contexts may coexist.
 *   - Every entry point returns a mra_status; on failure mra_last_error gives a
 *     one-line reason.  No entry point aborts, traps or prints.
 */
#ifndef MRA_H
#define MRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mra_ctx mra_ctx;

typedef enum {
    MRA_OK = 0,
    MRA_EINVAL = 1,    /* bad argument: sizes, J not 2/4, theta not positive, ... */
    MRA_ENOMEM = 2,    /* a host or device allocation failed, or the budget is too small */
    MRA_ENOTPD = 3,    /* a Cholesky factor met a non-positive pivot (singular prior) */
    MRA_ECUDA = 4,     /* a CUDA runtime call failed (message in mra_last_error) */
    MRA_ETIMEDOUT = 5, /* reserved: a bounded device wait ran out */
    MRA_EEMPTY = 6     /* no observation left after the eliminations of Sec. 1.2 */
} mra_status;

/* MRA_FP64: every step in FP64.  MRA_MIXED: FP32 storage and products; float
 * pairs (double-float on the FP32 pipe) for the covariances, the remainder
 * recursions C_l(., Q) = C - sum_k What^k What^k' of the prior and of the leaf
 * basis (exact products), the leaf covariance, every Cholesky factor,
 * log-determinant and quadratic form.  MRA_MIXED_FAST: as MRA_MIXED but the
 * remainder recursions in FP32 (faster; its error grows with tree depth and
 * covariance range, e.g. |dl|/n ~ 2e-5 at M = 14, range 0.3). */
enum { MRA_FP64 = 0, MRA_MIXED = 1, MRA_MIXED_FAST = 2 };

typedef struct {
    double offset;     /* knot offset f of Sec. 1.2; < 0 selects the paper's default e/100 */
    int dedup;         /* ELIMINATION_DUPLICATES_FLAG: drop repeated locations, keep the first */
    int precision;     /* MRA_FP64 (default), MRA_MIXED or MRA_MIXED_FAST */
    int device;        /* CUDA device ordinal; -1 builds the partition on the host only
                          (stats and tree queries work, likelihood calls give MRA_EINVAL) */
    int max_batch;     /* theta evaluated per device pass; 0 = choose from hbm_budget */
    size_t hbm_budget; /* bytes of per-theta scratch the context may hold; 0 = 60% of free HBM */
    int graphs;        /* 1 (default): a device pass seen before is replayed from a captured CUDA graph
                          (keyed by its theta/loglik/status pointers, batch and precision; recaptured
                          when the scratch moves); 0: every kernel is launched on each call */
} mra_opts;

typedef struct {
    int64_t n_in, n_used;       /* observations given / used */
    int64_t n_nan, n_dup, n_knot; /* dropped: NaN value, duplicate location, on a coarse knot */
    int64_t n_regions, n_leaves;
    int M, J, r, r_hat;
    int64_t max_leaf, empty_leaves;
    int max_batch;
    double flops_per_theta;     /* algorithmic FP operations of one evaluation (r_hat, not padding) */
    double cov_evals_per_theta; /* covariance-function evaluations of one evaluation */
    size_t device_bytes;        /* device memory held by the context */
    int launches_per_pass;      /* kernels launched by the last device pass (one batch chunk) */
    double flops_by_kernel[8];  /* flops_per_theta split by kernel family, in the order
                                   prior, leafbasis, leafpost, leafpost_big, leafgram, up, root */
    int device_levels;          /* levels the kernels run: M, or 2 (M - 1) + 1 when r_hat > 32
                                   (each non-leaf level enters its knots in two halves) */
    int subtree_level;          /* 0, or the device level S below which the leaf Gram and the upward
                                   pass run subtree by subtree (mra_tune_t.subtree_level) */
    int subtree_chunks;         /* chunks of level-S subtrees one pass runs (0 when not streamed) */
} mra_stats_t;

typedef struct {
    char name[24];    /* kernel family: prior, leafbasis, leafpost, leafpost_big, leafgram, up, root */
    int64_t launches; /* launches recorded since the last read */
    double ms;        /* summed device time of those launches (CUDA events on the call's stream) */
} mra_kernel_time;

/* Fill *opt with the defaults (offset e/100, no dedup, FP64, device 0, auto batch). */
void mra_default_opts(mra_opts *opt);

/*
 * mra_build -- partition, knots and observation layout (Sec. 1.2).
 *   lon, lat, z : host arrays of n doubles (locations and values).  A NaN value
 *                 marks a prediction site and is dropped; non-finite locations
 *                 give MRA_EINVAL.
 *   M >= 1 levels, J in {2, 4}, r >= 1 knots requested (r_hat placed,
 *   r_hat <= 64).  With r_hat > 32 every non-leaf level is run as two device
 *   levels of the same regions, the first ceil(r_hat/2) knots and then the
 *   rest (Sec. 1.1: the remainder after projecting on the two halves in turn
 *   is the remainder after projecting on all of them, so the likelihood is the
 *   same); 2 (M - 1) + 1 device levels must not exceed 35.
 *   The domain is the bounding box with its top and right edges pushed out by
 *   1% of the extent; regions are half-open [x0,x1) x [y0,y1); J = 4 halves both
 *   sides, J = 2 halves the longer side (ties: x).  Observations that sit exactly
 *   on a knot of levels 1..M-1 are dropped; duplicates too when opt->dedup.
 *   opt may be NULL (defaults).  On success *out owns a device copy of the tree
 *   and of the used observations in leaf order; on failure *out is NULL and
 *   mra_last_error(NULL) gives the reason.
 *   Errors: MRA_EINVAL (sizes, J, r, M, offset outside [0, 0.5), degenerate
 *   domain, r_hat > 64, a tree too deep for the shared-memory kernels in the
 *   requested precision), MRA_EEMPTY (nothing left), MRA_ENOMEM, MRA_ECUDA.
 */
mra_status mra_build(const double *lon, const double *lat, const double *z, int64_t n, int M,
                     int J, int r, const mra_opts *opt, mra_ctx **out);

/*
 * mra_loglik -- log-likelihood at a batch of theta (Sec. 2.2.5 "likelihood").
 *   theta  : host, batch x 3 doubles, row b = (sigma2, beta, tau2), all > 0.
 *   loglik : host, batch doubles, written for every b; NaN where theta b is
 *            invalid or a factorisation failed.
 *   Returns the first non-OK per-theta status (MRA_EINVAL, MRA_ENOTPD) or a
 *   call-level error.  Synchronous.
 */
mra_status mra_loglik(mra_ctx *ctx, const double *theta, int batch, double *loglik);

/*
 * mra_loglik_device -- as mra_loglik with device pointers, enqueued on
 *   `stream` (a cudaStream_t; NULL = legacy default stream) and not synchronised.
 *   theta_dev : device, batch x 3 doubles.  loglik_dev : device, batch doubles.
 *   status_dev: optional device int array of batch entries (per-theta mra_status),
 *               may be NULL.
 *   Returns MRA_OK once every kernel is enqueued; per-theta failures only show
 *   in loglik_dev (NaN) and status_dev.
 */
mra_status mra_loglik_device(mra_ctx *ctx, const double *theta_dev, int batch, double *loglik_dev,
                             int *status_dev, void *stream);

/*
 * mra_autotune -- choose the launch configuration of the context's current
 * precision by timing it on this tree.  Candidates: observation rows per
 * leaf-basis CTA (32 or, in the mixed mode, 64), one or two shared-memory
 * stages of ancestor blocks, the leaf-size buckets of the leaf posterior
 * ({<=32, <=40, <=48, <=64} or {<=32, <=64}), running those buckets on side
 * streams or one after another, and each bucket as one CTA per leaf or as a
 * persistent work queue.  Every candidate computes the same loglik,
 * bit for bit; only the time differs.  Each candidate runs 2 untimed and
 * `reps` timed passes of one theta (theta: host, 3 doubles) on a stream of
 * the library; the fastest is kept for later calls (mra_set_precision resets
 * it).  out (may be NULL) receives the choice and the times.
 */
typedef struct {
    int leafbasis_rows;   /* 32 or 64 (FP32 only); 16: the streaming kernel of deep trees (ancestor blocks
                             staged two at a time, the same results bit for bit), the default where 32-row
                             chunks leave room for one CTA per SM */
    int leafbasis_stages; /* 1 or 2 */
    int bucket_set;       /* 0: {<=32, <=40, <=48, <=64}, 1: {<=32, <=64} */
    int concurrent;       /* 1: leaf-posterior buckets on side streams */
    double ms_default;    /* mean pass time with the configuration before the call */
    double ms_best;       /* mean pass time with the chosen configuration */
    int tried;            /* candidates timed */
    int gram_tensor_cores; /* mixed modes: 0 (default) the leaf Gram on the CUDA cores (FP32 products, float-pair
                              sums of 32-row chunks); 1 on the tensor cores (tcgen05 BF16 MMAs of exact
                              fixed-grid slices, exact sums, rounded once per 320 rows).  The two differ in the
                              last bits, so the autotuner does not switch it: it reports the setting in force. */
    int leaf_queue;       /* 1: each leaf-size bucket runs as a persistent work-queue kernel (CTAs resident at
                             once take the leaves, largest first, through an atomic counter) instead of one CTA
                             per leaf; the same results bit for bit, so the autotuner tries both */
    int prior_stages;     /* ancestor blocks of the prior staged in 0: a form per level chosen by occupancy (two
                             blocks at a time where that fits more CTAs per SM on a level of more than one
                             wave, else one buffer where it fits more CTAs per SM and saves a wave, else two),
                             1: one buffer, 2: two where they fit (the next level prefetched), 3: two blocks
                             at a time; the same results bit for bit */
    int leafbasis_tensor_cores; /* MRA_MIXED: 1 runs the leaf basis's remainder products on the tensor cores
                                   (tcgen05 BF16 MMAs of five exact fixed-grid slices per value, sums exact in
                                   tensor memory, 128 rows per CTA); trees with (M - 2) x padded r_hat up to 192
                                   (EINVAL beyond).  It differs from the CUDA-core kernel in the last bits, so
                                   the autotuner reports it but does not switch it. */
    int subtree_level;    /* 0 (default): chosen by the memory plan.  S in 1 .. device levels - 2: the leaf
                             Gram and the upward pass of device levels M-1 .. S run chunk by chunk of
                             level-S subtrees (regions contiguous at every level), so that the per-theta
                             ATilde arrays of those levels hold one chunk instead of the whole level; levels
                             S-1 .. 1 then run whole.  The plan streams subtrees by itself where one
                             theta's scratch would not fit the budget otherwise (deep trees: ATilde grows
                             with the number of regions, not with n).  The same results bit for bit. */
    int subtree_chunk;    /* level-S regions per chunk; 0: the largest that fits the budget */
    int leafbasis_whole_chunks; /* 0 (default): a region's last leaf-basis chunk of at most half the rows (32-
                                   or 64-row chunks) runs in the kernel of half the rows, on a side stream
                                   beside the full chunks (less padding); 1: every chunk at full size.  The
                                   same results bit for bit; the autotuner keeps the setting in force. */
} mra_tune_t;

mra_status mra_autotune(mra_ctx *ctx, const double *theta, int reps, mra_tune_t *out);

/* Set the launch configuration directly (the four configuration fields of
 * cfg, gram_tensor_cores, leaf_queue, prior_stages, leafbasis_tensor_cores,
 * subtree_level, subtree_chunk and leafbasis_whole_chunks; the times are
 * ignored).  leafbasis_rows 0 and
 * leafbasis_stages 0 select the defaults; EINVAL for a value outside the
 * candidates or one whose shared memory does not fit. */
mra_status mra_set_launch(mra_ctx *ctx, const mra_tune_t *cfg);

/* Select MRA_FP64, MRA_MIXED or MRA_MIXED_FAST for later calls. */
mra_status mra_set_precision(mra_ctx *ctx, int precision);

/* Counts, sizes and the algorithmic work of one evaluation. */
mra_status mra_stats(const mra_ctx *ctx, mra_stats_t *out);

/*
 * mra_tree_export -- the built partition, for inspection and tests.
 *   Any pointer may be NULL.  Sizes: kx, ky: (n_regions - n_leaves) * r_hat
 *   knots of levels 1..M-1 (global region id order, knot index q*nx + p);
 *   leaf_off: n_leaves + 1 offsets into the leaf-ordered observations;
 *   perm: n_used input indices in leaf order; bounds: 4 * n_regions doubles
 *   (x0, x1, y0, y1).  Region ids: level 1 first, children of (m, i) are
 *   (m+1, J i + j).
 */
mra_status mra_tree_export(const mra_ctx *ctx, double *kx, double *ky, int64_t *leaf_off,
                           int64_t *perm, double *bounds);

/*
 * mra_region_terms -- per-region partial terms at one theta (host pointers,
 *   n_regions doubles each): d_R = log-determinant and u_R = quadratic form of
 *   the data below R after R's level is integrated out (leaves: log|V| and
 *   z'V^{-1}z), and log|W^m_R| = log|C_m(Q_R, Q_R)| for regions above the
 *   leaves (NaN at leaves).  loglik: host, 1 double.  Synchronous.
 */
mra_status mra_region_terms(mra_ctx *ctx, const double *theta, double *d, double *u,
                            double *logdetW, double *loglik);

/*
 * mra_predict -- posterior prediction of the latent process at new locations
 *   (the prediction mode of the paper's program, Sec. 2.2; the model of
 *   Sec. 1.1): mean[k] = E[y(s_k) | z] and var[k] = Var[y(s_k) | z] for the
 *   MRA covariance at theta (host, 3 doubles), i.e. kriging with Sigma_MRA.
 *   The variance is that of the process without the nugget; add theta[2] for
 *   a new observation.
 *   px, py: host, np locations each; mean, var: host, np doubles each.
 *   Points outside the partition's domain (the bounding box of the data
 *   extended by 1% at the top and right) get NaN in both outputs.
 *   Runs one likelihood pass at theta that keeps the upward pass's factors,
 *   the top-down pass for the posterior means of the basis weights, the
 *   basis functions at the points, then one warp per point, all in the
 *   context's precision for the pass and FP64 for the prediction
 *   arithmetic.  Temporary device memory: about
 *   8 (n_nonleaf (r^2 + 2 r + (M-2) r^2) + n_leaves 64 (65)) bytes plus
 *   (M-1) r + 40 bytes per point.
 *   Errors: EINVAL (null pointer, np < 0, theta not finite and positive),
 *   ENOMEM, ENOTPD (a factor not positive definite at theta), ECUDA.
 *   Synchronous.
 */
mra_status mra_predict(mra_ctx *ctx, const double *theta, const double *px, const double *py, int64_t np,
                       double *mean, double *var);

/*
 * mra_profile -- enable (1) or disable (0) per-kernel device timing: every
 *   later launch is bracketed by two CUDA events recorded on the call's
 *   stream.  Enabling clears the records.  Costs two event records per launch.
 *   A profiled pass runs the kernels that otherwise share the GPU on side
 *   streams (leaf-posterior buckets, leaf-basis tail chunks) one after
 *   another, so each pair of events times one kernel alone.
 */
mra_status mra_profile(mra_ctx *ctx, int enable);

/*
 * mra_profile_read -- wait for the recorded events, write up to cap entries
 *   (one per kernel family that launched) into out (host), clear the records
 *   and return the number of families (-1 on error).
 */
int mra_profile_read(mra_ctx *ctx, mra_kernel_time *out, int cap);

/*
 * mra_dense_loglik_noalloc -- the single-region likelihood (M = 1: the only
 *   region is the leaf, so the result is the exact Gaussian log-density
 *   log N(z; 0, C(S,S) + tau2 I) of the exponential covariance) in FP64, WITHOUT
 *   allocating device memory.  The paper has no counterpart: this entry point
 *   serves callers that must not allocate, e.g. code running inside a CUDA
 *   graph capture or a real-time loop whose memory is reserved up front, and
 *   runtimes that own every allocation on the device and forbid libraries from
 *   calling cudaMalloc.
 *   x_dev, y_dev, z_dev : device, n doubles each (locations and values; NaN is
 *                         not filtered here).
 *   n                   : 1 <= n <= 1024, else MRA_EINVAL with a message in
 *                         mra_last_error(NULL); nothing is launched then.
 *   theta_dev           : device, 3 doubles (sigma2, beta, tau2).
 *   loglik_dev          : device, 1 double (NaN if theta is invalid or V is
 *                         singular).  status_dev: optional device int
 *                         (per-call mra_status), may be NULL.
 *   stream              : cudaStream_t (NULL = legacy default stream); the call
 *                         enqueues one kernel and does not synchronise.
 *   Working memory: a fixed array of (1024^2 + 2048) doubles (about 8 MiB)
 *   compiled into the library, present on every device that loads it until
 *   the process exits.  The first call on a device looks up the array's device
 *   address (cudaGetSymbolAddress, with that device current); make that first
 *   call before any stream capture.  The lookup is made again when the
 *   device's current context is not the one of the last lookup (after a
 *   cudaDeviceReset, say), so the first call after such a reset must also come
 *   outside stream capture.  All calls on a device share the array and
 *   it keeps the previous call's contents (every element a call reads it first
 *   writes): calls whose kernels may overlap on the GPU (different streams
 *   without ordering) race and give wrong results.  Calls no cudaMalloc,
 *   cudaFree or other allocating routine.  Not reentrant across host threads
 *   on the same device for the same reason.
 */
mra_status mra_dense_loglik_noalloc(const double *x_dev, const double *y_dev, const double *z_dev,
                                    int64_t n, const double *theta_dev, double *loglik_dev,
                                    int *status_dev, void *stream);

/* Last error message of the context (never NULL).  With ctx == NULL: the reason
 * the calling thread's last mra_build (which returns no context on failure) or
 * mra_dense_loglik_noalloc failed. */
const char *mra_last_error(const mra_ctx *ctx);

/* Release the context and all its device memory.  NULL is a no-op. */
void mra_free(mra_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MRA_H */
