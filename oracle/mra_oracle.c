/*
 * mra_oracle.c -- plain, slow FP64 CPU reference of the multi-resolution
 * approximation (MRA) Gaussian-process log-likelihood.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or helper with the CUDA library; it is written from the
 * paper's definitions alone:
 *
 *   - Sec. 1.1: recursive J-ary partition of the domain into M levels; r knots
 *     per region at levels 1..M-1; at level M the knots are the observations.
 *   - Sec. 1.1 (display of C_2 .. C_M): remainder covariances
 *       C_1 = C,
 *       C_{m+1}(s1,s2) = C_m(s1,s2) - C_m(s1,Q)' C_m(Q,Q)^{-1} C_m(s2,Q)
 *     with Q the knots of the level-m region holding s1 and s2 (and 0 when s1,
 *     s2 lie in different level-(m+1) regions); tau_m(s) = C_m(s,Q)' eta with
 *     eta ~ N(0, C_m(Q,Q)^{-1}) independent over regions and levels.
 *   - Sec. 1.2: domain extension by 1% at the top and right, half-open
 *     regions, J=4 quadrant / J=2 longer-side splits, the
 *     ceil(sqrt r) x floor(r/ceil(sqrt r)) knot grid with the offset rule of
 *     App. A, elimination of observations that coincide with a coarse knot,
 *     optional duplicate elimination (Table "user parameters").
 *   - Sec. 2.2.4: exponential covariance with sill ALPHA, range BETA, nugget
 *     TAU.  Reading: C(a,b) = sigma2 * exp(-|a-b|_2 / beta), nugget variance
 *     tau2 added on observations only.
 *
 * The paper never prints the likelihood recursion; it evaluates
 * log N(z; 0, Sigma_MRA + tau2 I) in "likelihood" mode.  The recursion below is
 * the one that follows from the definitions above by integrating out the eta
 * of level M-1, then M-2, ..., then 1 with the Woodbury identity and the
 * matrix-determinant lemma, in the paper's own quantities: the remainder
 * covariance blocks W^l_R = C_l(Q_R, Q_{anc_l(R)}), the prior precision
 * K_R = (W^m_R)^{-1}, the leaf basis B^l = W^l of the observations and the
 * posterior information ATilde passed up to the parent (App. B):
 *
 *   leaf c:   V = W^M_c + tau2 I,  ATilde_c = B' V^{-1} B,
 *             wTilde_c = B' V^{-1} z,  d_c = log|V|,  u_c = z' V^{-1} z
 *   region R at level m < M:
 *             A = sum_children ATilde, w = sum_children wTilde,
 *             T = K_R^{-1} + A^{m,m} = W^m_R + A^{m,m},
 *             ATilde_R = A^{<m,<m} - A^{<m,m} T^{-1} A^{m,<m},
 *             wTilde_R = w^{<m} - A^{<m,m} T^{-1} w^m,
 *             d_R = sum d_c + log|T| - log|W^m_R|,
 *             u_R = sum u_c - (w^m)' T^{-1} w^m
 *   root:     loglik = -1/2 (d_1 + u_1 + n log 2 pi).
 *
 * Everything is FP64, row-major, with triple-loop products and a textbook
 * Cholesky.  OpenMP tasks split the tree over subtrees (the paper's own
 * intra-node strategy is OpenMP over regions, Sec. 4.1); the arithmetic of a
 * region does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_OK 0
#define O_EINVAL 1
#define O_ENOMEM 2
#define O_ENOTPD 3
#define O_EEMPTY 6

#define O_MAXM 32
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int M, J, r, nx, ny, rhat;
    double offset;
    int64_t nreg;
    int64_t lvl_off[O_MAXM + 2]; /* first global id of level m (1-based) */
    double *bx0, *bx1, *by0, *by1; /* region bounds, half-open [x0,x1) x [y0,y1) */
    double *kx, *ky;               /* knots of levels 1..M-1, rhat per region */
    int64_t nleaf;
    int64_t *leaf_off; /* nleaf + 1 */
    double *sx, *sy, *sz;
    int64_t *perm;
    int64_t n_in, n_used, n_nan, n_dup, n_knot;
} otree;

/* ---------------------------------------------------------------- tree -- */

/* Knot grid of one region (Sec. 1.2 and App. A): ceil(sqrt r) bars along x,
 * floor(r / ceil(sqrt r)) along y, bar p at x0 + L (f + p (1-2f)/(n-1)).
 * A single bar (n = 1) is put at the region centre.  Knot index q*nx + p. */
static void place_knots(double x0, double x1, double y0, double y1, int nx, int ny,
                        double f, double *kx, double *ky)
{
    double Lx = x1 - x0, Ly = y1 - y0;
    for (int q = 0; q < ny; q++) {
        for (int p = 0; p < nx; p++) {
            double xs, ys;
            if (nx > 1)
                xs = x0 + Lx * (f + (double)p * (1.0 - 2.0 * f) / (double)(nx - 1));
            else
                xs = x0 + 0.5 * Lx;
            if (ny > 1)
                ys = y0 + Ly * (f + (double)q * (1.0 - 2.0 * f) / (double)(ny - 1));
            else
                ys = y0 + 0.5 * Ly;
            kx[q * nx + p] = xs;
            ky[q * nx + p] = ys;
        }
    }
}

static void grid_dims(int r, int *nx, int *ny)
{
    int a = (int)ceil(sqrt((double)r));
    while (a * a < r) a++;            /* guard the library sqrt at squares */
    while (a > 1 && (a - 1) * (a - 1) >= r) a--;
    *nx = a;
    *ny = r / a;
}

void oracle_place_knots(double x0, double x1, double y0, double y1, int r, double offset,
                        double *kx, double *ky, int *rhat)
{
    int nx, ny;
    grid_dims(r, &nx, &ny);
    *rhat = nx * ny;
    place_knots(x0, x1, y0, y1, nx, ny, offset, kx, ky);
}

typedef struct { double x, y; int64_t i; } opt;

static int cmp_pt(const void *a, const void *b)
{
    const opt *p = (const opt *)a, *q = (const opt *)b;
    if (p->x < q->x) return -1;
    if (p->x > q->x) return 1;
    if (p->y < q->y) return -1;
    if (p->y > q->y) return 1;
    if (p->i < q->i) return -1;
    if (p->i > q->i) return 1;
    return 0;
}

void oracle_tree_free(void *h)
{
    otree *t = (otree *)h;
    if (!t) return;
    free(t->bx0); free(t->bx1); free(t->by0); free(t->by1);
    free(t->kx); free(t->ky); free(t->leaf_off);
    free(t->sx); free(t->sy); free(t->sz); free(t->perm);
    free(t);
}

/* Build the partition (Sec. 1.2).  Observations with NaN value are dropped
 * (they mark prediction sites), then duplicates if asked (first occurrence
 * kept), then the domain is the bounding box with its top and right edges
 * pushed out by 1% of the extent, then observations sitting exactly on a knot
 * of levels 1..M-1 are dropped. */
void *oracle_tree_new(const double *x, const double *y, const double *z, int64_t n, int M,
                      int J, int r, double offset, int dedup, int *status)
{
    *status = O_EINVAL;
    if (n < 0 || M < 1 || M > O_MAXM || (J != 2 && J != 4) || r < 1) return NULL;
    if (!(offset >= 0.0 && offset < 0.5)) return NULL;
    double total = 0.0, pw = 1.0;
    for (int m = 1; m <= M; m++) { total += pw; pw *= J; }
    if (total > 268435456.0) return NULL;
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i])) return NULL;

    otree *t = (otree *)calloc(1, sizeof(otree));
    if (!t) { *status = O_ENOMEM; return NULL; }
    t->M = M; t->J = J; t->r = r; t->offset = offset;
    grid_dims(r, &t->nx, &t->ny);
    t->rhat = t->nx * t->ny;
    t->n_in = n;

    /* 1. drop NaN values */
    int64_t *keep = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    unsigned char *drop = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t nk = 0;
    for (int64_t i = 0; i < n; i++) {
        if (isnan(z[i])) { drop[i] = 1; t->n_nan++; }
    }
    /* 2. duplicates */
    if (dedup && n > 0) {
        opt *ps = (opt *)malloc(sizeof(opt) * (size_t)n);
        int64_t np = 0;
        for (int64_t i = 0; i < n; i++)
            if (!drop[i]) { ps[np].x = x[i]; ps[np].y = y[i]; ps[np].i = i; np++; }
        qsort(ps, (size_t)np, sizeof(opt), cmp_pt);
        for (int64_t k = 1; k < np; k++)
            if (ps[k].x == ps[k - 1].x && ps[k].y == ps[k - 1].y) { drop[ps[k].i] = 1; t->n_dup++; }
        free(ps);
    }
    for (int64_t i = 0; i < n; i++)
        if (!drop[i]) keep[nk++] = i;
    if (nk == 0) {
        free(keep); free(drop); oracle_tree_free(t); *status = O_EEMPTY; return NULL;
    }
    /* 3. domain */
    double xmin = x[keep[0]], xmax = xmin, ymin = y[keep[0]], ymax = ymin;
    for (int64_t k = 1; k < nk; k++) {
        double a = x[keep[k]], b = y[keep[k]];
        if (a < xmin) xmin = a;
        if (a > xmax) xmax = a;
        if (b < ymin) ymin = b;
        if (b > ymax) ymax = b;
    }
    if (!(xmax > xmin) || !(ymax > ymin)) {
        free(keep); free(drop); oracle_tree_free(t); *status = O_EINVAL; return NULL;
    }
    double X0 = xmin, X1 = xmax + 0.01 * (xmax - xmin);
    double Y0 = ymin, Y1 = ymax + 0.01 * (ymax - ymin);

    /* 4. regions, level by level; children of (m, i) are (m+1, J i + j) */
    int64_t cnt = 1;
    t->lvl_off[1] = 0;
    for (int m = 1; m <= M; m++) { t->lvl_off[m + 1] = t->lvl_off[m] + cnt; cnt *= J; }
    t->nreg = t->lvl_off[M + 1];
    t->nleaf = t->lvl_off[M + 1] - t->lvl_off[M];
    t->bx0 = (double *)malloc(sizeof(double) * (size_t)t->nreg);
    t->bx1 = (double *)malloc(sizeof(double) * (size_t)t->nreg);
    t->by0 = (double *)malloc(sizeof(double) * (size_t)t->nreg);
    t->by1 = (double *)malloc(sizeof(double) * (size_t)t->nreg);
    t->bx0[0] = X0; t->bx1[0] = X1; t->by0[0] = Y0; t->by1[0] = Y1;
    /* J=2 cuts the longer side; all regions of one level share the nominal
     * side lengths, which halve exactly, so the choice is made per level
     * (ties cut x). */
    int cutx[O_MAXM + 1];
    double Lx = X1 - X0, Ly = Y1 - Y0;
    for (int m = 1; m < M; m++) {
        cutx[m] = (Lx >= Ly);
        if (J == 4) { Lx *= 0.5; Ly *= 0.5; }
        else if (cutx[m]) Lx *= 0.5;
        else Ly *= 0.5;
    }
    for (int m = 1; m < M; m++) {
        int64_t nm = t->lvl_off[m + 1] - t->lvl_off[m];
        for (int64_t i = 0; i < nm; i++) {
            int64_t g = t->lvl_off[m] + i;
            double x0 = t->bx0[g], x1 = t->bx1[g], y0 = t->by0[g], y1 = t->by1[g];
            double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
            int64_t c0 = t->lvl_off[m + 1] + i * J;
            if (J == 4) {
                t->bx0[c0 + 0] = x0; t->bx1[c0 + 0] = mx; t->by0[c0 + 0] = y0; t->by1[c0 + 0] = my;
                t->bx0[c0 + 1] = mx; t->bx1[c0 + 1] = x1; t->by0[c0 + 1] = y0; t->by1[c0 + 1] = my;
                t->bx0[c0 + 2] = x0; t->bx1[c0 + 2] = mx; t->by0[c0 + 2] = my; t->by1[c0 + 2] = y1;
                t->bx0[c0 + 3] = mx; t->bx1[c0 + 3] = x1; t->by0[c0 + 3] = my; t->by1[c0 + 3] = y1;
            } else if (cutx[m]) {
                t->bx0[c0 + 0] = x0; t->bx1[c0 + 0] = mx; t->by0[c0 + 0] = y0; t->by1[c0 + 0] = y1;
                t->bx0[c0 + 1] = mx; t->bx1[c0 + 1] = x1; t->by0[c0 + 1] = y0; t->by1[c0 + 1] = y1;
            } else {
                t->bx0[c0 + 0] = x0; t->bx1[c0 + 0] = x1; t->by0[c0 + 0] = y0; t->by1[c0 + 0] = my;
                t->bx0[c0 + 1] = x0; t->bx1[c0 + 1] = x1; t->by0[c0 + 1] = my; t->by1[c0 + 1] = y1;
            }
        }
    }
    /* knots of levels 1..M-1 */
    int R = t->rhat;
    int64_t nkr = t->lvl_off[M]; /* regions above the leaves */
    t->kx = (double *)malloc(sizeof(double) * (size_t)(nkr * R + 1));
    t->ky = (double *)malloc(sizeof(double) * (size_t)(nkr * R + 1));
    for (int64_t g = 0; g < nkr; g++)
        place_knots(t->bx0[g], t->bx1[g], t->by0[g], t->by1[g], t->nx, t->ny, offset,
                    t->kx + g * R, t->ky + g * R);
    /* 5. drop observations that coincide with any coarse knot (Sec. 1.2) */
    if (nkr > 0) {
        opt *ks = (opt *)malloc(sizeof(opt) * (size_t)(nkr * R));
        for (int64_t k = 0; k < nkr * R; k++) { ks[k].x = t->kx[k]; ks[k].y = t->ky[k]; ks[k].i = 0; }
        qsort(ks, (size_t)(nkr * R), sizeof(opt), cmp_pt);
        int64_t w = 0;
        for (int64_t k = 0; k < nk; k++) {
            opt key; key.x = x[keep[k]]; key.y = y[keep[k]]; key.i = 0;
            int64_t lo = 0, hi = nkr * R;
            int hit = 0;
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                const opt *p = &ks[mid];
                if (p->x < key.x || (p->x == key.x && p->y < key.y)) lo = mid + 1;
                else hi = mid;
            }
            if (lo < nkr * R && ks[lo].x == key.x && ks[lo].y == key.y) hit = 1;
            if (hit) t->n_knot++;
            else keep[w++] = keep[k];
        }
        nk = w;
        free(ks);
    }
    /* 6. leaf of every kept observation, then a stable counting sort */
    int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk > 0 ? nk : 1));
    for (int64_t k = 0; k < nk; k++) {
        double a = x[keep[k]], b = y[keep[k]];
        int64_t i = 0;
        for (int m = 1; m < M; m++) {
            int64_t g = t->lvl_off[m] + i;
            double mx = 0.5 * (t->bx0[g] + t->bx1[g]), my = 0.5 * (t->by0[g] + t->by1[g]);
            int j;
            if (J == 4) j = (a >= mx ? 1 : 0) + (b >= my ? 2 : 0);
            else if (cutx[m]) j = (a >= mx ? 1 : 0);
            else j = (b >= my ? 1 : 0);
            i = i * J + j;
        }
        leaf[k] = i;
    }
    t->leaf_off = (int64_t *)calloc((size_t)(t->nleaf + 1), sizeof(int64_t));
    for (int64_t k = 0; k < nk; k++) t->leaf_off[leaf[k] + 1]++;
    for (int64_t i = 0; i < t->nleaf; i++) t->leaf_off[i + 1] += t->leaf_off[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(t->nleaf + 1));
    memcpy(fill, t->leaf_off, sizeof(int64_t) * (size_t)(t->nleaf + 1));
    t->n_used = nk;
    t->sx = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    t->sy = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    t->sz = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk > 0 ? nk : 1));
    for (int64_t k = 0; k < nk; k++) {
        int64_t p = fill[leaf[k]]++;
        t->sx[p] = x[keep[k]]; t->sy[p] = y[keep[k]]; t->sz[p] = z[keep[k]];
        t->perm[p] = keep[k];
    }
    free(fill); free(leaf); free(keep); free(drop);
    if (nk == 0) { oracle_tree_free(t); *status = O_EEMPTY; return NULL; }
    *status = O_OK;
    return t;
}

/* counts: n_in, n_used, n_nan, n_dup, n_knot, nreg, nleaf, rhat, nx, ny */
void oracle_tree_counts(void *h, int64_t *out)
{
    otree *t = (otree *)h;
    out[0] = t->n_in; out[1] = t->n_used; out[2] = t->n_nan; out[3] = t->n_dup;
    out[4] = t->n_knot; out[5] = t->nreg; out[6] = t->nleaf; out[7] = t->rhat;
    out[8] = t->nx; out[9] = t->ny;
}

void oracle_tree_export(void *h, double *kx, double *ky, int64_t *leaf_off, int64_t *perm,
                        double *bounds)
{
    otree *t = (otree *)h;
    int64_t nk = t->lvl_off[t->M] * t->rhat;
    if (kx) memcpy(kx, t->kx, sizeof(double) * (size_t)nk);
    if (ky) memcpy(ky, t->ky, sizeof(double) * (size_t)nk);
    if (leaf_off) memcpy(leaf_off, t->leaf_off, sizeof(int64_t) * (size_t)(t->nleaf + 1));
    if (perm) memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n_used);
    if (bounds)
        for (int64_t g = 0; g < t->nreg; g++) {
            bounds[4 * g + 0] = t->bx0[g]; bounds[4 * g + 1] = t->bx1[g];
            bounds[4 * g + 2] = t->by0[g]; bounds[4 * g + 3] = t->by1[g];
        }
}

/* ------------------------------------------------------- dense algebra -- */

/* In-place lower Cholesky of the n x n row-major A (upper part left as is).
 * Returns 0, or -1 when the matrix is singular: Sec. 1.2 notes that coincident
 * knots make the covariance singular; in finite precision a pivot at or below
 * O_SINGULAR times the largest diagonal entry of A is taken as singular. */
#define O_SINGULAR 1e-12
static int ochol(double *A, int n)
{
    double scale = 0.0;
    for (int j = 0; j < n; j++)
        if (A[j * n + j] > scale) scale = A[j * n + j];
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (!(s > O_SINGULAR * scale)) return -1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    return 0;
}

/* Solve L X = B in place; B is n x nc row-major. */
static void osolve_l(const double *L, int n, double *B, int nc)
{
    for (int i = 0; i < n; i++) {
        for (int c = 0; c < nc; c++) {
            double s = B[i * nc + c];
            for (int k = 0; k < i; k++) s -= L[i * n + k] * B[k * nc + c];
            B[i * nc + c] = s / L[i * n + i];
        }
    }
}

/* Solve L' X = B in place. */
static void osolve_lt(const double *L, int n, double *B, int nc)
{
    for (int i = n - 1; i >= 0; i--) {
        for (int c = 0; c < nc; c++) {
            double s = B[i * nc + c];
            for (int k = i + 1; k < n; k++) s -= L[k * n + i] * B[k * nc + c];
            B[i * nc + c] = s / L[i * n + i];
        }
    }
}

/* S^{-1} B for S = L L' (B overwritten). */
static void ospd_solve(const double *L, int n, double *B, int nc)
{
    osolve_l(L, n, B, nc);
    osolve_lt(L, n, B, nc);
}

static double ologdet_chol(const double *L, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += log(L[i * n + i]);
    return 2.0 * s;
}

/* ---------------------------------------------------------- the method -- */

typedef struct {
    double sigma2, beta, tau2;
} otheta;

static double ocov(const otheta *th, double ax, double ay, double bx, double by)
{
    double dx = ax - bx, dy = ay - by;
    return th->sigma2 * exp(-sqrt(dx * dx + dy * dy) / th->beta);
}

/* Prior quantities of one region R on the current root-to-R path. */
typedef struct {
    int m;
    int64_t g;
    double *W;      /* m blocks R x R: W^l_R = C_l(Q_R, Q_{anc_l(R)}), block m = W^m_R */
    double *K;      /* R x R: K_R = (W^m_R)^{-1} */
    double logdetW; /* log|W^m_R| */
} onode;

typedef struct {
    const otree *t;
    otheta th;
    int task_level;
    double *rd, *ru, *rlw; /* optional per-region records */
} octx;

/* Remainder covariances of a point set P (p points, inside one region of
 * level `lev`) with the knots of its ancestors at levels 1..lev-1:
 *   W^l_P = C(P, Q_{A_l}) - sum_{k<l} W^k_P K_{A_k} (W^k_{A_l})'
 * which is C_l(P, Q_{A_l}) by telescoping the Sec. 1.1 recursion.  Also the
 * self block C_lev(P,P) = C(P,P) - sum_{k<lev} W^k_P K_{A_k} (W^k_P)'.
 * B: (lev-1) blocks of p x R; S: p x p. */
static void oremainder(const octx *c, onode *const *path, int lev, const double *px,
                       const double *py, int p, double *B, double *S)
{
    const otree *t = c->t;
    int R = t->rhat;
    double *G = (double *)malloc(sizeof(double) * (size_t)((lev > 1 ? lev - 1 : 1) * p * R));
    for (int l = 1; l < lev; l++) {
        const onode *A = path[l];
        const double *qx = t->kx + A->g * R, *qy = t->ky + A->g * R;
        double *Wl = B + (size_t)(l - 1) * p * R;
        for (int i = 0; i < p; i++)
            for (int j = 0; j < R; j++) Wl[i * R + j] = ocov(&c->th, px[i], py[i], qx[j], qy[j]);
        for (int k = 1; k < l; k++) {
            const double *Gk = G + (size_t)(k - 1) * p * R;  /* W^k_P K_{A_k} */
            const double *WkA = A->W + (size_t)(k - 1) * R * R; /* W^k_{A_l} */
            for (int i = 0; i < p; i++)
                for (int j = 0; j < R; j++) {
                    double s = 0.0;
                    for (int a = 0; a < R; a++) s += Gk[i * R + a] * WkA[j * R + a];
                    Wl[i * R + j] -= s;
                }
        }
        /* G^l = W^l_P K_{A_l} */
        double *Gl = G + (size_t)(l - 1) * p * R;
        for (int i = 0; i < p; i++)
            for (int j = 0; j < R; j++) {
                double s = 0.0;
                for (int a = 0; a < R; a++) s += Wl[i * R + a] * A->K[a * R + j];
                Gl[i * R + j] = s;
            }
    }
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) S[i * p + j] = ocov(&c->th, px[i], py[i], px[j], py[j]);
    for (int k = 1; k < lev; k++) {
        const double *Gk = G + (size_t)(k - 1) * p * R;
        const double *Wk = B + (size_t)(k - 1) * p * R;
        for (int i = 0; i < p; i++)
            for (int j = 0; j < p; j++) {
                double s = 0.0;
                for (int a = 0; a < R; a++) s += Gk[i * R + a] * Wk[j * R + a];
                S[i * p + j] -= s;
            }
    }
    free(G);
}

/* Leaf c (level M): knots are its observations. Output ATilde (D x D,
 * D=(M-1)R), wTilde (D), d, u. */
static int oleaf(const octx *c, int64_t i, onode *const *path, double *At, double *wt,
                 double *d, double *u)
{
    const otree *t = c->t;
    int M = t->M, R = t->rhat, D = (M - 1) * R;
    int64_t o0 = t->leaf_off[i], o1 = t->leaf_off[i + 1];
    int p = (int)(o1 - o0);
    memset(At, 0, sizeof(double) * (size_t)D * D);
    memset(wt, 0, sizeof(double) * (size_t)D);
    *d = 0.0; *u = 0.0;
    int64_t g = t->lvl_off[M] + i;
    if (p == 0) {
        if (c->rd) { c->rd[g] = 0.0; c->ru[g] = 0.0; c->rlw[g] = NAN; }
        return O_OK;
    }
    const double *px = t->sx + o0, *py = t->sy + o0, *pz = t->sz + o0;
    double *B = (double *)malloc(sizeof(double) * (size_t)((M > 1 ? M - 1 : 1) * p * R));
    double *V = (double *)malloc(sizeof(double) * (size_t)p * p);
    oremainder(c, path, M, px, py, p, B, V);
    for (int a = 0; a < p; a++) V[a * p + a] += c->th.tau2;
    if (ochol(V, p) != 0) { free(B); free(V); return O_ENOTPD; }
    /* Bcat = [B^1 ... B^{M-1} | z], p x (D+1) */
    int nc = D + 1;
    double *X = (double *)malloc(sizeof(double) * (size_t)p * nc);
    for (int a = 0; a < p; a++) {
        for (int l = 1; l < M; l++)
            for (int j = 0; j < R; j++)
                X[a * nc + (l - 1) * R + j] = B[(size_t)(l - 1) * p * R + a * R + j];
        X[a * nc + D] = pz[a];
    }
    double *Y = (double *)malloc(sizeof(double) * (size_t)p * nc);
    memcpy(Y, X, sizeof(double) * (size_t)p * nc);
    ospd_solve(V, p, Y, nc); /* Y = V^{-1} [B | z] */
    for (int a = 0; a < D; a++) {
        for (int b = 0; b < D; b++) {
            double s = 0.0;
            for (int k = 0; k < p; k++) s += X[k * nc + a] * Y[k * nc + b];
            At[a * D + b] = s;
        }
        double s = 0.0;
        for (int k = 0; k < p; k++) s += X[k * nc + a] * Y[k * nc + D];
        wt[a] = s;
    }
    double s = 0.0;
    for (int k = 0; k < p; k++) s += pz[k] * Y[k * nc + D];
    *u = s;
    *d = ologdet_chol(V, p);
    if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = NAN; }
    free(B); free(V); free(X); free(Y);
    return O_OK;
}

/* Region (m, i): prior of R from its ancestors, then the subtree, then the
 * Woodbury step that integrates out eta_R.  Output ATilde ((m-1)R square),
 * wTilde ((m-1)R), d, u. */
static int ovisit(const octx *c, int m, int64_t i, onode *const *path, double *At, double *wt,
                  double *d, double *u)
{
    const otree *t = c->t;
    int M = t->M, R = t->rhat, J = t->J;
    if (m == M) return oleaf(c, i, path, At, wt, d, u);

    /* A subtree with no observation has A = 0 and w = 0, so T = W^m_R and
     * every term of the step is exactly zero (Sec. 1.2 eliminations can empty
     * whole regions): return zeros without forming its prior.  In the region
     * terms its regions read d = u = 0 and log|W^m| = NaN (not formed). */
    {
        int64_t l0 = i, l1 = i + 1;
        for (int l = m; l < M; l++) { l0 *= J; l1 *= J; }
        if (t->leaf_off[l1] == t->leaf_off[l0]) {
            int E0 = (m - 1) * R;
            memset(At, 0, sizeof(double) * (size_t)E0 * E0);
            memset(wt, 0, sizeof(double) * (size_t)E0);
            *d = 0.0;
            *u = 0.0;
            if (c->rd) {
                int64_t a = i, b = i + 1;
                for (int l = m; l <= M; l++) {
                    for (int64_t q = a; q < b; q++) { c->rd[t->lvl_off[l] + q] = 0.0; c->ru[t->lvl_off[l] + q] = 0.0; }
                    a *= J; b *= J;
                }
            }
            return O_OK;
        }
    }

    int64_t g = t->lvl_off[m] + i;
    onode self;
    self.m = m; self.g = g;
    self.W = (double *)malloc(sizeof(double) * (size_t)m * R * R);
    self.K = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *L = (double *)malloc(sizeof(double) * (size_t)R * R);
    const double *qx = t->kx + g * R, *qy = t->ky + g * R;
    oremainder(c, path, m, qx, qy, R, self.W, self.W + (size_t)(m - 1) * R * R);
    memcpy(L, self.W + (size_t)(m - 1) * R * R, sizeof(double) * (size_t)R * R);
    int st = O_OK;
    if (ochol(L, R) != 0) st = O_ENOTPD;
    if (st == O_OK) {
        self.logdetW = ologdet_chol(L, R);
        for (int a = 0; a < R; a++)
            for (int b = 0; b < R; b++) self.K[a * R + b] = (a == b) ? 1.0 : 0.0;
        ospd_solve(L, R, self.K, R);
    }
    if (st != O_OK) { free(self.W); free(self.K); free(L); return st; }

    onode *npath[O_MAXM + 1];
    for (int l = 1; l < m; l++) npath[l] = path[l];
    npath[m] = &self;

    int D = m * R; /* dimension of the children's ATilde */
    double *cA = (double *)malloc(sizeof(double) * (size_t)J * D * D);
    double *cw = (double *)malloc(sizeof(double) * (size_t)J * D);
    double cd[4], cu[4];
    int cst[4];
    int spawn = (m + 1) <= c->task_level;
    for (int j = 0; j < J; j++) {
#pragma omp task if (spawn) default(shared) firstprivate(j)
        cst[j] = ovisit(c, m + 1, i * J + j, npath, cA + (size_t)j * D * D, cw + (size_t)j * D,
                        &cd[j], &cu[j]);
    }
#pragma omp taskwait
    for (int j = 0; j < J; j++)
        if (cst[j] != O_OK && st == O_OK) st = cst[j];
    if (st != O_OK) { free(cA); free(cw); free(self.W); free(self.K); free(L); return st; }

    /* A = sum of the children's ATilde, in child order */
    double *A = (double *)calloc((size_t)D * D, sizeof(double));
    double *w = (double *)calloc((size_t)D, sizeof(double));
    double ds = 0.0, us = 0.0;
    for (int j = 0; j < J; j++) {
        for (int64_t k = 0; k < (int64_t)D * D; k++) A[k] += cA[(size_t)j * D * D + k];
        for (int k = 0; k < D; k++) w[k] += cw[(size_t)j * D + k];
        ds += cd[j]; us += cu[j];
    }
    free(cA); free(cw);
    int E = (m - 1) * R; /* coarser part */
    /* T = W^m_R + A^{m,m} */
    double *T = (double *)malloc(sizeof(double) * (size_t)R * R);
    for (int a = 0; a < R; a++)
        for (int b = 0; b < R; b++)
            T[a * R + b] = self.W[(size_t)(m - 1) * R * R + a * R + b] + A[(E + a) * D + E + b];
    if (ochol(T, R) != 0) st = O_ENOTPD;
    if (st == O_OK) {
        double logdetT = ologdet_chol(T, R);
        /* Z = T^{-1} [A^{m,<m} | w^m], R x (E+1) */
        int nc = E + 1;
        double *Z = (double *)malloc(sizeof(double) * (size_t)R * nc);
        for (int a = 0; a < R; a++) {
            for (int b = 0; b < E; b++) Z[a * nc + b] = A[(E + a) * D + b];
            Z[a * nc + E] = w[E + a];
        }
        ospd_solve(T, R, Z, nc);
        for (int a = 0; a < E; a++) {
            for (int b = 0; b < E; b++) {
                double s = 0.0;
                for (int k = 0; k < R; k++) s += A[a * D + E + k] * Z[k * nc + b];
                At[a * E + b] = A[a * D + b] - s;
            }
            double s = 0.0;
            for (int k = 0; k < R; k++) s += A[a * D + E + k] * Z[k * nc + E];
            wt[a] = w[a] - s;
        }
        double q = 0.0;
        for (int k = 0; k < R; k++) q += w[E + k] * Z[k * nc + E];
        *d = ds + logdetT - self.logdetW;
        *u = us - q;
        if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = self.logdetW; }
        free(Z);
    }
    free(T); free(A); free(w); free(self.W); free(self.K); free(L);
    return st;
}

static int task_level_for(const otree *t)
{
    int lev = 1;
    double cnt = 1.0;
    while (lev < t->M && cnt < 256.0) { lev++; cnt *= t->J; }
    return lev;
}

static int ologlik_one(const otree *t, const double *th3, double *out, double *rd, double *ru,
                       double *rlw, int nthreads)
{
    octx c;
    c.t = t;
    c.th.sigma2 = th3[0]; c.th.beta = th3[1]; c.th.tau2 = th3[2];
    c.rd = rd; c.ru = ru; c.rlw = rlw;
    c.task_level = task_level_for(t);
    if (!(isfinite(c.th.sigma2) && isfinite(c.th.beta) && isfinite(c.th.tau2)) ||
        !(c.th.sigma2 > 0.0 && c.th.beta > 0.0 && c.th.tau2 > 0.0)) {
        *out = NAN;
        return O_EINVAL;
    }
    double d = 0.0, u = 0.0;
    int st = O_OK;
    onode *path[O_MAXM + 1] = {0};
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#pragma omp single
#endif
    {
        double At0[1], wt0[1];
        if (t->M == 1) {
            /* root = leaf: ATilde is 0 x 0 */
            st = oleaf(&c, 0, path, At0, wt0, &d, &u);
        } else {
            st = ovisit(&c, 1, 0, path, At0, wt0, &d, &u);
        }
    }
    if (st != O_OK) { *out = NAN; return st; }
    *out = -0.5 * (d + u + (double)t->n_used * log(2.0 * M_PI));
    return O_OK;
}

/* loglik for a batch of theta = (sigma2, beta, tau2); NaN where a theta fails.
 * Returns the first non-OK status (or OK). */
int oracle_loglik(void *h, const double *theta, int batch, double *out, int nthreads)
{
    const otree *t = (const otree *)h;
    int first = O_OK;
    for (int b = 0; b < batch; b++) {
        int st = ologlik_one(t, theta + 3 * b, out + b, NULL, NULL, NULL, nthreads);
        if (st != O_OK && first == O_OK) first = st;
    }
    return first;
}

/* Per-region partial terms at one theta (arrays of length nreg, global ids):
 * d_R and u_R after R's step (leaves: log|V| and z'V^{-1}z), log|W^m_R| for
 * regions above the leaves (NaN at leaves). */
int oracle_region_terms(void *h, const double *theta, double *rd, double *ru, double *rlw,
                        double *loglik, int nthreads)
{
    const otree *t = (const otree *)h;
    for (int64_t g = 0; g < t->nreg; g++) { rd[g] = NAN; ru[g] = NAN; rlw[g] = NAN; }
    return ologlik_one(t, theta, loglik, rd, ru, rlw, nthreads);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
