// mra_bigleaf.cuh -- leaf posterior of the large leaves (more observations
// than the largest shared-memory bucket), blocked in 32 x 32 tiles and
// batched over all such leaves and all theta of a pass.
//
// For a leaf with n observations (Sec. 1.1, finest level): V = C(S,S) -
// U U' + tau2 I with U the whitened basis of its observations (n x UC),
// V = L L', d = log|V|, y = L^{-1} z, u = y'y, Y = L^{-1} U and w = Y'y.
// With nt = ceil(n / 32) tile rows the work is the right-looking blocked
// Cholesky, carried along with the two right-hand sides:
//   assemble   every lower tile (I, J) of V                         (1 launch)
//   for k = 0 .. nt-1:
//     potrf    tile (k,k) = L_kk L_kk', d += log|L_kk L_kk'|,
//              y_k = L_kk^{-1} z_k, u += |y_k|^2, Y_k = L_kk^{-1} U_k
//     trsm     L_ik = V_ik L_kk^{-T} (i > k); z_i -= L_ik y_k;
//              U_i -= L_ik Y_k (the right-hand sides use the leading floats
//              of L in both modes' storage type, y in float pairs, so y and Y
//              belong to one operator)
//     update   V_ij -= L_ik L_jk' (k < j <= i)
//   finish     w = Y'y; (d, u) and the status to the leaf's outputs
// One launch covers the tiles of every large leaf that has them at step k
// (host-built item lists), so the launches per pass grow with the largest
// leaf's tile count, not with the number of leaves.
//
// Precision: the factor and the right-hand side z are carried in the factor
// type F (float pairs in the mixed mode, FP64 otherwise); the products of
// the trailing update are exact in the mixed mode (TwoProd of the leading
// parts, FP32 cross terms of a leading and a trailing part), so the factor
// keeps double-float accuracy.  U and Y are in the storage type T.
//
// Scratch of one large leaf (8-byte slots at BigLeaf::voff): V [n][n] (F,
// row-major; lower tiles hold V and then L, the upper triangle of each
// diagonal tile holds that tile's factor transposed as chol_small leaves
// it), z/y [n] (F), 1/L_jj [n] (F), (d, u) [2] (FP64).
#pragma once

namespace mra {

constexpr int TB = kBigTile;

template <typename F>
struct BigView {
    F *V, *y, *rs;
    double *du;
    int n;
    int64_t o0, c;
};

template <typename T>
__device__ __forceinline__ BigView<typename FacT<T>::type> big_view(const DevTree &t, const Work<T> &w,
                                                                    const BigLeaf &bl, int b)
{
    using F = typename FacT<T>::type;
    BigView<F> v;
    v.c = bl.leaf;
    v.o0 = t.leaf_off[bl.leaf];
    v.n = (int)(t.leaf_off[bl.leaf + 1] - v.o0);
    double *base = w.Vbig + (size_t)b * w.V_stride + bl.voff;
    v.V = (F *)base;
    v.y = (F *)(base + (size_t)v.n * v.n);
    v.rs = v.y + v.n;
    v.du = base + (size_t)v.n * v.n + 2 * (size_t)v.n;
    return v;
}

template <typename T, int RP>
__host__ __device__ constexpr size_t smem_big_assemble_bytes(int M)
{
    return (size_t)2 * TB * ((M - 1) * RP + 4) * sizeof(T) + (size_t)4 * TB * 8 + 64;
}

// Deep trees (mixed modes): the U rows of the two tiles in KP column parts.
template <typename T, int RP, int KP>
__host__ __device__ constexpr size_t smem_big_assemble_parts_bytes(int M)
{
    return (size_t)2 * TB * ((M - 1) * RP / KP + 4) * sizeof(T) + (size_t)4 * TB * 8 + 64;
}

// V tile (I, J), I >= J, of a large leaf: C(S_I, S_J) - U_I U_J' (+ tau2 on
// the diagonal), lower part only for I == J.  U U' is the exact float-float
// product sum: large leaves are the dense clusters, where C and U U' agree
// to many digits.
// KP > 1 (FP32 storage only): the rows are read and summed in KP column
// parts, the grid accumulation carried from part to part (the same sums).
template <typename T, int RP, int KP = 1>
__global__ void __launch_bounds__(NT) k_big_assemble(DevTree t, Work<T> w, const BigLeaf *leaves, const BigTile *items)
{
    using F = typename FacT<T>::type;
    static_assert(KP == 1 || sizeof(T) == 4, "column parts: FP32 storage only");
    const BigTile it = items[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const BigView<F> v = big_view(t, w, leaves[it.bl], b);
    const int M = t.M, n = v.n, UC = (M - 1) * RP, KC = UC / KP, LDU = KC + 4;
    const int rI = it.i * TB, rJ = it.j * TB;
    const int nI = min(TB, n - rI), nJ = min(TB, n - rJ);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sUI = (T *)smem_raw;
    T *sUJ = sUI + (size_t)TB * LDU;
    double *sc = (double *)(sUJ + (size_t)TB * LDU); // x_I, y_I, x_J, y_J relative to the parent corner
    const T *Ub = w.U + (size_t)b * w.U_stride + (size_t)v.o0 * UC;
    if (KP == 1) {
        const int cpr = UC * (int)sizeof(T) / 16;
        for (int e = tid; e < nI * cpr; e += NT) {
            const int a = e / cpr, q = e % cpr;
            cp_async16((char *)(sUI + (size_t)a * LDU) + 16 * q, (const char *)(Ub + (size_t)(rI + a) * UC) + 16 * q);
        }
        for (int e = tid; e < nJ * cpr; e += NT) {
            const int a = e / cpr, q = e % cpr;
            cp_async16((char *)(sUJ + (size_t)a * LDU) + 16 * q, (const char *)(Ub + (size_t)(rJ + a) * UC) + 16 * q);
        }
        cp_async_commit();
    }
    const int64_t gp = M > 1 ? t.lvl_off[M - 1] + anc_index(t, v.c, M, M - 1) : -1;
    const double ox = gp >= 0 ? t.cx[gp] : t.sx[v.o0], oy = gp >= 0 ? t.cy[gp] : t.sy[v.o0];
    // coordinates once per point (mixed mode: as float pairs, one conversion a
    // thread; FP64 conversions are slow on this GPU)
    ff *scf = reinterpret_cast<ff *>(sc);
    for (int e = tid; e < 4 * TB; e += NT) {
        const int a = e % TB, which = e / TB; // x_I, y_I, x_J, y_J
        const bool in = which < 2 ? a < nI : a < nJ;
        const int64_t row = v.o0 + (which < 2 ? rI : rJ) + a;
        const double cval = in ? ((which & 1) ? t.sy[row] - oy : t.sx[row] - ox) : 0.0;
        if constexpr (sizeof(T) == 4)
            scf[e] = ff_from_double(cval);
        else
            sc[e] = cval;
    }
    __shared__ double s_ib;
    __shared__ ff s_par[3]; // sigma2, 1/beta, tau2 as float pairs
    set_cov_params<T>(th, &s_ib, s_par);
    if (tid == 2) s_par[2] = ff_from_double(th[2]);
    const int a0 = 2 * (tid / (TB / 2)), q0 = 2 * (tid % (TB / 2));
    T hi[2][2], lo[2][2];
    if constexpr (KP == 1) {
        cp_async_wait<0>();
        __syncthreads();
        dot2x2_exact(sUI + a0 * LDU, sUI + min(a0 + 1, TB - 1) * LDU, sUJ + q0 * LDU, sUJ + min(q0 + 1, TB - 1) * LDU,
                     UC, grid_constant(th[0]), hi, lo);
    } else {
        const float Cq = grid_constant(th[0]);
        grid_acc g[2][2];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) grid_init(g[i][j], Cq);
        const int cpr = KC * (int)sizeof(T) / 16;
        for (int p = 0; p < KP; p++) {
            for (int e = tid; e < nI * cpr; e += NT) {
                const int a = e / cpr, q = e % cpr;
                cp_async16((char *)(sUI + (size_t)a * LDU) + 16 * q,
                           (const char *)(Ub + (size_t)(rI + a) * UC + (size_t)p * KC) + 16 * q);
            }
            for (int e = tid; e < nJ * cpr; e += NT) {
                const int a = e / cpr, q = e % cpr;
                cp_async16((char *)(sUJ + (size_t)a * LDU) + 16 * q,
                           (const char *)(Ub + (size_t)(rJ + a) * UC + (size_t)p * KC) + 16 * q);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            dot2x2_grid_add(g, sUI + a0 * LDU, sUI + min(a0 + 1, TB - 1) * LDU, sUJ + q0 * LDU,
                            sUJ + min(q0 + 1, TB - 1) * LDU, KC);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const ff gv = grid_value(g[i][j], Cq);
                hi[i][j] = gv.hi;
                lo[i][j] = gv.lo;
            }
    }
    const double tau2 = th[2], ib64 = s_ib; // after the barriers above (s_ib)
    const ff s2f = s_par[0], ibf = s_par[1], tau2f = s_par[2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int a = a0 + i, q = q0 + j;
            if (a >= nI || q >= nJ || (it.i == it.j && q > a)) continue;
            const bool diag = it.i == it.j && a == q;
            F val;
            if constexpr (sizeof(T) == 4) {
                const ff cv = ff_cov_exp(s2f, ibf, scf[a], scf[TB + a], scf[2 * TB + q], scf[3 * TB + q]);
                val = ff_sub_sloppy(cv, ff{(float)hi[i][j], (float)lo[i][j]});
                if (diag) val = ff_add_sloppy(val, tau2f);
            } else {
                const double cv = cov64(th[0], ib64, sc[a] - sc[2 * TB + q], sc[TB + a] - sc[3 * TB + q]);
                val = cancel_sub(cv, hi[i][j], lo[i][j]) + (diag ? tau2 : 0.0);
            }
            v.V[(size_t)(rI + a) * n + rJ + q] = val;
        }
}

template <typename T, int RP>
__host__ __device__ constexpr size_t smem_big_potrf_bytes(int M)
{
    return (size_t)TB * (TB + 1) * 8 + (size_t)(3 * TB + 4) * 8 + 8 * 8 + (size_t)((tri_count(TB) * 2 + 15) & ~15) +
           64 + (size_t)TB * ((M - 1) * RP + 4) * sizeof(T) + 64;
}

// Step k, diagonal tile: factor, log-determinant, and the diagonal solves of
// the two right-hand sides.
template <typename T, int RP>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 4 : 1)) k_big_potrf(DevTree t, Work<T> w, const BigLeaf *leaves, const BigTile *items,
                                                  int k)
{
    using F = typename FacT<T>::type;
    const BigTile it = items[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const BigView<F> v = big_view(t, w, leaves[it.bl], b);
    const int M = t.M, n = v.n, UC = (M - 1) * RP, LDU = UC + 4;
    const int r0 = k * TB, nk = min(TB, n - r0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sL = (F *)smem_raw;                    // TB x (TB+1)
    F *sy = sL + TB * (TB + 1);               // TB
    F *srs = sy + TB;                         // TB + 2
    F *sr2 = srs + TB + 2;                    // TB + 2
    double *red = (double *)(sr2 + TB + 2);   // 8
    int *flag = (int *)((unsigned char *)(red + 8) + ((tri_count(TB) * 2 + 15) & ~15));
    T *sU = (T *)(flag + 16);                 // TB x LDU
    T *Ub = w.U + (size_t)b * w.U_stride + (size_t)(v.o0 + r0) * UC;
    {
        const int cpr = UC * (int)sizeof(T) / 16;
        for (int e = tid; e < nk * cpr; e += NT) {
            const int a = e / cpr, q = e % cpr;
            cp_async16((char *)(sU + (size_t)a * LDU) + 16 * q, (const char *)(Ub + (size_t)a * UC) + 16 * q);
        }
        cp_async_commit();
    }
    if (tid == 0) flag[0] = 0;
    for (int e = tid; e < nk * nk; e += NT) {
        const int a = e / nk, q = e % nk;
        if (q <= a) sL[a * (TB + 1) + q] = v.V[(size_t)(r0 + a) * n + r0 + q];
    }
    for (int a = tid; a < nk; a += NT) sy[a] = k == 0 ? f_of<F>(t.sz[v.o0 + a]) : v.y[r0 + a];
    __syncthreads();
    if constexpr (sizeof(T) == 4)
        chol_blocked<TB>(sL, TB + 1, nk, srs, flag, MRA_SINGULAR, red);
    else
        chol_small<F, (tri_count(TB) + NT - 1) / NT>(sL, TB + 1, nk, srs, sr2, flag, MRA_SINGULAR);
    const double ld = logdet_small(sL, TB + 1, nk, red);
    // factor (transposed, upper triangle of the tile) and 1/L_jj to the scratch
    for (int e = tid; e < nk * nk; e += NT) {
        const int j = e / nk, i = e % nk;
        if (i >= j) v.V[(size_t)(r0 + j) * n + r0 + i] = sL[j * (TB + 1) + i];
    }
    for (int j = tid; j < nk; j += NT) v.rs[r0 + j] = srs[j];
    fwd_solve_vec_lead<F, TB>(sL, TB + 1, srs, nk, sy);
    if (tid < 32) {
        F q = tid < nk ? f_sqr(sy[tid]) : f_of<F>(0.0);
        q = warp_sum_f(q);
        if (tid == 0) red[0] = f_dbl(q);
    }
    for (int a = tid; a < nk; a += NT) v.y[r0 + a] = sy[a];
    cp_async_wait<0>();
    __syncthreads();
    const double uk = red[0];
    fwd_solve_warp<T, TB>(sL, TB + 1, srs, sU, 1, LDU, sU, LDU, UC, nk);
    {
        const int cpr = UC * (int)sizeof(T) / 16;
        for (int e = tid; e < nk * cpr; e += NT) {
            const int a = e / cpr, q = e % cpr;
            reinterpret_cast<int4 *>(Ub + (size_t)a * UC)[q] = reinterpret_cast<const int4 *>(sU + (size_t)a * LDU)[q];
        }
    }
    if (tid == 0) {
        v.du[0] = (k == 0 ? 0.0 : v.du[0]) + ld;
        v.du[1] = (k == 0 ? 0.0 : v.du[1]) + uk;
        if (flag[0]) w.status[b] = ST_ENOTPD;
    }
}

constexpr int kBigUcChunk = 64;

template <typename T, int RP>
__host__ __device__ constexpr size_t smem_big_trsm_bytes()
{
    return (size_t)2 * TB * (TB + 1) * 8 + (size_t)2 * TB * 8 + (size_t)2 * TB * kBigUcChunk * sizeof(T) + 64;
}

// Step k, tile column below the diagonal: L_ik = V_ik L_kk^{-T}, then the
// right-hand sides of row block i take their share of block k.  The rows of
// Y_k (final since step k's diagonal tile) are staged kBigUcChunk columns at
// a time into two buffers by asynchronous copies, the first before the
// solve, each next one while the previous is used.
template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_big_trsm(DevTree t, Work<T> w, const BigLeaf *leaves, const BigTile *items,
                                                 int k)
{
    using F = typename FacT<T>::type;
    const BigTile it = items[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const BigView<F> v = big_view(t, w, leaves[it.bl], b);
    const int M = t.M, n = v.n, UC = (M - 1) * RP;
    const int rk = k * TB, nk = min(TB, n - rk), ri = it.i * TB, ni = min(TB, n - ri);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sK = (F *)smem_raw;          // factor of tile (k,k), transposed: sK[m][c] = L_cm (c >= m)
    F *sA = sK + TB * (TB + 1);     // tile (i,k), then L_ik
    F *srs = sA + TB * (TB + 1);    // TB
    F *syk = srs + TB;              // TB
    T *sY = (T *)(syk + TB);        // 2 x TB x kBigUcChunk
    T *Ui = w.U + (size_t)b * w.U_stride + (size_t)(v.o0 + ri) * UC;
    const T *Yk = w.U + (size_t)b * w.U_stride + (size_t)(v.o0 + rk) * UC;
    // columns [cb, cb + kBigUcChunk) of the nk rows of Y_k into buffer q, zeros
    // past the tile and past UC (a multiple of 16 elements, so a 16-byte
    // vector is all in or all out)
    auto stage_y = [&](int cb, int q) {
        constexpr int V = 16 / (int)sizeof(T), VPR = kBigUcChunk / V;
        T *dst = sY + (size_t)q * TB * kBigUcChunk;
        for (int e = tid; e < TB * VPR; e += NT) {
            const int m = e / VPR, cc = (e % VPR) * V;
            if (m < nk && cb + cc < UC)
                cp_async16(dst + m * kBigUcChunk + cc, Yk + (size_t)m * UC + cb + cc);
            else
#pragma unroll
                for (int q2 = 0; q2 < V; q2++) dst[m * kBigUcChunk + cc + q2] = T(0);
        }
        cp_async_commit();
    };
    stage_y(0, 0);
    for (int e = tid; e < nk * nk; e += NT) {
        const int m = e / nk, c = e % nk;
        if (c >= m) sK[m * (TB + 1) + c] = v.V[(size_t)(rk + m) * n + rk + c];
    }
    for (int e = tid; e < ni * nk; e += NT) {
        const int r = e / nk, c = e % nk;
        sA[r * (TB + 1) + c] = v.V[(size_t)(ri + r) * n + rk + c];
    }
    for (int m = tid; m < nk; m += NT) {
        srs[m] = v.rs[rk + m];
        syk[m] = v.y[rk + m];
    }
    __syncthreads();
    // rows r = warp + 8q; lanes own columns; x_m final at step m, broadcast
    {
        const int warp = tid >> 5, lane = tid & 31;
        constexpr int RPW = TB / (NT / 32);
        F a[RPW];
#pragma unroll
        for (int q = 0; q < RPW; q++) {
            const int r = warp + (NT / 32) * q;
            a[q] = (r < ni && lane < nk) ? sA[r * (TB + 1) + lane] : f_of<F>(0.0);
        }
        for (int m = 0; m < nk; m++) {
            const F lcm = lane > m && lane < nk ? sK[m * (TB + 1) + lane] : f_of<F>(0.0);
            const F rm = srs[m];
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const F xm = f_shfl(f_mul(a[q], rm), m);
                a[q] = lane == m ? xm : f_sub(a[q], f_mul(lcm, xm));
            }
        }
#pragma unroll
        for (int q = 0; q < RPW; q++) {
            const int r = warp + (NT / 32) * q;
            if (r < ni && lane < nk) {
                sA[r * (TB + 1) + lane] = a[q];
                v.V[(size_t)(ri + r) * n + rk + lane] = a[q];
            }
        }
        __syncthreads();
        // z_i -= L_ik y_k
#pragma unroll
        for (int q = 0; q < RPW; q++) {
            const int r = warp + (NT / 32) * q;
            F p = lane < nk && r < ni ? f_mul(f_lead(sA[r * (TB + 1) + lane]), syk[lane]) : f_of<F>(0.0);
            p = warp_sum_f(p);
            if (lane == 0 && r < ni) v.y[ri + r] = f_sub(k == 0 ? f_of<F>(t.sz[v.o0 + ri + r]) : v.y[ri + r], p);
        }
    }
    // U_i -= L_ik Y_k, kBigUcChunk columns at a time
    constexpr int CPT = TB * kBigUcChunk / NT; // outputs per thread (8)
    const int r = tid / (kBigUcChunk / CPT), c0 = (tid % (kBigUcChunk / CPT)) * CPT;
    const int nchunk = (UC + kBigUcChunk - 1) / kBigUcChunk;
    for (int ci = 0; ci < nchunk; ci++) {
        const int cb = ci * kBigUcChunk;
        if (ci + 1 < nchunk) {
            stage_y(cb + kBigUcChunk, (ci + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *sYc = sY + (size_t)(ci & 1) * TB * kBigUcChunk;
        if (r < ni) {
            // this thread's U values, loaded before the products
            T uo[CPT];
#pragma unroll
            for (int cc = 0; cc < CPT; cc++) uo[cc] = cb + c0 + cc < UC ? Ui[(size_t)r * UC + cb + c0 + cc] : T(0);
            T acc[CPT];
#pragma unroll
            for (int cc = 0; cc < CPT; cc++) acc[cc] = T(0);
            for (int m = 0; m < nk; m++) {
                const T l = (T)f_hi(sA[r * (TB + 1) + m]);
#pragma unroll
                for (int cc = 0; cc < CPT; cc++) acc[cc] = fma(l, sYc[m * kBigUcChunk + c0 + cc], acc[cc]);
            }
#pragma unroll
            for (int cc = 0; cc < CPT; cc++)
                if (cb + c0 + cc < UC) Ui[(size_t)r * UC + cb + c0 + cc] = uo[cc] - acc[cc];
        }
        __syncthreads();
    }
}

template <typename T, int RP>
__host__ __device__ constexpr size_t smem_big_update_bytes()
{
    return (size_t)2 * TB * (TB + 1) * 8 + 64;
}

// Step k, trailing tile (i, j), k < j <= i: V_ij -= L_ik L_jk'.
template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_big_update(DevTree t, Work<T> w, const BigLeaf *leaves, const BigTile *items,
                                                   int k)
{
    using F = typename FacT<T>::type;
    const BigTile it = items[blockIdx.x];
    const int b = blockIdx.y, tid = threadIdx.x;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const BigView<F> v = big_view(t, w, leaves[it.bl], b);
    const int n = v.n;
    const int rk = k * TB, nk = min(TB, n - rk);
    const int ri = it.i * TB, ni = min(TB, n - ri), rj = it.j * TB, nj = min(TB, n - rj);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *sLi = (F *)smem_raw;
    F *sLj = sLi + TB * (TB + 1);
    for (int e = tid; e < TB * TB; e += NT) {
        const int r = e / TB, m = e % TB;
        sLi[r * (TB + 1) + m] = (r < ni && m < nk) ? v.V[(size_t)(ri + r) * n + rk + m] : f_of<F>(0.0);
        sLj[r * (TB + 1) + m] = (r < nj && m < nk) ? v.V[(size_t)(rj + r) * n + rk + m] : f_of<F>(0.0);
    }
    __syncthreads();
    const int a0 = 2 * (tid / (TB / 2)), q0 = 2 * (tid % (TB / 2));
    F sum[2][2];
    if constexpr (sizeof(T) == 4) {
        // Rows of L satisfy sum_m L_am^2 = V_aa <= sigma2 + tau2, so every
        // partial sum of |L_am L_qm| stays below sigma2 + tau2
        // (Cauchy-Schwarz): grid accumulation of ff_math.h.
        const float Cq = grid_constant(th[0] + th[2]);
        grid_acc g[2][2];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) grid_init(g[i][j], Cq);
        for (int m = 0; m < nk; m++) {
            const ff x[2] = {sLi[a0 * (TB + 1) + m], sLi[(a0 + 1) * (TB + 1) + m]};
            const ff y[2] = {sLj[q0 * (TB + 1) + m], sLj[(q0 + 1) * (TB + 1) + m]};
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) grid_add(g[i][j], x[i], y[j]);
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) sum[i][j] = grid_value(g[i][j], Cq);
    } else {
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                double acc = 0.0;
                for (int m = 0; m < nk; m++) acc = fma(sLi[(a0 + i) * (TB + 1) + m], sLj[(q0 + j) * (TB + 1) + m], acc);
                sum[i][j] = acc;
            }
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int a = a0 + i, q = q0 + j;
            if (a < ni && q < nj && (it.i != it.j || q <= a)) {
                F *p = v.V + (size_t)(ri + a) * n + rj + q;
                *p = f_sub(*p, sum[i][j]);
            }
        }
}

// Per leaf after the last step: w = Y'y and the (d, u) terms.
template <typename T, int RP>
__global__ void __launch_bounds__(NT) k_big_finish(DevTree t, Work<T> w, const BigLeaf *leaves)
{
    using F = typename FacT<T>::type;
    const int b = blockIdx.y;
    const double *th = w.theta + 3 * b;
    if (!theta_ok(th)) return;
    const BigView<F> v = big_view(t, w, leaves[blockIdx.x], b);
    const int M = t.M, UC = (M - 1) * RP;
    const T *Y = w.U + (size_t)b * w.U_stride + (size_t)v.o0 * UC;
    gram_vec(Y, UC, UC, v.y, v.n, w.leaf_w + (size_t)b * w.leafw_stride + (size_t)v.c * UC);
    if (threadIdx.x == 0) {
        double *du = w.leaf_du + (size_t)b * w.leafdu_stride + 2 * v.c;
        du[0] = v.du[0];
        du[1] = v.du[1];
        if (w.reg_du) {
            double *r = w.reg_du + (size_t)b * w.regdu_stride + 2 * (t.lvl_off[M] + v.c);
            r[0] = v.du[0];
            r[1] = v.du[1];
        }
    }
}

} // namespace mra
