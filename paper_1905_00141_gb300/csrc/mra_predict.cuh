// mra_predict.cuh -- posterior prediction of the latent process at new
// locations: kriging with the MRA covariance of Sec. 1.1 (the model the
// likelihood is evaluated under), computed from the factors of the upward pass.
//
// In whitened form the process is y(s) = sum_{l<M} What^l(s) xi_{R_l(s)} +
// delta(s), with xi_R ~ N(0, I) per region of levels 1..M-1 and delta the
// finest-level remainder (covariance C_M within a leaf, zero across leaves);
// observations z = y(S) + N(0, tau2 I).  For a point s* in leaf R with
// a* = What(s*) (the M-1 ancestor blocks), c = C(S_R, s*) and the leaf's
// factor V_R = L L', Y = L^{-1} U_R, y = L^{-1} z_R:
//   L^{-1} c* = L^{-1} c - Y a*               (c* = C_M(S_R, s*))
//   mean      = a*' xi + (L^{-1} c*)' (y - Y xi)
//   var       = sigma2 - |a*|^2 - |L^{-1} c*|^2 + g' P^{-1} g,
//               g = a* - Y' L^{-1} c*,
// where xi = E[xi | z] and P = I + sum_R U_R' V_R^{-1} U_R is the posterior
// precision of the basis weights.  The upward pass factors P block by block,
// finest level first (Woodbury over the tree); xi comes from the matching
// back substitution (k_down) and g' P^{-1} g from the forward sweep along the
// point's ancestor chain (k_predict), with the same L~ and Z blocks the
// likelihood's quadratic form uses.  Everything here runs in FP64.
#pragma once

namespace mra {

__device__ __forceinline__ double warp_sum_all(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Posterior means of the basis weights, one level top-down:
// xi_R = L~^{-T} (v_R - sum_{k<m} Z^k_R xi_{anc_k(R)}).  One warp per region
// of level m, lanes own rows.
template <int RP>
__global__ void __launch_bounds__(32) k_down(DevTree t, const double *keep, size_t stride, double *xi, int m)
{
    const int64_t i = blockIdx.x, g = t.lvl_off[m] + i;
    const int lane = threadIdx.x, M = t.M, ldk = (M - 2) * RP;
    const double *kp = keep + (size_t)g * stride;
    const double *Lt = kp, *rinv = kp + RP * RP, *v = rinv + RP, *Z = v + RP;
    double acc = lane < RP ? v[lane] : 0.0;
    for (int k = 1; k < m; k++) {
        const int64_t anc = t.lvl_off[k] + anc_index(t, i, m, k);
        const double *xa = xi + (size_t)anc * RP;
        if (lane < RP)
            for (int bc = 0; bc < RP; bc++) acc -= Z[(size_t)lane * ldk + (k - 1) * RP + bc] * xa[bc];
    }
    // L~' x = acc, from the last row up
    for (int a = RP - 1; a >= 0; a--) {
        const double xa = __shfl_sync(0xffffffffu, acc, a) * rinv[a];
        if (lane == a)
            acc = xa;
        else if (lane < a)
            acc -= Lt[(size_t)a * RP + lane] * xa;
    }
    if (lane < RP) xi[(size_t)g * RP + lane] = acc;
}

// One warp per prediction point (theta of batch slot 0).
template <typename T, int RP>
__global__ void __launch_bounds__(256) k_predict(DevTree t, Work<T> w, PredArgs q)
{
    using F = typename FacT<T>::type;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * q.wpb + warp;
    if (p >= q.np) return;
    const int M = t.M, UC = (M - 1) * RP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sa = (double *)smem_raw + (size_t)warp * predict_warp_doubles(M, RP, q.nl);
    double *sxi = sa + UC, *sg = sxi + UC, *sc = sg + UC, *sl = sc + q.nl, *sw = sl + q.nl;
    const int64_t c = q.leaf[p];
    if (c < 0) {
        if (lane == 0) {
            q.mean[p] = qnan();
            q.var[p] = qnan();
        }
        return;
    }
    const double s2 = w.theta[0], ib = 1.0 / w.theta[1];
    const int64_t o0 = t.leaf_off[c];
    const int n = (int)(t.leaf_off[c + 1] - o0);
    const T *Ua = (const T *)q.Ua + (size_t)p * UC;
    for (int j = lane; j < UC; j += 32) {
        sa[j] = (double)Ua[j];
        const int l = j / RP + 1;
        const int64_t anc = t.lvl_off[l] + anc_index(t, c, M, l);
        sxi[j] = q.xi[(size_t)anc * RP + (j % RP)];
    }
    const double x0 = q.px[p], y0 = q.py[p];
    for (int k = lane; k < n; k += 32) sc[k] = cov64(s2, ib, x0 - t.sx[o0 + k], y0 - t.sy[o0 + k]);
    __syncwarp();
    // sl = L^{-1} c
    const int bi = q.bigidx[c];
    const double *y_small = nullptr;
    const F *y_big = nullptr;
    if (bi < 0) {
        const T *Li = w.keep_li + (size_t)c * kKeepLd * kKeepLd; // k-major: Li[k][r] = (L^{-1})_rk
        for (int r = lane; r < n; r += 32) {
            double s = 0.0;
            for (int k = 0; k <= r; k++) s += (double)Li[k * kKeepLd + r] * sc[k];
            sl[r] = s;
        }
        y_small = w.keep_y + (size_t)c * kKeepLd;
    } else {
        // the tiled factor in the large-leaf scratch: lower tiles row-major,
        // diagonal tiles transposed (L_ik at [k][i])
        const double *vb = w.Vbig + q.big[bi].voff;
        const F *V = (const F *)vb;
        y_big = (const F *)(vb + (size_t)n * n);
        const F *rs = y_big + n;
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int k = lane; k < i; k += 32) {
                const F l = (i / TB == k / TB) ? V[(size_t)k * n + i] : V[(size_t)i * n + k];
                s += f_dbl(l) * sl[k];
            }
            s = warp_sum_all(s);
            if (lane == 0) sl[i] = (sc[i] - s) * f_dbl(rs[i]);
            __syncwarp();
        }
    }
    __syncwarp();
    // L^{-1} c* = L^{-1} c - Y a*, and the residual y - Y xi (into sc)
    const T *Y = w.U + (size_t)o0 * UC;
    for (int i = lane; i < n; i += 32) {
        double ya = 0.0, yx = 0.0;
        const T *row = Y + (size_t)i * UC;
        for (int j = 0; j < UC; j++) {
            const double yv = (double)row[j];
            ya += yv * sa[j];
            yx += yv * sxi[j];
        }
        const double yi = y_small ? y_small[i] : f_dbl(y_big[i]);
        sl[i] -= ya;
        sc[i] = yi - yx;
    }
    __syncwarp();
    double mu = 0.0, aa = 0.0, ll = 0.0;
    for (int j = lane; j < UC; j += 32) {
        mu += sa[j] * sxi[j];
        aa += sa[j] * sa[j];
    }
    for (int i = lane; i < n; i += 32) {
        mu += sl[i] * sc[i];
        ll += sl[i] * sl[i];
    }
    mu = warp_sum_all(mu);
    aa = warp_sum_all(aa);
    ll = warp_sum_all(ll);
    // g = a* - Y' L^{-1} c*
    for (int j = lane; j < UC; j += 32) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += (double)Y[(size_t)i * UC + j] * sl[i];
        sg[j] = sa[j] - s;
    }
    __syncwarp();
    // g' P^{-1} g: forward sweep up the ancestor chain with the kept blocks
    double qf = 0.0;
    const int ldk = (M - 2) * RP;
    for (int m = M - 1; m >= 1; m--) {
        const int64_t anc = t.lvl_off[m] + anc_index(t, c, M, m);
        const double *kp = q.keep_up + (size_t)anc * q.keep_stride;
        const double *Lt = kp, *rinv = kp + RP * RP, *Z = kp + RP * RP + 2 * RP;
        double wa = lane < RP ? sg[(m - 1) * RP + lane] : 0.0;
        for (int i = 0; i < RP; i++) {
            const double wi = __shfl_sync(0xffffffffu, wa, i) * rinv[i];
            if (lane == i)
                wa = wi;
            else if (lane > i && lane < RP)
                wa -= Lt[(size_t)lane * RP + i] * wi;
        }
        if (lane < RP) {
            qf += wa * wa;
            sw[lane] = wa;
        }
        __syncwarp();
        for (int col = lane; col < (m - 1) * RP; col += 32) {
            double s = 0.0;
            for (int a = 0; a < RP; a++) s += Z[(size_t)a * ldk + col] * sw[a];
            sg[col] -= s;
        }
        __syncwarp();
    }
    qf = warp_sum_all(qf);
    if (lane == 0) {
        q.mean[p] = mu;
        q.var[p] = s2 - aa - ll + qf;
    }
}

} // namespace mra
