// ff_math.h -- double-float ("ff") arithmetic on the FP32 pipe: a value is an
// unevaluated pair hi + lo of floats (about 48 significant bits).  GB300
// executes FP32 at 64 times its FP64 rate, so the few places of the mixed
// mode that need more than FP32 accuracy use these error-free transformations
// instead of FP64 instructions.
//
// Building blocks: TwoSum and FastTwoSum (Knuth; Dekker), TwoProd with a
// fused multiply-add, and the double-float add/multiply/square-root built on
// them (Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971).  exp(-x) is table driven (Tang, ACM TOMS
// 15, 1989): x = k ln2/64 + r with |r| <= ln2/128, exp(-x) = 2^(-k/64) exp(-r),
// 2^(-j/64) tabulated as float pairs, exp(-r) by its Taylor series.
//
// Every operation goes through FADD/FMUL/FFMA so that neither nvcc nor the
// host compiler can contract or reassociate it; the host build (CPU tests)
// must use -ffp-contract=off.
#pragma once
#include <math.h>
#include <stdint.h>

#include "ff_tables.h"

#ifdef __CUDACC__
#define MRA_HD __host__ __device__ __forceinline__
#else
#define MRA_HD inline
#endif

namespace mra {

#if defined(__CUDA_ARCH__)
#define FADD(a, b) __fadd_rn((a), (b))
#define FSUB(a, b) __fsub_rn((a), (b))
#define FMUL(a, b) __fmul_rn((a), (b))
#define FFMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define FADD(a, b) ((a) + (b))
#define FSUB(a, b) ((a) - (b))
#define FMUL(a, b) ((a) * (b))
#define FFMA(a, b, c) fmaf((a), (b), (c))
#endif

struct ff {
    float hi, lo;
};

MRA_HD ff ff_from_double(double v)
{
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}
MRA_HD double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

MRA_HD ff two_sum(float a, float b)
{
    const float s = FADD(a, b);
    const float z = FSUB(s, a);
    const float e = FADD(FSUB(a, FSUB(s, z)), FSUB(b, z));
    return ff{s, e};
}
// |a| >= |b|
MRA_HD ff fast_two_sum(float a, float b)
{
    const float s = FADD(a, b);
    return ff{s, FSUB(b, FSUB(s, a))};
}
MRA_HD ff two_prod(float a, float b)
{
    const float p = FMUL(a, b);
    return ff{p, FFMA(a, b, -p)};
}
MRA_HD ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    ff u = fast_two_sum(s.hi, FADD(s.lo, t.hi));
    return fast_two_sum(u.hi, FADD(u.lo, t.lo));
}
MRA_HD ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
MRA_HD ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
// a - b with an absolute error of a few 2^-48 (|a| + |b|) ("sloppy" add:
// one TwoSum of the leading parts, the trailing parts added in FP32).  Enough
// for the updates of a Cholesky factorisation, whose backward error is
// measured against |L| |L'| anyway; 11 operations instead of 20.
MRA_HD ff ff_sub_sloppy(ff a, ff b)
{
    const ff s = two_sum(a.hi, -b.hi);
    return fast_two_sum(s.hi, FADD(s.lo, FSUB(a.lo, b.lo)));
}
// a + b when the sum does not cancel (both non-negative, say): one TwoSum of
// the leading parts, the trailing parts added in FP32; relative error a few
// 2^-48.  11 operations instead of 20.
MRA_HD ff ff_add_sloppy(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, FADD(s.lo, FADD(a.lo, b.lo)));
}
MRA_HD ff ff_add_f(ff a, float b)
{
    const ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, FADD(s.lo, a.lo));
}
MRA_HD ff ff_mul(ff a, ff b)
{
    const ff p = two_prod(a.hi, b.hi);
    const float c = FFMA(a.hi, b.lo, FMUL(a.lo, b.hi));
    return fast_two_sum(p.hi, FADD(p.lo, c));
}
MRA_HD ff ff_sqr(ff a)
{
    const ff p = two_prod(a.hi, a.hi);
    const float c = FMUL(FADD(a.hi, a.hi), a.lo);
    return fast_two_sum(p.hi, FADD(p.lo, c));
}
MRA_HD ff ff_sqrt(ff a)
{
    if (!(a.hi > 0.f)) return ff{0.f, 0.f};
    // s ~ sqrt(a.hi) from the reciprocal square root y, then one Newton step
    // s + (a - s^2) y / 2 with s^2 exact: the error after it is O(ulp^2)
#if defined(__CUDA_ARCH__)
    const float y = rsqrtf(a.hi);
#else
    const float y = 1.0f / sqrtf(a.hi);
#endif
    const float s = FMUL(a.hi, y);
    const ff p = two_prod(s, s);
    const float r = FADD(FSUB(FSUB(a.hi, p.hi), p.lo), a.lo);
    return fast_two_sum(s, FMUL(r, FMUL(0.5f, y)));
}

MRA_HD ff ff_mul_f(ff a, float b)
{
    const ff p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, FFMA(a.lo, b, p.lo));
}

// Sums of products sum_t a_t b_t whose absolute values add up to less than a
// bound known in advance, to an absolute error near 1e-11 of the bound, in
// four FP32 operations a product.  With 2^E > bound, the high sum h starts at
// C = 1.5 * 2^(E + 2) and stays inside [2^(E + 2), 2^(E + 3)), where the FP32
// grid is delta = 2^(E - 21): fma(a, b, h) adds the product rounded onto that
// grid, the change of h is exact (same binade), and fma(a, b, -change) is the
// part of the product left over (|.| <= delta / 2) to within 2^-24 of itself.
// Those parts add up in a second FP32 sum l.  The value is (h - C) + l.
struct grid_acc {
    float h, l;
};
MRA_HD float grid_constant(double bound)
{
#if defined(__CUDA_ARCH__)
    // bound = m 2^E with m in [0.5, 1) for a positive normal bound, read off
    // the exponent field (integer operations instead of FP64 ones)
    const int E = (int)((__double_as_longlong(bound) >> 52) & 0x7ff) - 1022;
#else
    int E;
    frexp(bound, &E); // bound < 2^E
#endif
    return ldexpf(1.5f, E + 2);
}
MRA_HD void grid_init(grid_acc &s, float c)
{
    s.h = c;
    s.l = 0.f;
}
MRA_HD void grid_add(grid_acc &s, float a, float b)
{
    const float h = FFMA(a, b, s.h);
    s.l = FADD(s.l, FFMA(a, b, -FSUB(h, s.h)));
    s.h = h;
}
// float-pair operands: the leading product on the grid, the cross terms
// (below 2^-23 of it) by FP32 FMAs into l
MRA_HD void grid_add(grid_acc &s, ff a, ff b)
{
    const float h = FFMA(a.hi, b.hi, s.h);
    const float p = FFMA(a.hi, b.hi, -FSUB(h, s.h));
    s.l = FFMA(a.hi, b.lo, FFMA(a.lo, b.hi, FADD(s.l, p)));
    s.h = h;
}
MRA_HD ff grid_value(const grid_acc &s, float c) { return two_sum(FSUB(s.h, c), s.l); }
// 1/sqrt(d) for d > 0: FP32 estimate and one Newton step evaluated in pairs.
MRA_HD ff ff_rsqrt(ff d)
{
#if defined(__CUDA_ARCH__)
    const float r = rsqrtf(d.hi);
#else
    const float r = 1.0f / sqrtf(d.hi);
#endif
    const ff t = ff_mul(d, two_prod(r, r));
    const float e = FSUB(FSUB(1.0f, t.hi), t.lo);
    return fast_two_sum(r, FMUL(FMUL(r, e), 0.5f));
}
// 1/d: FP32 estimate and one Newton step evaluated in pairs.
MRA_HD ff ff_rcp(ff d)
{
    const float q = 1.0f / d.hi;
    const ff t = ff_mul_f(d, q);
    const float e = FSUB(FSUB(1.0f, t.hi), t.lo);
    return fast_two_sum(q, FMUL(q, e));
}
// log of a positive pair: natural log of hi plus the first-order term lo/hi.
MRA_HD double ff_log(ff a) { return (double)logf(a.hi) + (double)(a.lo / a.hi); }

// 2^(-j/64) as float pairs; device copy in global memory (per-lane indices
// diverge, which constant memory would serialise).
#ifdef __CUDACC__
static __device__ const ff kFFExp2Dev[64] = MRA_FF_EXP2_TABLE;
#endif
static const ff kFFExp2Host[64] = MRA_FF_EXP2_TABLE;

// exp(-x) for x >= 0 (x as a float pair); 0 below float range.
MRA_HD ff ff_exp_neg(ff x)
{
    if (!(x.hi < 87.0f)) return ff{0.f, 0.f};
#if defined(__CUDA_ARCH__)
    const ff *tab = kFFExp2Dev;
#else
    const ff *tab = kFFExp2Host;
#endif
    const float kf = rintf(FMUL(x.hi, MRA_FF_INV_C));
    const int k = (int)kf;
    // r = x - k (C1 + C2 + C3); k C1 is exact and close to x.hi
    const float t1 = FSUB(x.hi, FMUL(kf, MRA_FF_C1));
    const ff p2 = two_prod(kf, MRA_FF_C2);
    ff r = two_sum(t1, -p2.hi);
    r = fast_two_sum(r.hi, FADD(r.lo, FSUB(FSUB(x.lo, p2.lo), FMUL(kf, MRA_FF_C3))));
    // exp(-r) = 1 - r + r^2/2 - r^3 (1/6 - r/24 + r^2/120), |r| <= ln2/128:
    // 1 - r.hi and + r.hi^2/2 as exact pairs, every other term (each below
    // 2^-24) added in FP32
    const float rh = r.hi, rl = r.lo;
    const ff s0 = fast_two_sum(1.0f, -rh);
    const ff p = two_prod(rh, rh);
    const ff s1 = fast_two_sum(s0.hi, FMUL(p.hi, 0.5f));
    const float poly = FFMA(rh, FFMA(rh, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f);
    const float q = FMUL(FMUL(p.hi, rh), poly);
    float t = FSUB(FADD(s0.lo, s1.lo), rl);
    t = FFMA(p.lo, 0.5f, t);
    t = FFMA(rh, rl, t);
    t = FSUB(t, q);
    const ff e = ff_mul(fast_two_sum(s1.hi, t), tab[k & 63]);
    // times 2^-(k >> 6), 0 <= k >> 6 <= 125 for 0 <= x < 87
#if defined(__CUDA_ARCH__)
    const float sc = __int_as_float((127 - (k >> 6)) << 23);
#else
    const float sc = ldexpf(1.0f, -(k >> 6));
#endif
    return ff{FMUL(e.hi, sc), FMUL(e.lo, sc)};
}
// sigma2 exp(-|p - q| / beta) from float-pair coordinates, sigma2 and 1/beta
MRA_HD ff ff_cov_exp(ff s2, ff ib, ff px, ff py, ff qx, ff qy)
{
    const ff dx = ff_sub_sloppy(px, qx), dy = ff_sub_sloppy(py, qy);
    const ff d = ff_sqrt(ff_add_sloppy(ff_sqr(dx), ff_sqr(dy)));
    return ff_mul(s2, ff_exp_neg(ff_mul(d, ib)));
}
// the same for FP32 coordinates (differences exact by TwoSum)
MRA_HD ff ff_cov_exp(ff s2, ff ib, float px, float py, float qx, float qy)
{
    const ff dx = two_sum(px, -qx), dy = two_sum(py, -qy);
    const ff d = ff_sqrt(ff_add_sloppy(ff_sqr(dx), ff_sqr(dy)));
    return ff_mul(s2, ff_exp_neg(ff_mul(d, ib)));
}

} // namespace mra
