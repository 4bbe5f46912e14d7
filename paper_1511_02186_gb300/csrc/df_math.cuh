// Double-float arithmetic for the AIDW_F64X phase-2 scan: a value is the unevaluated sum hi + lo
// of two floats (about 48 significant bits), computed on the FP32 pipes, which on GB300 run at
// 64 times the rate of the FP64 pipe (128 FP32 lanes against 2 FP64 per clock per SM).
//
// Building blocks: the error-free sum of two floats (Knuth's two-sum, and Dekker's fast two-sum
// when the first operand's exponent is at least the second's) and the error-free product by one
// fused multiply-add. Every operation is written with the _rn intrinsics so that the compiler
// neither contracts nor reorders them.
//
// The weight of one (query, data point) pair, w = 2^(-kappa log2(d^2 / d1^2)) with kappa = alpha/2
// (Eq. 1 with the nearest distance d1 factored out, so that w <= 1):
//   log2(d^2) = e + log2(F_j) + log2(1 + r): e and the 8-bit index j read from the FP64 d^2's
//     bits, m - F_j (44 bits) split exactly into two floats, u = r / ln 2 by the table pair
//     1 / (F_j ln 2), then log2(1 + r) = u - (ln 2 / 2) u^2 + u^3 (c3 + c4 u + c5 u^2 + c6 u^3)
//     with the first two terms in double-float (|u| < 2^-7.47).
//   log2(d^2 / d1^2) = (e - e1) + (f - f1), f = log2 F_j + log2(1 + r) and d1^2 = 2^e1 2^f1
//     split the same way per query: the integer part is exact and f - f1 is formed exactly from
//     the two normalised pairs, so the result carries an absolute error of about 2^-48 (1 +
//     |result|) even where d is close to d1, and is exactly 0 at d = d1.
//   2^y: k = round(128 y) (|y| <= 127), t = (y - k/128) ln 2 in double-float (|t| < 2^-8.5),
//     e^t = 1 + t + t^2/2 + t^3 (1/6 + t/24 + t^2/120), times the table pair 2^((k & 127)/128)
//     and the exact power of two 2^(k >> 7). y <= -127 gives w = 0 (below 2^-126 of the nearest
//     point's weight).
// Per pair the relative error of w is about 2^-47 (1 + |y|); the double-float sums of Eq. 1 add
// about 2^-44 of the sum of the magnitudes at worst.
#pragma once

#include <cstdint>

#include "aidw_internal.cuh"

namespace aidw {
namespace dfm {

#include "df_math_tables.inc"

// Shared-memory copy of the tables for one CTA.
struct Tables {
    float4 lg[256];  // (1/(F_j ln 2) hi, lo, log2 F_j hi, lo)
    float2 ex[128];  // 2^(k/128) hi, lo
};

// Every thread of the CTA takes part; the caller synchronises before the first use.
__device__ __forceinline__ void load_tables(Tables &t)
{
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        t.lg[i] = make_float4(kDfInvFLn2[2 * i], kDfInvFLn2[2 * i + 1], kDfLog2F[2 * i],
                              kDfLog2F[2 * i + 1]);
    for (int i = threadIdx.x; i < 128; i += blockDim.x)
        t.ex[i] = make_float2(kDfExp2K[2 * i], kDfExp2K[2 * i + 1]);
}

// s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when a == 0 or exponent(a) >= exponent(b).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (ph, pl) ~ (ah + al)(bh + bl): ah bh exact, the cross terms rounded (al bl dropped).
__device__ __forceinline__ void mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    ph = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -ph);
    pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
}

// Accurate sum of two double-floats (both parts through two-sum), normalised.
__device__ __forceinline__ void add(float &h, float &l, float bh, float bl)
{
    float s, e, t, f;
    two_sum(h, bh, s, e);
    two_sum(l, bl, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, h, l);
}

// float of the integer v, |v| < 2^22, without the conversion unit.
__device__ __forceinline__ float small_int_to_float(int v)
{
    return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// log2 of a positive normal (or +inf) double x as e + (lh + ll) + (sh + sl): e the exponent,
// lh + ll = log2 F_j, sh + sl = log2(1 + r) with |sh| < 2^-7.4.
struct LogParts {
    int e;
    float lh, ll, sh, sl;
};

__device__ __forceinline__ LogParts log2_parts(double x, const Tables &t)
{
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    LogParts p;
    p.e = static_cast<int>(hi >> 20) - 1023;
    const int j = static_cast<int>((hi >> 12) & 255u);
    // m - F_j = (A 2^22 + C) 2^-52 with A the next 22 mantissa bits and C the last 22; each
    // becomes a float exactly as (1 + bits 2^-22) - 1, scaled.
    const uint32_t a = (__funnelshift_l(lo, hi, 11) & 0x7FFFFEu) | 0x3F800000u;
    const uint32_t c = ((lo << 1) & 0x7FFFFEu) | 0x3F800000u;
    const float th = __fmaf_rn(__uint_as_float(a), 0x1p-8f, -0x1p-8f);
    const float tl = __fmaf_rn(__uint_as_float(c), 0x1p-30f, -0x1p-30f);
    const float4 g = t.lg[j];
    // u = (m - F_j) / (F_j ln 2)
    float uh, ul;
    mul(th, tl, g.x, g.y, uh, ul);
    // (ln 2 / 2) u^2 in double-float, the rest in float.
    const float q = __fmul_rn(uh, uh);
    const float qe = __fmaf_rn(uh, uh, -q);
    const float ql = __fmaf_rn(__fadd_rn(uh, uh), ul, qe);
    float ph, pl;
    mul(kDfC2h, kDfC2l, q, ql, ph, pl);
    // The pair (uh, ul) is not normalised (ul can reach 2^-22 uh), so the float terms take
    // u = uh + ul rounded once.
    const float u1 = __fadd_rn(uh, ul);
    float c3 = __fmaf_rn(u1, kDfC6, kDfC5);
    c3 = __fmaf_rn(u1, c3, kDfC4);
    c3 = __fmaf_rn(u1, c3, kDfC3);
    const float tail = __fmul_rn(__fmul_rn(__fmul_rn(u1, u1), u1), c3);
    float se;
    fast_two_sum(uh, ph, p.sh, se);
    p.sl = __fadd_rn(__fadd_rn(__fadd_rn(ul, pl), tail), se);
    p.lh = g.z;
    p.ll = g.w;
    return p;
}

// log2 of the mantissa, log2 F_j + log2(1 + r), normalised.
__device__ __forceinline__ void frac_log(const LogParts &p, float &fh, float &fl)
{
    float s, e;
    two_sum(p.lh, p.sh, s, e);
    e = __fadd_rn(e, __fadd_rn(p.ll, p.sl));
    fast_two_sum(s, e, fh, fl);
}

// Per-query constants of log2(d^2 / d1^2): d1^2 = 2^e1 * 2^(f1h + f1l).
struct RefLog {
    int e1;
    float f1h, f1l;
};

__device__ __forceinline__ RefLog ref_log(double d1sq, const Tables &t)
{
    const LogParts p = log2_parts(d1sq, t);
    RefLog r;
    r.e1 = p.e;
    frac_log(p, r.f1h, r.f1l);
    return r;
}

// log2(d^2 / d1^2) as (vh, vl): the mantissa logarithms are formed by the same operations as
// the reference's, so d^2 == d1^2 gives exactly 0 (the nearest point's weight is exactly 1).
__device__ __forceinline__ void log2_ratio(double d2, const RefLog &ref, const Tables &t,
                                           float &vh, float &vl)
{
    const LogParts p = log2_parts(d2, t);
    float fh, fl, s, e1, e2;
    frac_log(p, fh, fl);
    two_sum(fh, -ref.f1h, s, e2);  // |s| < 1
    // d^2 = +inf (a padding point): a ratio beyond every weight's reach.
    const float a = p.e == 1024 ? 1e38f : small_int_to_float(p.e - ref.e1);
    fast_two_sum(a, s, vh, e1);    // a is an integer
    vl = __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(fl, ref.f1l));
}

// 2^(yh + yl) as (wh, wl); yh <= -127 (or -inf, or NaN) gives 0, yh is clamped at 126.
__device__ __forceinline__ void exp2_df(float yh, float yl, const Tables &t, float &wh, float &wl)
{
    const float y = fminf(fmaxf(yh, -127.0f), 126.0f);
    yl = fminf(fmaxf(yl, -1.0f), 1.0f);  // bounded where yh was clamped (then w is 0 anyway)
    const float kf = __fmaf_rn(y, 128.0f, 12582912.0f);  // 1.5 * 2^23 + round(128 y)
    const int k = __float_as_int(kf) - 0x4B400000;
    const float kd = __fsub_rn(kf, 12582912.0f);
    float sh, sl;  // y - k/128: the first part exact; |yl| may be large next to it
    two_sum(__fmaf_rn(kd, -0.0078125f, y), yl, sh, sl);
    float th, tl;
    mul(sh, sl, kDfLn2h, kDfLn2l, th, tl);
    // e^t - 1 = t + t^2/2 + (t^2/2) t (1/3 + t/12 + t^2/60)
    const float half = __fmul_rn(0.5f, th);
    const float q = __fmul_rn(half, th);
    const float qe = __fmaf_rn(half, th, -q);
    const float ql = __fmaf_rn(th, tl, qe);
    float c = __fmaf_rn(th, 1.0f / 60.0f, 1.0f / 12.0f);
    c = __fmaf_rn(th, c, 1.0f / 3.0f);
    const float tail = __fmul_rn(__fmul_rn(q, th), c);
    float mh, me;
    fast_two_sum(th, q, mh, me);
    const float ml = __fadd_rn(__fadd_rn(__fadd_rn(tl, ql), tail), me);
    const float2 T = t.ex[k & 127];
    float ph, pl;
    mul(T.x, T.y, mh, ml, ph, pl);
    float we;
    fast_two_sum(T.x, ph, wh, we);
    wl = __fadd_rn(__fadd_rn(T.y, pl), we);
    const float scale = __int_as_float(((k >> 7) + 127) << 23);  // 2^(k >> 7); 0 at k >> 7 = -127
    wh = __fmul_rn(wh, scale);
    wl = __fmul_rn(wl, scale);
}

}  // namespace dfm
}  // namespace aidw
