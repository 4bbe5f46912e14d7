// Table-driven FP64 log2 and exp2 for the FP64 path's per-pair weights (the method after
// Tang's table-driven logarithm and exponential; the constants and how they were obtained are
// in gen_f64_math_tables.py / f64_math_tables.inc).
//
//   log2(x), x a positive normal double or +inf: x = 2^e m with m in [1, 2); F = 1 + j/1024 from
//     the top 10 bits of m (exact); r = (m - F) / F in [0, 2^-10) (m - F exact, one rounding in
//     the product with 1/F); log2(x) = e + (log2 F + log2(1 + r)), the logarithm by the
//     degree-5 Taylor polynomial of ln(1 + r) / ln 2, its last step adding log2 F. Absolute
//     error about one ulp of max(1, |log2 x|).
//   exp2(y), y < 1023: y <= -1021 gives 0 (far below any weight that matters next to the nearest
//     point's, which is 1); else k = round(256 y) by the 1.5 * 2^52 rounding constant,
//     r = y - k/256 in [-1/512, 1/512] (exact), 2^y = 2^(k >> 8) * 2^((k & 255)/256)
//     * e^(r ln 2) with a degree-4 Taylor polynomial; the power of two is added to the exponent
//     field. Relative error a few ulps.
// The range tests read the operands' bits on the integer pipe, so that the FP64 pipe, GB300's
// scarcest, runs only the arithmetic: 8 and 8 double-precision operations, against several
// times that for the general library functions; the weights of Eq. 1 need the absolute accuracy
// of log2 (it is scaled by alpha / 2 and exponentiated), which these keep.
#pragma once

#include <cstdint>

#include <math_constants.h>

#include "aidw_internal.cuh"

namespace aidw {
namespace f64math {

#include "f64_math_tables.inc"

// Shared-memory copy of the tables for one CTA.
struct Tables {
    double2 lf[1024];  // (log2 F_j, 1 / F_j)
    double e2[256];    // 2^(j/256)
};

// Every thread of the CTA takes part; the caller synchronises before the first use.
__device__ __forceinline__ void load_tables(Tables &t)
{
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        t.lf[i] = make_double2(kLog2F[i], kInvF[i]);
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        t.e2[i] = kExp2J[i];
}

__device__ __forceinline__ int log2_index(double x)
{
    return static_cast<int>((__double_as_longlong(x) >> 42) & 1023);
}

// log2(x) from the table entries (log2 F_j, 1 / F_j) of j = log2_index(x).
__device__ __forceinline__ double log2_finish(double x, double log2f, double invf)
{
    const long long b = __double_as_longlong(x);
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double F = __longlong_as_double((b & 0x000FFC0000000000LL) | 0x3FF0000000000000LL);
    const double r = __dmul_rn(__dsub_rn(m, F), invf);
    double p = __fma_rn(kL2C5, r, kL2C4);
    p = __fma_rn(p, r, kL2C3);
    p = __fma_rn(p, r, kL2C2);
    p = __fma_rn(p, r, kL2C1);
    const double e = static_cast<double>(static_cast<int>(b >> 52) - 1023);
    const double v = __dadd_rn(e, __fma_rn(p, r, log2f));
    return ((b >> 52) & 0x7FF) == 0x7FF ? CUDART_INF : v;  // +inf, and NaN (as +inf)
}

__device__ __forceinline__ double log2_t(double x, const Tables &t)
{
    const double2 lf = t.lf[log2_index(x)];
    return log2_finish(x, lf.x, lf.y);
}

// log2 with the tables read from constant memory (per-query use).
__device__ __forceinline__ double log2_c(double x)
{
    const int j = log2_index(x);
    return log2_finish(x, kLog2F[j], kInvF[j]);
}

__device__ __forceinline__ double exp2_t(double y, const Tables &t)
{
    constexpr double kRound = 6755399441055744.0;  // 1.5 * 2^52
    // y <= -1021 (also -inf): the high word of a negative double grows with its magnitude.
    if (static_cast<uint32_t>(__double2hiint(y)) >= 0xC08FE800u)
        return 0.0;
    const double s = __fma_rn(y, 256.0, kRound);
    const double kd = __dsub_rn(s, kRound);                      // round(256 y)
    const double r = __fma_rn(kd, -0.00390625, y);               // y - k/256, exact
    const long long k = __double_as_longlong(s) - 0x4338000000000000LL;
    double p = __fma_rn(kExpC4, r, kExpC3);
    p = __fma_rn(p, r, kExpC2);
    p = __fma_rn(p, r, kExpC1);
    p = __fma_rn(p, r, kExpC0);
    const double v = __dmul_rn(t.e2[static_cast<int>(k & 255)], p);
    return __longlong_as_double(__double_as_longlong(v) + ((k >> 8) << 52));
}

}  // namespace f64math
}  // namespace aidw
