// Table-driven FP64 log2 and exp2 for the FP64 path's per-pair weights (the method after
// Tang's table-driven logarithm and exponential; the constants and how they were obtained are
// in gen_f64_math_tables.py / f64_math_tables.inc).
//
//   log2(x), x a positive normal double or +inf: x = 2^e m with m in [1, 2); F = 1 + j/2048
//     from the top 11 bits of m (exact); r = (m - F) / F in [0, 2^-11) (m - F exact, one
//     rounding in the product with 1/F); log2(x) = e + (log2 F + log2(1 + r)), the logarithm by
//     the degree-4 Taylor polynomial of ln(1 + r) / ln 2, its last step adding log2 F. Absolute
//     error about one ulp of max(1, |log2 x|).
//   exp2(y), y < 1023: y <= -1021 gives 0 (far below any weight that matters next to the nearest
//     point's, which is 1); else k = round(2048 y), r = y - k/2048 in [-2^-12, 2^-12] (exact),
//     2^y = 2^(k >> 11) * T_j e^(r ln 2), T_j = 2^(j/2048), j = k & 2047, with the degree-3
//     Taylor polynomial multiplied out with T_j (its four coefficients tabulated per j, so three
//     fused steps evaluate it); the power of two is added to the exponent field. Relative error
//     a few ulps.
// GB300 runs FP64 arithmetic at 2 operations per clock per SM against 64 integer operations, so
// every step whose result is exact is done on the integer pipe from the operands' bits: the
// range tests, m - F, e as a double, and exp2's reduction (k and r). The FP64 pipe runs only the
// rounded operations: 6 for log2 and 3 for exp2, against several times that for the general
// library functions; the weights of Eq. 1 need the absolute accuracy of log2 (it is scaled by
// alpha / 2 and exponentiated), which these keep.
#pragma once

#include <cstdint>

#include <math_constants.h>

#include "aidw_internal.cuh"

namespace aidw {
namespace f64math {

#include "f64_math_tables.inc"

constexpr int kLogBits = 11;                   // log2 table index bits
constexpr int kLogN = 1 << kLogBits;           // 2,048 entries
constexpr int kExpBits = 11;                   // exp2 table: 2^(j / 2048)
constexpr int kExpN = 1 << kExpBits;
constexpr long long kMant = 0x000FFFFFFFFFFFFFLL;

// Shared-memory copy of the tables for one CTA (96 KB: dynamic shared memory).
struct Tables {
    double2 lf[kLogN];  // (log2 F_j, 1 / F_j)
    double2 ea[kExpN];  // (T_j, T_j ln 2)
    double2 eb[kExpN];  // (T_j (ln 2)^2 / 2, T_j (ln 2)^3 / 6)
};
constexpr size_t kTablesBytes = sizeof(Tables);

// Every thread of the CTA takes part; the caller synchronises before the first use.
__device__ __forceinline__ void load_tables(Tables &t)
{
    for (int i = threadIdx.x; i < kLogN; i += blockDim.x)
        t.lf[i] = make_double2(kLog2F[i], kInvF[i]);
    for (int i = threadIdx.x; i < kExpN; i += blockDim.x) {
        t.ea[i] = make_double2(kExp2J[i], kExp2C1[i]);
        t.eb[i] = make_double2(kExp2C2[i], kExp2C3[i]);
    }
}

__device__ __forceinline__ int log2_index(double x)
{
    return static_cast<int>((__double_as_longlong(x) >> (52 - kLogBits)) & (kLogN - 1));
}

// The double a * 2^(q - 1075) for an integer 0 <= a < 2^53 and a biased exponent q with
// q - 1075 + 63 - clz(a) >= -1022 (the result is normal or zero): exact, integer operations only.
__device__ __forceinline__ double scaled_int(unsigned long long a, int q)
{
    const int lz = __clzll(a);  // >= 11
    const unsigned long long mant = (a << (lz - 11)) & static_cast<unsigned long long>(kMant);
    const unsigned long long ex = static_cast<unsigned long long>(q + 11 - lz) << 52;
    return a == 0 ? 0.0 : __longlong_as_double(static_cast<long long>(ex | mant));
}

// -v if neg, else v, by the sign bit (an integer operation: a negation written in FP64 would
// run on the FP64 pipe).
__device__ __forceinline__ double flip_sign(double v, bool neg)
{
    return __longlong_as_double(__double_as_longlong(v) ^
                                (static_cast<long long>(neg) << 63));
}

// The double of a small integer |e| <= 2048, exact, integer operations only.
__device__ __forceinline__ double small_int(int e)
{
    const unsigned a = static_cast<unsigned>(e < 0 ? -e : e);
    return flip_sign(scaled_int(a, 1075), e < 0);
}

// log2(x) from the table entries (log2 F_j, 1 / F_j) of j = log2_index(x).
__device__ __forceinline__ double log2_finish(double x, double log2f, double invf)
{
    const long long b = __double_as_longlong(x);
    // m - F: the mantissa bits below the index, exactly, as (those bits) * 2^-52.
    const unsigned long long low = static_cast<unsigned long long>(b) &
                                   ((1ull << (52 - kLogBits)) - 1);
    const double r = __dmul_rn(scaled_int(low, 1023), invf);
    double p = __fma_rn(kL2C4, r, kL2C3);
    p = __fma_rn(p, r, kL2C2);
    p = __fma_rn(p, r, kL2C1);
    const int eb = static_cast<int>(b >> 52);
    const double v = __dadd_rn(small_int(eb - 1023), __fma_rn(p, r, log2f));
    return (eb & 0x7FF) == 0x7FF ? CUDART_INF : v;  // +inf, and NaN (as +inf)
}

__device__ __forceinline__ double log2_t(double x, const Tables &t)
{
    const double2 lf = t.lf[log2_index(x)];
    return log2_finish(x, lf.x, lf.y);
}

// log2 with the tables read from global memory (per-query use).
__device__ __forceinline__ double log2_c(double x)
{
    const int j = log2_index(x);
    return log2_finish(x, kLog2F[j], kInvF[j]);
}

__device__ __forceinline__ double exp2_t(double y, const Tables &t)
{
    const long long b = __double_as_longlong(y);
    // y <= -1021 (also -inf): the high word of a negative double grows with its magnitude.
    if (static_cast<uint32_t>(b >> 32) >= 0xC08FE800u)
        return 0.0;
    const int E = static_cast<int>((b >> 52) & 0x7FF);
    if (E >= 1033)
        return CUDART_INF;  // y >= 1024, +inf, NaN
    // 2048 |y| = M 2^-sh with the 53-bit significand M; sh >= 32 here.
    const int sh = 1075 - kExpBits - E;
    long long k = 0;
    double r = y;
    if (sh <= 54) {
        const unsigned long long M =
            (static_cast<unsigned long long>(b) & static_cast<unsigned long long>(kMant)) |
            (1ull << 52);
        const unsigned long long ka = (M + (1ull << (sh - 1))) >> sh;  // round(2048 |y|)
        // |y| - ka/2048 = (M - ka 2^sh) 2^(E - 1075), |M - ka 2^sh| <= 2^(sh - 1) < 2^53.
        const long long rm = static_cast<long long>(M) - static_cast<long long>(ka << sh);
        const bool neg_r = (rm < 0) != (b < 0);
        r = flip_sign(scaled_int(static_cast<unsigned long long>(rm < 0 ? -rm : rm), E), neg_r);
        k = b < 0 ? -static_cast<long long>(ka) : static_cast<long long>(ka);
    }
    // T_j e^(r ln 2) = ((c3 r + c2) r + c1) r + T_j.
    const int j = static_cast<int>(k & (kExpN - 1));
    const double2 a = t.ea[j], c = t.eb[j];
    const double v = __fma_rn(r, __fma_rn(r, __fma_rn(r, c.y, c.x), a.y), a.x);
    return __longlong_as_double(__double_as_longlong(v) + ((k >> kExpBits) << 52));
}

}  // namespace f64math
}  // namespace aidw
