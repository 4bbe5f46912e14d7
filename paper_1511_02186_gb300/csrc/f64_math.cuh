// Table-driven FP64 log2 and exp2 for the FP64 path's per-pair weights (the method after
// Tang's table-driven logarithm and exponential; the constants and how they were obtained are
// in gen_f64_math_tables.py / f64_math_tables.inc).
//
//   log2(x), x a positive normal double or +inf: x = 2^e (F + u) with F = 1 + j/1024 from the
//     top 10 mantissa bits and u in [0, 2^-10) the rest (both exact); log2(x) = e + (log2 F +
//     u q_j(u)), q_j a cubic per table entry (near-minimax: the polynomial interpolating
//     log2(1 + u/F) / u at the Chebyshev nodes of [0, 2^-10]), evaluated by four fused steps, the
//     last adding log2 F. Absolute error about one ulp of max(1, |log2 x|).
//   exp2(y), y < 1023: y <= -1021 gives 0 (far below any weight that matters next to the nearest
//     point's, which is 1); else k = round(1024 y), r = y - k/1024 in [-2^-11, 2^-11] (exact),
//     2^y = 2^(k >> 10) * T_j 2^r, T_j = 2^(j/1024), j = k & 1023, with T_j 2^r = T_j + r q_j(r)
//     and q_j a quadratic per entry (near-minimax likewise), three fused steps; the power of two
//     is added to the exponent field. Relative error a few ulps.
// GB300 runs FP64 arithmetic at 2 operations per clock per SM against 64 integer operations, so
// every step whose result is exact is done on the integer pipe from the operands' bits: the
// range tests, u, e as a double, and exp2's reduction (k and r). The FP64 pipe runs only the
// rounded operations: 5 for log2 and 3 for exp2, against several times that for the general
// library functions; the weights of Eq. 1 need the absolute accuracy of log2 (it is scaled by
// alpha / 2 and exponentiated), which these keep.
#pragma once

#include <cstdint>

#include <math_constants.h>

#include "aidw_internal.cuh"

namespace aidw {
namespace f64math {

#include "f64_math_tables.inc"

constexpr int kLogBits = 10;                   // log2 table index bits
constexpr int kLogN = 1 << kLogBits;           // 1,024 entries
constexpr int kExpBits = 10;                   // exp2 table: 2^(j / 1024)
constexpr int kExpN = 1 << kExpBits;
constexpr long long kMant = 0x000FFFFFFFFFFFFFLL;

// Shared-memory copy of the tables for one CTA (72 KB: dynamic shared memory).
struct Tables {
    double2 la[kLogN];  // (D4, D3) of q_j
    double2 lb[kLogN];  // (D2, D1)
    double lc[kLogN];   // log2 F_j
    double2 ea[kExpN];  // (E3, E2) of q_j
    double2 eb[kExpN];  // (E1, T_j)
};
constexpr size_t kTablesBytes = sizeof(Tables);

// Every thread of the CTA takes part; the caller synchronises before the first use.
__device__ __forceinline__ void load_tables(Tables &t)
{
    for (int i = threadIdx.x; i < kLogN; i += blockDim.x) {
        t.la[i] = make_double2(kL2D4[i], kL2D3[i]);
        t.lb[i] = make_double2(kL2D2[i], kL2D1[i]);
        t.lc[i] = kLog2F[i];
    }
    for (int i = threadIdx.x; i < kExpN; i += blockDim.x) {
        t.ea[i] = make_double2(kExp2E3[i], kExp2E2[i]);
        t.eb[i] = make_double2(kExp2E1[i], kExp2J[i]);
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

// log2(x) from the table entries of j = log2_index(x): q_j's coefficients and log2 F_j.
__device__ __forceinline__ double log2_finish(double x, double d4, double d3, double d2,
                                              double d1, double log2f)
{
    const long long b = __double_as_longlong(x);
    // u: the mantissa bits below the index, exactly, as (those bits) * 2^-52.
    const unsigned long long low = static_cast<unsigned long long>(b) &
                                   ((1ull << (52 - kLogBits)) - 1);
    const double u = scaled_int(low, 1023);
    double p = __fma_rn(d4, u, d3);
    p = __fma_rn(p, u, d2);
    p = __fma_rn(p, u, d1);
    const int eb = static_cast<int>(b >> 52);
    const double v = __dadd_rn(small_int(eb - 1023), __fma_rn(p, u, log2f));
    return (eb & 0x7FF) == 0x7FF ? CUDART_INF : v;  // +inf, and NaN (as +inf)
}

__device__ __forceinline__ double log2_t(double x, const Tables &t)
{
    const int j = log2_index(x);
    const double2 a = t.la[j], c = t.lb[j];
    return log2_finish(x, a.x, a.y, c.x, c.y, t.lc[j]);
}

// log2 with the tables read from global memory (per-query use).
__device__ __forceinline__ double log2_c(double x)
{
    const int j = log2_index(x);
    return log2_finish(x, kL2D4[j], kL2D3[j], kL2D2[j], kL2D1[j], kLog2F[j]);
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
    // 1024 |y| = M 2^-sh with the 53-bit significand M; sh >= 33 here.
    const int sh = 1075 - kExpBits - E;
    long long k = 0;
    double r = y;
    if (sh <= 54) {
        const unsigned long long M =
            (static_cast<unsigned long long>(b) & static_cast<unsigned long long>(kMant)) |
            (1ull << 52);
        const unsigned long long ka = (M + (1ull << (sh - 1))) >> sh;  // round(1024 |y|)
        // |y| - ka/1024 = (M - ka 2^sh) 2^(E - 1075), |M - ka 2^sh| <= 2^(sh - 1) < 2^53.
        const long long rm = static_cast<long long>(M) - static_cast<long long>(ka << sh);
        const bool neg_r = (rm < 0) != (b < 0);
        r = flip_sign(scaled_int(static_cast<unsigned long long>(rm < 0 ? -rm : rm), E), neg_r);
        k = b < 0 ? -static_cast<long long>(ka) : static_cast<long long>(ka);
    }
    // T_j 2^r = ((E3 r + E2) r + E1) r + T_j.
    const int j = static_cast<int>(k & (kExpN - 1));
    const double2 a = t.ea[j], c = t.eb[j];
    const double v = __fma_rn(r, __fma_rn(r, __fma_rn(a.x, r, a.y), c.x), c.y);
    return __longlong_as_double(__double_as_longlong(v) + ((k >> kExpBits) << 52));
}

}  // namespace f64math
}  // namespace aidw
