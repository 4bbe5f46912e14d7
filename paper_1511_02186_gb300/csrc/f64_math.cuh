// Table-driven log2 and exp2 for the FP64 path's per-pair weights (the method after Tang's
// table-driven logarithm and exponential; the constants and how they were obtained are in
// gen_f64_math_tables.py / f64_math_tables.inc), evaluated in fixed point on the integer pipe.
//
//   log2(x), x a positive normal double or +inf: x = 2^e (F + u) with F = 1 + j/1024 from the
//     top 10 mantissa bits and u in [0, 2^-10) the rest (both exact); log2(x) = e + (log2 F +
//     u q_j(u)), q_j a cubic per table entry (near-minimax: the polynomial interpolating
//     log2(1 + u/F) / u at the Chebyshev nodes of [0, 2^-10]). The fraction log2 F + u q_j(u)
//     is formed in 64-bit fixed point with 62 fraction bits, e added exactly at 52 fraction
//     bits, and the sum rounded once to a double: absolute error within 0.75 ulp of
//     max(1, |log2 x|).
//   exp2(y), y < 1023: y <= -1021 gives 0 (far below any weight that matters next to the nearest
//     point's, which is 1); else k = round(1024 y), r = y - k/1024 in [-2^-11, 2^-11] (exact,
//     from the significand's bits), 2^y = 2^(k >> 10) T_j 2^r, T_j = 2^(j/1024), j = k & 1023,
//     T_j 2^r = T_j + r q_j(r) with q_j a quadratic per entry (near-minimax likewise), in the
//     same fixed point; the result is rounded once to a double (relative error about an ulp)
//     and, for the scan's sum of the weights, also given as an integer with 96 fraction bits.
// GB300 runs FP64 arithmetic at 2 operations per clock per SM against 64 integer operations, so
// both functions run on the integer pipe, in unsigned fixed point: every coefficient is kept as a
// magnitude at 2^62 and every variable as a magnitude at 2^73, so a product's high word lands at
// 2^71 and a shift brings it back to 2^62; the signs are known (log2's coefficients alternate,
// exp2's are positive and only r has a sign) and become subtractions. The innermost Horner steps
// need fewer bits (their terms are scaled by further powers of u or r, at most 2^-10 each) and
// take one 32 x 32-bit product on the operands' high words; the outer steps take the high word of
// a full 64 x 64-bit product. Every step truncates far below a double's rounding; the
// polynomials' own error (below 2^-58.5 for log2, at most 2^-52.7 relative for exp2) and the
// final rounding to a double set the accuracy.
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
    ulonglong2 la[kLogN];        // (A4, A3) of q_j (magnitudes)
    ulonglong2 lb[kLogN];        // (A2, A1)
    unsigned long long lc[kLogN];  // log2 F_j
    ulonglong2 ea[kExpN];        // (E3, E2) of q_j
    ulonglong2 eb[kExpN];        // (E1, T_j)
};
constexpr size_t kTablesBytes = sizeof(Tables);

__device__ __forceinline__ unsigned long long tab(long long v)
{
    return static_cast<unsigned long long>(v);
}

// Every thread of the CTA takes part; the caller synchronises before the first use.
__device__ __forceinline__ void load_tables(Tables &t)
{
    for (int i = threadIdx.x; i < kLogN; i += blockDim.x) {
        t.la[i] = make_ulonglong2(tab(kFxL2A4[i]), tab(kFxL2A3[i]));
        t.lb[i] = make_ulonglong2(tab(kFxL2A2[i]), tab(kFxL2A1[i]));
        t.lc[i] = tab(kFxLog2F[i]);
    }
    for (int i = threadIdx.x; i < kExpN; i += blockDim.x) {
        t.ea[i] = make_ulonglong2(tab(kFxExp2E3[i]), tab(kFxExp2E2[i]));
        t.eb[i] = make_ulonglong2(tab(kFxExp2E1[i]), tab(kFxExp2T[i]));
    }
}

__device__ __forceinline__ int log2_index(double x)
{
    return static_cast<int>((__double_as_longlong(x) >> (52 - kLogBits)) & (kLogN - 1));
}

// p v at 2^62 for p at 2^62 and v at 2^73 (both below 2^63): the high word of the full product.
__device__ __forceinline__ unsigned long long fx_mul(unsigned long long p, unsigned long long v)
{
    return __umul64hi(p, v) >> 9;
}

// The same from the operands' high words (32 x 32 bits; truncation about 2^-30 relative).
__device__ __forceinline__ unsigned long long fx_mul32(unsigned long long p, unsigned long long v)
{
    return (static_cast<unsigned long long>(static_cast<uint32_t>(p >> 32)) *
            static_cast<uint32_t>(v >> 32)) >> 9;
}

// The double nearest to a * 2^-52 for |a| < 2^63 (ties away from zero), integer steps only.
__device__ __forceinline__ double fx52_to_double(long long a)
{
    const unsigned long long s = static_cast<unsigned long long>(a) & (1ull << 63);
    const unsigned long long m = static_cast<unsigned long long>(a < 0 ? -a : a);
    const int lz = __clzll(static_cast<long long>(m | 1));  // >= 1 (m == 0 gives 0.0 below)
    // The 53-bit significand, rounded (the bit below it added after the shift, so that nothing
    // overflows); a carry into bit 53 moves into the exponent field.
    const unsigned long long mn = m << lz;
    const unsigned long long sig = (mn >> 11) + ((mn >> 10) & 1ull);
    const unsigned long long b =
        (static_cast<unsigned long long>(1034 - lz) << 52) + sig - (1ull << 52);
    return m == 0 ? 0.0 : __longlong_as_double(static_cast<long long>(b | s));
}

// log2(x) from the table entries of j = log2_index(x): q_j's coefficient magnitudes and
// log2 F_j, all at 2^62. Horner in magnitudes: q(u) = A1 - u (A2 - u (A3 - u A4)), every
// bracket positive.
__device__ __forceinline__ double log2_finish(double x, unsigned long long a4,
                                              unsigned long long a3, unsigned long long a2,
                                              unsigned long long a1, unsigned long long log2f)
{
    const long long b = __double_as_longlong(x);
    // u: the mantissa bits below the index, exactly, at 2^73 (u 2^73 < 2^63).
    const unsigned long long u =
        static_cast<unsigned long long>(b & ((1ll << (52 - kLogBits)) - 1)) << 21;
    unsigned long long p = a3 - fx_mul32(a4, u);  // its error is scaled by u^3 below
    p = a2 - fx_mul32(p, u);                       // ... by u^2
    p = a1 - fx_mul(p, u);
    const unsigned long long f = log2f + fx_mul(p, u);  // log2 F + u q(u) in [0, 1), at 2^62
    const int eb = static_cast<int>(b >> 52);
    // e + f at 2^52 (|e| <= 1074: below 2^63), f rounded to 2^-53.
    const long long v = static_cast<long long>(eb - 1023) * (1ll << 52) +
                        static_cast<long long>((f + (1ull << 9)) >> 10);
    return (eb & 0x7FF) == 0x7FF ? CUDART_INF : fx52_to_double(v);  // +inf, and NaN (as +inf)
}

__device__ __forceinline__ double log2_t(double x, const Tables &t)
{
    const int j = log2_index(x);
    const ulonglong2 a = t.la[j], c = t.lb[j];
    return log2_finish(x, a.x, a.y, c.x, c.y, t.lc[j]);
}

// log2 with the tables read from global memory (per-query use): the same arithmetic, so the same
// double as log2_t for every x.
__device__ __forceinline__ double log2_c(double x)
{
    const int j = log2_index(x);
    return log2_finish(x, tab(kFxL2A4[j]), tab(kFxL2A3[j]), tab(kFxL2A2[j]), tab(kFxL2A1[j]),
                       tab(kFxLog2F[j]));
}

// 2^y as a double; with W96, *w96 = 2^y in fixed point with 96 fraction bits (truncated; 0 when
// 2^y < 2^-96; meaningful for y < 32).
template <bool W96>
__device__ __forceinline__ double exp2_t(double y, const Tables &t, unsigned __int128 *w96)
{
    const long long b = __double_as_longlong(y);
    // y <= -1021 (also -inf): the high word of a negative double grows with its magnitude.
    if (static_cast<uint32_t>(b >> 32) >= 0xC08FE800u) {
        if (W96)
            *w96 = 0;
        return 0.0;
    }
    const int E = static_cast<int>((b >> 52) & 0x7FF);
    if (E >= 1033) {
        if (W96)
            *w96 = 0;
        return CUDART_INF;  // y >= 1024, +inf, NaN
    }
    const unsigned long long M =
        (static_cast<unsigned long long>(b) & static_cast<unsigned long long>(kMant)) |
        (E != 0 ? (1ull << 52) : 0ull);
    // 1024 |y| = M 2^-sh with the 53-bit significand M.
    const int sh = 1075 - kExpBits - E;
    long long k = 0;
    long long r;  // |y| - |k|/1024 at 2^73, |r| <= 2^62
    if (sh <= 54) {  // E >= 1011
        const unsigned long long ka = (M + (1ull << (sh - 1))) >> sh;  // round(1024 |y|)
        // |y| - ka/1024 = (M - ka 2^sh) 2^(E - 1075), |M - ka 2^sh| <= 2^(sh - 1); at 2^73 that
        // is the difference shifted left by E - 1002 >= 9.
        const long long rm = static_cast<long long>(M) - static_cast<long long>(ka << sh);
        r = static_cast<long long>(static_cast<unsigned long long>(rm) << (E - 1002));
        k = static_cast<long long>(ka);
    } else {  // |y| < 2^-11: k = 0, r = |y|
        const int s = E - 1002;
        r = static_cast<long long>(s >= 0 ? (M << s) : (-s < 64 ? (M >> -s) : 0ull));
    }
    if (b < 0) {
        r = -r;
        k = -k;
    }
    const int j = static_cast<int>(k & (kExpN - 1));
    const long long kk = k >> kExpBits;  // the power of two, floor(k / 1024)
    const ulonglong2 a = t.ea[j], c = t.eb[j];
    // T_j 2^r = T_j + r (E1 + r (E2 + r E3)) at 2^62, in (2^61.99, 2^63): in magnitudes, each
    // product added or subtracted by the sign of r.
    const bool rn = r < 0;
    const unsigned long long ra = static_cast<unsigned long long>(rn ? -r : r);
    unsigned long long q = fx_mul32(a.x, ra);  // its error is scaled by r^2 below
    unsigned long long p = rn ? a.y - q : a.y + q;
    q = fx_mul(p, ra);
    p = rn ? c.x - q : c.x + q;
    q = fx_mul(p, ra);
    const unsigned long long uv = rn ? c.y - q : c.y + q;
    const long long v = static_cast<long long>(uv);
    if (W96) {
        // v 2^(kk - 62) 2^96 = v 2^(34 + kk).
        const long long sft = 34 + kk;
        const unsigned __int128 w = uv;
        *w96 = sft >= 0 ? (w << (sft < 127 ? sft : 127)) : (-sft < 127 ? (w >> -sft) : 0);
    }
    // The double: v has its leading one at bit 62 (lz = 1) or 61 (lz = 2).
    const int lz = __clzll(v);
    const unsigned long long sig = ((uv << (lz - 1)) + (1ull << 9)) >> 10;  // 53 bits, rounded
    const unsigned long long eb = static_cast<unsigned long long>(1024 - lz + kk);
    return __longlong_as_double(static_cast<long long>((eb << 52) + sig - (1ull << 52)));
}

}  // namespace f64math
}  // namespace aidw
