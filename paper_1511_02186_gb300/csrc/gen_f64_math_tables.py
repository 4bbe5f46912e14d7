"""Writes the constant tables of the table-driven log2 / exp2 of the phase-2 scans: the FP64 path's
(``f64_math_tables.inc``) and the double-float ones of the AIDW_F64X scan (``df_math_tables.inc``),
both beside this script. Run ``python gen_f64_math_tables.py``.

Method (after Tang's table-driven logarithm and exponential):
  log2(x): x = 2^e (F + u), F = 1 + j/1024 from the top 10 bits of the mantissa, u in
           [0, 2^-10) the rest (exact); log2(x) = e + log2(F) + u q_j(u) with a cubic q_j per
           entry, the polynomial interpolating log2(1 + u/F) / u at the Chebyshev nodes of
           [0, 2^-10] (near-minimax; the error of u q_j(u) is below 2^-58.5).
  exp2(y): k = round(1024 y), r = y - k/1024 in [-2^-11, 2^-11]; 2^y = 2^(k >> 10)
           * T_j 2^r, T_j = 2^(j/1024), j = k & 1023, with T_j 2^r = T_j + r q_j(r) and q_j the
           quadratic interpolating T_j (2^r - 1) / r at the Chebyshev nodes of [-2^-11, 2^-11]
           (relative error at most 2^-52.7).
The FP64 path evaluates both in unsigned fixed point on the integer pipe, so its tables hold
every value as the nearest integer to value * 2^62 (all values are below 2), q_j's coefficients
of log2 as magnitudes (their signs alternate, the same for every entry: +, -, +, -), those of
exp2 as they are (all positive).
Double-float (a value as the unevaluated sum hi + lo of two floats, about 48 bits):
  log2(x): F = 1 + j/256 from the top 8 bits of the mantissa; u = (m - F) / (F ln 2) by the
           pair (1 / (F ln 2)); log2(1 + r) = u - (ln 2 / 2) u^2 + sum_{i=3..6} c_i u^i with
           |u| < 2^-7.47 (the u^7 term is below 2^-57).
  exp2(y): k = round(128 y), s = y - k/128, t = s ln 2 in [-2^-8.5, 2^-8.5]; 2^y = 2^(k >> 7)
           * 2^((k & 127)/128) * e^t with e^t - 1 = t + t^2/2 + t^3 (1/6 + t/24 + t^2/120)
           (the t^6 term is below 2^-61).
Every value is evaluated with 200-bit arithmetic and rounded to the nearest integer multiple of
2^-62 (FP64 path's tables, written as hexadecimal integer literals) or split into the nearest
float and the nearest float to the remainder (double-float tables, written as exact hexadecimal
floating-point literals).
"""
import os

import mpmath as mp
import numpy as np
from mpmath import libmp

mp.mp.prec = 200
HERE = os.path.dirname(os.path.abspath(__file__))


def dbl(x) -> float:
    """Nearest double to the mpf x."""
    return libmp.to_float(mp.mpf(x)._mpf_, rnd=libmp.round_nearest)


FX_BITS = 62  # fixed-point tables: value * 2^62


def fx(x) -> int:
    """Nearest integer to the mpf x * 2^62."""
    return int(mp.nint(mp.mpf(x) * mp.mpf(2) ** FX_BITS))


def ilit(v: int) -> str:
    return ("-" if v < 0 else "") + f"0x{abs(v):016x}LL"


def fx_table(name, values, per_line=3, space="__device__ const"):
    out = [f"{space} long long {name}[{len(values)}] = {{"]
    for i in range(0, len(values), per_line):
        out.append("    " + ", ".join(ilit(fx(v)) for v in values[i:i + per_line]) + ",")
    out.append("};")
    return "\n".join(out)


def flt(x) -> float:
    """Nearest float to the mpf x (through the nearest double; the lo part absorbs any
    double-rounding difference)."""
    return float(np.float32(dbl(x)))


def split(x):
    """(hi, lo) floats with hi + lo = x to about 2^-48 relative."""
    h = flt(x)
    return h, flt(mp.mpf(x) - mp.mpf(h))


def flit(x: float) -> str:
    return float.hex(x) + "f"


def df_table(name, pairs, per_line=2):
    out = [f"__device__ __constant__ float {name}[{2 * len(pairs)}] = {{"]
    for i in range(0, len(pairs), per_line):
        out.append("    " + ", ".join(f"{flit(h)}, {flit(l)}" for h, l in pairs[i:i + per_line])
                   + ",")
    out.append("};")
    return "\n".join(out)


def df_tables(ln2):
    g = [split(1 / ((1 + mp.mpf(j) / 256) * ln2)) for j in range(256)]
    l2f = [split(mp.log(1 + mp.mpf(j) / 256) / ln2) for j in range(256)]
    t = [split(mp.power(2, mp.mpf(k) / 128)) for k in range(128)]
    # log2(1 + u ln 2) = sum_i (-1)^(i+1) (ln 2)^(i-1) / i * u^i
    c = {i: (-1) ** (i + 1) * ln2 ** (i - 1) / i for i in range(2, 7)}
    c2h, c2l = split(-c[2])
    l2h, l2l = split(ln2)
    lines = [
        "// Generated by gen_f64_math_tables.py: double-float (hi, lo float pairs) constants of",
        "// the AIDW_F64X phase-2 scan, as exact hexadecimal literals.",
        "// 1 / (F_j ln 2), F_j = 1 + j/256",
        df_table("kDfInvFLn2", g),
        "// log2(F_j)",
        df_table("kDfLog2F", l2f),
        "// 2^(k/128)",
        df_table("kDfExp2K", t),
        "// log2(1 + r) with u = r / ln 2: u + kDfC2 u^2 + kDfC3 u^3 + ... + kDfC6 u^6",
        f"constexpr float kDfC2h = {flit(-c2h)};",
        f"constexpr float kDfC2l = {flit(-c2l)};",
        *(f"constexpr float kDfC{i} = {flit(flt(c[i]))};" for i in range(3, 7)),
        "// ln 2 as a pair",
        f"constexpr float kDfLn2h = {flit(l2h)};",
        f"constexpr float kDfLn2l = {flit(l2l)};",
        "",
    ]
    return "\n".join(lines)


def cheb_fit(g, a, b, deg):
    """Coefficients c_0..c_deg of the polynomial interpolating g at the deg + 1 Chebyshev nodes
    of [a, b] (near the minimax polynomial of that degree), at the working precision."""
    n = deg + 1
    xs = [(a + b) / 2 - (b - a) / 2 * mp.cos((2 * i + 1) * mp.pi / (2 * n)) for i in range(n)]
    A = mp.matrix([[x ** k for k in range(n)] for x in xs])
    c = mp.lu_solve(A, mp.matrix([g(x) for x in xs]))
    return [c[k] for k in range(n)]


def main():
    ln2 = mp.log(2)
    dev = "__device__ const"  # 72 KB: global memory, copied to shared memory per CTA
    # log2: x = 2^e (F_j + u), F_j = 1 + j/1024, u in [0, 2^-10) exact; log2(1 + u/F_j) = u q_j(u)
    # with q_j the cubic through g(u) = log2(1 + u/F_j) / u (g(0) = 1 / (F_j ln 2)) at the
    # Chebyshev nodes of [0, 2^-10].
    h = mp.mpf(2) ** -10
    log2_f, l2d = [], [[], [], [], []]
    for j in range(1024):
        F = 1 + mp.mpf(j) / 1024
        log2_f.append(mp.log(F) / ln2)
        c = cheb_fit(lambda u: mp.log1p(u / F) / (u * ln2), 0, h, 3)
        for i in range(4):
            l2d[i].append(c[i])
    # exp2: y = k/1024 + r, r in [-2^-11, 2^-11]; T_j 2^r = T_j + r q_j(r), T_j = 2^(j/1024),
    # q_j the quadratic through T_j (2^r - 1) / r (T_j ln 2 at 0) at the Chebyshev nodes.
    he = mp.mpf(2) ** -11
    exp2_j, e2e = [], [[], [], []]
    for j in range(1024):
        T = mp.power(2, mp.mpf(j) / 1024)
        exp2_j.append(T)
        c = cheb_fit(lambda r: T * ln2 if r == 0 else T * mp.expm1(r * ln2) / r, -he, he, 2)
        for i in range(3):
            e2e[i].append(c[i])
    lines = [
        "// Generated by gen_f64_math_tables.py: constants of the FP64 path's table-driven log2 /",
        "// exp2, in fixed point: every entry the nearest integer to value * 2^62.",
        "// log2 F_j, F_j = 1 + j/1024",
        fx_table("kFxLog2F", log2_f, space=dev),
        "// log2(1 + u/F_j) = u (kFxL2A1 - kFxL2A2 u + kFxL2A3 u^2 - kFxL2A4 u^3)[j] 2^-62,",
        "// u in [0, 2^-10)",
        *(fx_table(f"kFxL2A{i + 1}", [(-1) ** i * c for c in l2d[i]], space=dev)
          for i in range(4)),
        "// T_j = 2^(j/1024)",
        fx_table("kFxExp2T", exp2_j, space=dev),
        "// T_j 2^r = (kFxExp2T + r (kFxExp2E1 + kFxExp2E2 r + kFxExp2E3 r^2))[j] 2^-62,",
        "// r in [-2^-11, 2^-11]",
        *(fx_table(f"kFxExp2E{i + 1}", e2e[i], space=dev) for i in range(3)),
        "",
    ]
    path = os.path.join(HERE, "f64_math_tables.inc")
    with open(path, "w") as f:
        f.write("\n".join(lines))
    print(path)
    path = os.path.join(HERE, "df_math_tables.inc")
    with open(path, "w") as f:
        f.write(df_tables(ln2))
    print(path)


if __name__ == "__main__":
    main()
