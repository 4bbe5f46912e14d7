"""Writes the constant tables of the table-driven log2 / exp2 of the phase-2 scans: the FP64 ones
(``f64_math_tables.inc``) and the double-float ones of the AIDW_F64X scan (``df_math_tables.inc``),
both beside this script. Run ``python gen_f64_math_tables.py``.

Method (after Tang's table-driven logarithm and exponential):
  log2(x): x = 2^e m, m in [1, 2); F = 1 + j/2048 from the top 11 bits of m; r = (m - F) / F
           in [0, 2^-11); log2(x) = e + log2(F) + log2(1 + r) with the degree-4 Taylor
           polynomial of ln(1 + r) divided by ln 2 (truncation below 2^-56.8).
  exp2(y): k = round(2048 y), r = y - k/2048 in [-2^-12, 2^-12]; 2^y = 2^(k >> 11)
           * T_j e^(r ln 2), T_j = 2^(j/2048), j = k & 2047, with the degree-3 Taylor polynomial
           of e^(r ln 2) multiplied out with T_j: T_j + T_j ln 2 r + T_j (ln 2)^2/2 r^2
           + T_j (ln 2)^3/6 r^3, each coefficient tabulated per j (truncation below 2^-54.7
           relative).
Double-float (a value as the unevaluated sum hi + lo of two floats, about 48 bits):
  log2(x): F = 1 + j/256 from the top 8 bits of the mantissa; u = (m - F) / (F ln 2) by the
           pair (1 / (F ln 2)); log2(1 + r) = u - (ln 2 / 2) u^2 + sum_{i=3..6} c_i u^i with
           |u| < 2^-7.47 (the u^7 term is below 2^-57).
  exp2(y): k = round(128 y), s = y - k/128, t = s ln 2 in [-2^-8.5, 2^-8.5]; 2^y = 2^(k >> 7)
           * 2^((k & 127)/128) * e^t with e^t - 1 = t + t^2/2 + t^3 (1/6 + t/24 + t^2/120)
           (the t^6 term is below 2^-61).
Every value is evaluated with 200-bit arithmetic and rounded to the nearest double (FP64
tables) or split into the nearest float and the nearest float to the remainder (double-float
tables); the files hold them as hexadecimal floating-point literals (exact).
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


def lit(x) -> str:
    return float.hex(dbl(x))


def table(name, values, per_line=3, space="__device__ __constant__"):
    out = [f"{space} double {name}[{len(values)}] = {{"]
    for i in range(0, len(values), per_line):
        out.append("    " + ", ".join(lit(v) for v in values[i:i + per_line]) + ",")
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


def main():
    ln2 = mp.log(2)
    log2_f = [mp.log(1 + mp.mpf(j) / 2048) / ln2 for j in range(2048)]
    inv_f = [1 / (1 + mp.mpf(j) / 2048) for j in range(2048)]
    exp2_j = [mp.power(2, mp.mpf(j) / 2048) for j in range(2048)]
    exp2_c = [[t * ln2 ** i / mp.factorial(i) for t in exp2_j] for i in range(1, 4)]
    ln_coef = [mp.mpf((-1) ** (i + 1)) / i / ln2 for i in range(1, 5)]    # r, r^2 .. r^4
    dev = "__device__ const"  # 96 KB: global memory, copied to shared memory per CTA
    lines = [
        "// Generated by gen_f64_math_tables.py: constants of the table-driven FP64 log2 / exp2",
        "// (values rounded to the nearest double, written as exact hexadecimal literals).",
        table("kLog2F", log2_f, space=dev),
        table("kInvF", inv_f, space=dev),
        table("kExp2J", exp2_j, space=dev),
        "// T_j (ln 2)^i / i!, i = 1, 2, 3: the exp2 polynomial's coefficients for entry j",
        *(table(f"kExp2C{i + 1}", c, space=dev) for i, c in enumerate(exp2_c)),
        "// log2(1 + r) = sum_{i=1..4} kL2C<i> r^i",
        *(f"constexpr double kL2C{i + 1} = {lit(c)};" for i, c in enumerate(ln_coef)),
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
