"""Writes the constant tables of the table-driven FP64 log2 / exp2 used by the FP64 phase-2 scan
(``f64_math_tables.inc`` beside this script). Run ``python gen_f64_math_tables.py``.

Method (after Tang's table-driven logarithm and exponential):
  log2(x): x = 2^e m, m in [1, 2); F = 1 + j/128 from the top 7 bits of m; r = (m - F) / F in
           [0, 1/128); log2(x) = e + log2(F) + ln(1 + r) / ln 2 with a degree-7 Taylor
           polynomial for ln(1 + r) (truncation below 2^-59).
  exp2(y): k = round(64 y), r = y - k/64 in [-1/128, 1/128]; 2^y = 2^(k >> 6) * 2^((k & 63)/64)
           * e^(r ln 2) with a degree-5 Taylor polynomial (truncation below 4e-17 relative).
Every value is evaluated with 200-bit arithmetic and rounded to the nearest double; the file
holds them as hexadecimal floating-point literals (exact).
"""
import os

import mpmath as mp
from mpmath import libmp

mp.mp.prec = 200
HERE = os.path.dirname(os.path.abspath(__file__))


def dbl(x) -> float:
    """Nearest double to the mpf x."""
    return libmp.to_float(mp.mpf(x)._mpf_, rnd=libmp.round_nearest)


def lit(x) -> str:
    return float.hex(dbl(x))


def table(name, values, per_line=3):
    out = [f"__device__ __constant__ double {name}[{len(values)}] = {{"]
    for i in range(0, len(values), per_line):
        out.append("    " + ", ".join(lit(v) for v in values[i:i + per_line]) + ",")
    out.append("};")
    return "\n".join(out)


def main():
    ln2 = mp.log(2)
    log2_f = [mp.log(1 + mp.mpf(j) / 128) / ln2 for j in range(128)]
    inv_f = [1 / (1 + mp.mpf(j) / 128) for j in range(128)]
    exp2_j = [mp.power(2, mp.mpf(j) / 64) for j in range(64)]
    ln_coef = [mp.mpf((-1) ** (i + 1)) / i for i in range(1, 8)]          # r, r^2 .. r^7
    exp_coef = [ln2 ** i / mp.factorial(i) for i in range(0, 6)]          # 1, r ln2 .. r^5
    lines = [
        "// Generated by gen_f64_math_tables.py: constants of the table-driven FP64 log2 / exp2",
        "// (values rounded to the nearest double, written as exact hexadecimal literals).",
        table("kLog2F", log2_f),
        table("kInvF", inv_f),
        table("kExp2J", exp2_j),
        "// ln(1 + r) = sum_{i=1..7} kLnC<i> r^i",
        *(f"constexpr double kLnC{i + 1} = {lit(c)};" for i, c in enumerate(ln_coef)),
        "// e^(r ln 2) = sum_{i=0..5} kExpC<i> r^i",
        *(f"constexpr double kExpC{i} = {lit(c)};" for i, c in enumerate(exp_coef)),
        "constexpr double kInvLn2 = " + lit(1 / ln2) + ";",
        "",
    ]
    path = os.path.join(HERE, "f64_math_tables.inc")
    with open(path, "w") as f:
        f.write("\n".join(lines))
    print(path)


if __name__ == "__main__":
    main()
