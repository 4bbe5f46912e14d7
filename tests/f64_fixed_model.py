"""A bit-exact Python model of the FP64 path's fixed-point log2 / exp2 (the integer steps that
csrc/f64_math.cuh runs on the GPU, with every 64-bit wrap and shift written out), reading the
same tables from csrc/f64_math_tables.inc. It is test infrastructure: the CPU tests check the
model's accuracy against 120-bit references (so the integer algorithm itself is pinned), and a
GPU test checks that the library's kernels give the model's doubles bit for bit."""
from __future__ import annotations

import os
import re
import struct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_1511_02186_gb300", "csrc", "f64_math_tables.inc")
M64 = (1 << 64) - 1
MANT = (1 << 52) - 1


def load_tables(path: str = TABLES) -> dict:
    """name -> list of int (the fixed-point tables at 2^62)."""
    text = open(path).read()
    out = {}
    for m in re.finditer(r"__device__ const long long (\w+)\[(\d+)\] = \{(.*?)\};", text, re.S):
        vals = [int(t.strip().rstrip("L"), 16) for t in m.group(3).split(",") if t.strip()]
        assert len(vals) == int(m.group(2)), m.group(1)
        out[m.group(1)] = vals
    return out


def bits(x: float) -> int:
    """The double's bits as a signed 64-bit integer."""
    return struct.unpack("<q", struct.pack("<d", x))[0]


def from_bits(b: int) -> float:
    b &= M64
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def s64(v: int) -> int:
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def clz64(v: int) -> int:
    return 64 - (v & M64).bit_length()


def fx_mul(p: int, v: int) -> int:
    """High word of the unsigned 64 x 64-bit product, shifted right by 9."""
    return ((p * v) >> 64) >> 9


def fx_mul32(p: int, v: int) -> int:
    """The same from the operands' high 32-bit words."""
    return (((p >> 32) & 0xFFFFFFFF) * ((v >> 32) & 0xFFFFFFFF)) >> 9


def fx52_to_double(a: int) -> float:
    """The double nearest to a * 2^-52 (ties away from zero), as the integer steps do it."""
    s = (a & M64) & (1 << 63)
    m = (-a if a < 0 else a) & M64
    lz = clz64(m | 1)
    mn = (m << lz) & M64
    sig = (mn >> 11) + ((mn >> 10) & 1)
    b = (((1034 - lz) << 52) + sig - (1 << 52)) & M64
    return 0.0 if m == 0 else from_bits(b | s)


def log2_fx(x: float, t: dict) -> float:
    b = bits(x)
    j = (b >> 42) & 1023
    u = ((b & ((1 << 42) - 1)) << 21) & M64
    p = (t["kFxL2A3"][j] - fx_mul32(t["kFxL2A4"][j], u)) & M64
    p = (t["kFxL2A2"][j] - fx_mul32(p, u)) & M64
    p = (t["kFxL2A1"][j] - fx_mul(p, u)) & M64
    f = (t["kFxLog2F"][j] + fx_mul(p, u)) & M64
    eb = b >> 52
    v = s64((eb - 1023) * (1 << 52) + ((f + (1 << 9)) >> 10))
    return float("inf") if (eb & 0x7FF) == 0x7FF else fx52_to_double(v)


def exp2_fx(y: float, t: dict):
    """(2^y as a double, 2^y as an integer with 96 fraction bits or None)."""
    b = bits(y)
    if ((b >> 32) & 0xFFFFFFFF) >= 0xC08FE800:
        return 0.0, 0
    E = (b >> 52) & 0x7FF
    if E >= 1033:
        return float("inf"), 0
    M = (b & MANT) | ((1 << 52) if E != 0 else 0)
    sh = 1065 - E
    k = 0
    if sh <= 54:
        ka = (M + (1 << (sh - 1))) >> sh
        rm = s64(M - ((ka << sh) & M64))
        r = s64((rm & M64) << (E - 1002))
        k = ka
    else:
        s = E - 1002
        r = s64((M << s) if s >= 0 else ((M >> -s) if -s < 64 else 0))
    if b < 0:
        r, k = -r, -k
    j = k & 1023
    kk = k >> 10
    rn = r < 0
    ra = (-r if rn else r) & M64
    e1, e2, e3, tj = (t["kFxExp2E1"][j], t["kFxExp2E2"][j], t["kFxExp2E3"][j],
                      t["kFxExp2T"][j])
    q = fx_mul32(e3, ra)
    p = (e2 - q if rn else e2 + q) & M64
    q = fx_mul(p, ra)
    p = (e1 - q if rn else e1 + q) & M64
    q = fx_mul(p, ra)
    uv = (tj - q if rn else tj + q) & M64
    sft = 34 + kk
    w96 = (uv << min(sft, 127)) & ((1 << 128) - 1) if sft >= 0 else (
        (uv >> -sft) if -sft < 127 else 0)
    lz = clz64(uv)
    sig = (((uv << (lz - 1)) & M64) + (1 << 9)) >> 10
    eb = 1024 - lz + kk
    return from_bits(((eb << 52) + sig - (1 << 52)) & M64), w96
