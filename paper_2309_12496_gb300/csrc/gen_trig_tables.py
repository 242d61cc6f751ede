"""Writes rich_trig_tables.h: sin and cos of 2 pi j / 256 (j = 0..255) and
the constants of the double-word sine/cosine of the refinement pass, each
as an unevaluated sum of two FP32 numbers (hi + lo), from 50-digit values
(Taylor series of sin and cos in `decimal`). Run from this directory:
python gen_trig_tables.py"""
from decimal import Decimal, getcontext

getcontext().prec = 60
N = 256


def pi():
    # Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(x):
        x = Decimal(x)
        s, t, k, x2 = Decimal(0), 1 / x, 0, x * x
        while abs(t) > Decimal(10) ** -58:
            s += t / (2 * k + 1) * (1 if k % 2 == 0 else -1)
            t /= x2
            k += 1
        return s
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def sin_cos(a):
    s, c, term, k = Decimal(0), Decimal(0), Decimal(1), 0
    # term = a^k / k!
    while abs(term) > Decimal(10) ** -58 or k < 4:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
    return s, c


def f32(x):
    import struct
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def split(v):
    hi = f32(v)
    lo = f32(v - Decimal(repr(hi)))
    return hi, lo


def h(x):
    return float(x).hex() + "f"


P = pi()
lines = ["// rich_trig_tables.h -- generated by gen_trig_tables.py; do not edit.",
         "#pragma once", "", "namespace rich {", "",
         "// (sin hi, sin lo, cos hi, cos lo) of 2 pi j / 256, j = 0..255",
         f"__device__ const float g_sincos_tab[{N}][4] = {{"]
for j in range(N):
    s, c = sin_cos(2 * P * j / N)
    sh, sl = split(s)
    ch, cl = split(c)
    lines.append(f"    {{{h(sh)}, {h(sl)}, {h(ch)}, {h(cl)}}},")
lines.append("};")
th, tl = split(2 * P / Decimal(2) ** 24)
s6h, s6l = split(Decimal(1) / 6)
lines += ["", "// 2 pi / 2^24 and 1/6 as hi + lo",
          f"constexpr float kTwoPi24Hi = {h(th)}, kTwoPi24Lo = {h(tl)};",
          f"constexpr float kSixthHi = {h(s6h)}, kSixthLo = {h(s6l)};",
          "", "}  // namespace rich"]
open("rich_trig_tables.h", "w").write("\n".join(lines) + "\n")
