"""Writes rich_log_tables.h: the tables of the kernels' FP64 logarithm
(the dispersive radiator's yield integral), of the double-word logarithm
and of log k! (exact to 40 digits with `decimal`, then rounded to FP64, or
split into two FP32 numbers hi + lo). Run from this directory:
python gen_log_tables.py"""
import math
import struct
from decimal import Decimal, getcontext

getcontext().prec = 50
LOG_BITS = 7               # table index: the top 7 mantissa bits
N_LOGFACT = 2048           # log k! for k < 2048


def d(x):
    return float(x).hex()


def split(v):
    hi = float(v)
    lo = float(v - Decimal(hi))
    return hi, lo


def f32(x):
    """x (a Python float) rounded to FP32."""
    return struct.unpack("f", struct.pack("f", x))[0]


def f32_nearest(v):
    """The FP32 number nearest to the Decimal v (the FP64 rounding first can
    land one FP32 step off; its neighbours are checked)."""
    h = f32(float(v))
    cands = [h, f32(math.nextafter(h, math.inf)), f32(math.nextafter(h, -math.inf))]
    # nextafter steps in FP64; step to the FP32 neighbours instead
    up = struct.unpack("f", struct.pack("I", struct.unpack("I", struct.pack("f", h))[0] + 1))[0]
    dn = struct.unpack("f", struct.pack("I", struct.unpack("I", struct.pack("f", h))[0] - 1))[0]
    cands = [h, up, dn] if h > 0 else [h, dn, up]
    return min(cands, key=lambda c: abs(v - Decimal(c)))


def split32(v):
    """v = hi + lo with hi, lo FP32 and |lo| <= ulp(hi) / 2."""
    if v == 0:
        return 0.0, 0.0
    hi = f32_nearest(v)
    lo = f32_nearest(v - Decimal(hi)) if v != Decimal(hi) else 0.0
    return hi, lo


def fx(x):
    return float(x).hex() + "f"


lines = ["// rich_log_tables.h -- generated by gen_log_tables.py; do not edit.",
         "#pragma once", "", "namespace rich {", ""]
n = 1 << LOG_BITS
lines.append(f"// log2 of the table size of the FP64 logarithm")
lines.append(f"constexpr int kLogTableBits = {LOG_BITS};")
lines.append("// per index i: 1/c_i (c_i = 1 + (i + 1/2) / 128, rounded), and -log of")
lines.append("// that stored reciprocal as an unevaluated sum hi + lo")
lines.append(f"__device__ const double g_log_tab[{n}][3] = {{")
for i in range(n):
    c = Decimal(1) + (Decimal(i) + Decimal("0.5")) / n
    inv = float(Decimal(1) / c)
    hi, lo = split(-Decimal(inv).ln())
    lines.append(f"    {{{d(inv)}, {d(hi)}, {d(lo)}}},")
lines.append("};")
lines.append("")
lines.append("// FP32 forms for the double-word logarithm: per index i, F_i = 1/c_i")
lines.append("// rounded to FP32 and -log F_i as hi + lo")
lines.append(f"__device__ const float g_log_tab_f[{n}][3] = {{")
for i in range(n):
    c = Decimal(1) + (Decimal(i) + Decimal("0.5")) / n
    inv = f32_nearest(Decimal(1) / c)
    hi, lo = split32(-Decimal(inv).ln())
    lines.append(f"    {{{fx(inv)}, {fx(hi)}, {fx(lo)}}},")
lines.append("};")
lines.append("")
lines.append(f"constexpr int kLogFactTable = {N_LOGFACT};")
lines.append("// log k! for k < kLogFactTable as a double-word (hi, lo)")
lines.append(f"__device__ const float g_logfact_ff[{N_LOGFACT}][2] = {{")
acc = Decimal(0)
for k in range(N_LOGFACT):
    if k > 1:
        acc += Decimal(k).ln()
    hi, lo = split32(acc)
    lines.append(f"    {{{fx(hi)}, {fx(lo)}}},")
lines.append("};")
lines.append("")
lines.append("}  // namespace rich")
open("rich_log_tables.h", "w").write("\n".join(lines) + "\n")
