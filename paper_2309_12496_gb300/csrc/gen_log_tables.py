"""Writes rich_log_tables.h: the tables of the yield kernel's FP64
logarithm and of log k! (exact to 40 digits with `decimal`, then rounded
to FP64). Run from this directory: python gen_log_tables.py"""
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
lines.append(f"constexpr int kLogFactTable = {N_LOGFACT};")
lines.append("// log k! for k < kLogFactTable")
lines.append(f"__device__ const double g_logfact[{N_LOGFACT}] = {{")
acc = Decimal(0)
vals = []
for k in range(N_LOGFACT):
    if k > 1:
        acc += Decimal(k).ln()
    vals.append(d(float(acc)))
for i in range(0, N_LOGFACT, 4):
    lines.append("    " + ", ".join(vals[i:i + 4]) + ",")
lines.append("};")
lines.append("")
lines.append("}  // namespace rich")
open("rich_log_tables.h", "w").write("\n".join(lines) + "\n")
