"""The generated constant tables of the kernels (csrc/rich_log_tables.h,
csrc/rich_trig_tables.h), read as text and checked against 50-digit values
from mpmath; and the table-driven logarithm's decomposition (the steps of
ff_log: exponent, interval index, r = m F - 1, the series) evaluated on
the host with these tables against math.log. CPU only."""
import math
import os
import re
import struct

import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2309_12496_gb300", "csrc")


def _array(src, name):
    """The numbers of `name`'s initialiser, as floats, row by row."""
    start = src.index(name)
    body = src[src.index("{", start) + 1:src.index("};", start)]
    rows = re.findall(r"\{([^{}]*)\}", body)
    if not rows:                    # flat array
        rows = [body]
    return [[float.fromhex(v.strip().rstrip("f")) for v in r.split(",") if v.strip()]
            for r in rows]


def _f32(x):
    return struct.unpack("f", struct.pack("f", x))[0]


def _ulp32(x):
    return math.ulp(_f32(x)) * 2.0 ** 29   # FP32 ulp from the FP64 ulp


LOG = open(os.path.join(CSRC, "rich_log_tables.h")).read()
TRIG = open(os.path.join(CSRC, "rich_trig_tables.h")).read()


def test_fp64_log_table():
    tab = _array(LOG, "g_log_tab[")
    assert len(tab) == 128
    for i, (inv_c, hi, lo) in enumerate(tab):
        c = 1 + (mp.mpf(i) + mp.mpf("0.5")) / 128
        assert abs(mp.mpf(inv_c) * c - 1) < mp.mpf(2) ** -52
        assert abs(mp.mpf(hi) + mp.mpf(lo) + mp.log(mp.mpf(inv_c))) < mp.mpf(2) ** -100


def test_fp32_log_table_is_an_exact_split():
    tab = _array(LOG, "g_log_tab_f[")
    assert len(tab) == 128
    for i, (F, hi, lo) in enumerate(tab):
        assert _f32(F) == F and _f32(hi) == hi and _f32(lo) == lo
        c = 1 + (mp.mpf(i) + mp.mpf("0.5")) / 128
        assert abs(mp.mpf(F) * c - 1) <= mp.mpf(2) ** -24
        exact = -mp.log(mp.mpf(F))
        # hi + lo is the double-word nearest -log F: |error| << ulp(lo)
        assert abs(mp.mpf(hi) + mp.mpf(lo) - exact) <= mp.mpf(2) ** -49 * max(abs(exact), 2 ** -8)
        if hi != 0.0:
            assert abs(lo) <= _ulp32(hi) / 2


def test_log_factorial_table():
    tff = _array(LOG, "g_logfact_ff[")
    assert len(tff) == 2048
    for k in list(range(0, 64)) + list(range(64, 2048, 37)) + [2047]:
        exact = mp.loggamma(k + 1)
        hi, lo = tff[k]
        assert abs(mp.mpf(hi) + mp.mpf(lo) - exact) <= mp.mpf(2) ** -47 * max(abs(exact), 1)
        if hi != 0.0:
            assert abs(lo) <= _ulp32(hi) / 2


def test_sincos_table_and_constants():
    tab = _array(TRIG, "g_sincos_tab[")
    assert len(tab) == 256
    for j, (sh, sl, ch, cl) in enumerate(tab):
        a = 2 * mp.pi * j / 256
        assert abs(mp.mpf(sh) + mp.mpf(sl) - mp.sin(a)) <= mp.mpf(2) ** -48
        assert abs(mp.mpf(ch) + mp.mpf(cl) - mp.cos(a)) <= mp.mpf(2) ** -48
    consts = dict(re.findall(r"(k\w+) = ([-0-9a-fx.p+]+)f", TRIG))
    two_pi_24 = mp.mpf(float.fromhex(consts["kTwoPi24Hi"])) + mp.mpf(float.fromhex(consts["kTwoPi24Lo"]))
    assert abs(two_pi_24 / (2 * mp.pi / 2 ** 24) - 1) < mp.mpf(2) ** -46
    sixth = mp.mpf(float.fromhex(consts["kSixthHi"])) + mp.mpf(float.fromhex(consts["kSixthLo"]))
    assert abs(sixth * 6 - 1) < mp.mpf(2) ** -46


def test_table_driven_log_decomposition():
    """ff_log's steps on the host (FP64 evaluation with the FP32 table): the
    exponent and the 7-bit interval index from hi, r = m F - 1 below 2^-7,
    log x = e log 2 - log F + log(1 + r) to 1e-15 of max(1, |log x|)."""
    tab = _array(LOG, "g_log_tab_f[")
    import random
    rnd = random.Random(5)
    worst = 0.0
    for _ in range(20000):
        x = math.exp(rnd.uniform(-80.0, 20.0))
        hi = _f32(x)
        lo = _f32(x - hi)
        bits = struct.unpack("I", struct.pack("f", hi))[0]
        e = ((bits >> 23) & 0xFF) - 127
        i = (bits >> 16) & 127
        F, chi, clo = tab[i]
        m = (hi + lo) * 2.0 ** -e
        r = m * F - 1.0
        assert abs(r) < 2.0 ** -7
        l1p = r - r * r / 2 + r ** 3 * (1 / 3 - r * (1 / 4 - r * (1 / 5 - r * (1 / 6 - r / 7))))
        v = e * math.log(2.0) + (chi + clo) + l1p
        ref = math.log(hi + lo)
        worst = max(worst, abs(v - ref) / max(1.0, abs(ref)))
    assert worst < 2e-15
