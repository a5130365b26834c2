"""Constants of the table-driven binary64 exp used by the binary64 substep
kernels (Tang's method, 256 entries): each table entry within one unit in the
last place of 2^(j/256) or 2^(-j/256), the split of ln 2 / 256, that the
committed header is what its generator writes, and the method itself carried
out step for step on the host (exact fused multiply-adds) within one unit in
the last place of the host's exp.  CPU only."""
import math
import os
import re
import struct
import subprocess
import sys
from fractions import Fraction

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2103_01597_gb300", "csrc")
HEADER = os.path.join(CSRC, "exp_table.cuh")


def _read():
    s = open(HEADER).read()
    consts = {m.group(1): float.fromhex(m.group(2))
              for m in re.finditer(r"constexpr double (EXP_\w+) = (-?0x[0-9a-fp.+-]+);", s)}
    body = s[s.index("EXP_TAB[512] = {") + len("EXP_TAB[512] = {"):s.index("};")]
    tab = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fp.+-]+", body)]
    return consts, tab


def test_table_entries_within_one_ulp():
    _, tab = _read()
    assert len(tab) == 512
    for j in range(256):
        for v, e in ((tab[j], j / 256), (tab[256 + j], -j / 256)):
            assert abs(v - 2.0 ** e) <= math.ulp(v), (j, e, v)
    assert tab[0] == 1.0 and tab[256] == 1.0
    # monotone: 2^(j/256) increasing, 2^(-j/256) decreasing
    assert all(tab[j] < tab[j + 1] for j in range(255))
    assert all(tab[256 + j] > tab[257 + j] for j in range(255))


def test_reduction_constants():
    c, _ = _read()
    l1 = Fraction(c["EXP_L1"])
    assert (l1 * 2 ** 40).denominator == 1          # a multiple of 2^-40
    sig = (l1 * 2 ** 40).numerator
    while sig % 2 == 0:
        sig //= 2
    assert sig.bit_length() <= 29                   # N * L1 exact for |N| < 2^24
    assert abs(c["EXP_L2"]) < 2.0 ** -40
    assert abs((c["EXP_L1"] + c["EXP_L2"]) * 256 - math.log(2)) <= 2 * math.ulp(math.log(2))
    assert abs(c["EXP_INV"] - 256 / math.log(2)) <= math.ulp(c["EXP_INV"])


def test_header_is_generated(tmp_path):
    # the generator writes beside itself: run a copy in a scratch directory
    src = open(os.path.join(CSRC, "gen_exp_table.py")).read()
    gen = tmp_path / "gen_exp_table.py"
    gen.write_text(src)
    subprocess.run([sys.executable, str(gen)], check=True, cwd=tmp_path)
    assert (tmp_path / "exp_table.cuh").read_text() == open(HEADER).read()


# ---- the method, step for step on the host ---------------------------------
# fma(a, b, c) rounded once: exact rational arithmetic, then Python's correctly
# rounded int/int division.

def _fma(a, b, c):
    v = Fraction(a) * Fraction(b) + Fraction(c)
    return v.numerator / v.denominator


def _bits(v):
    return struct.unpack("<q", struct.pack("<d", v))[0]


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _exp_pm(x, c, tab):
    sh = 6755399441055744.0  # 1.5 * 2^52
    t = _fma(x, c["EXP_INV"], sh)
    nd = t - sh
    low = _bits(t) & 0xFFFFFFFF
    n = low - (1 << 32) if low >= 1 << 31 else low
    r = _fma(-nd, c["EXP_L2"], _fma(-nd, c["EXP_L1"], x))
    p = _fma(r, 1.0 / 24.0, 1.0 / 6.0)
    p = _fma(p, r, 0.5)
    p = _fma(p * r, r, r)
    q = _fma(r, 1.0 / 24.0, -1.0 / 6.0)
    q = _fma(q, r, 0.5)
    q = _fma(q * r, r, -r)
    j, m = n & 255, n >> 8
    ep = _from_bits(_bits(_fma(tab[j], p, tab[j])) + (m << 52))
    em = _from_bits(_bits(_fma(tab[256 + j], q, tab[256 + j])) - (m << 52))
    return ep, em


def test_method_on_the_host_within_one_ulp():
    c, tab = _read()
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(-699.9, 699.9, 1500)) + list(rng.uniform(-2, 2, 1500))
    xs += [k * math.log(2) / 256 for k in range(-40, 41)] + [0.0, 1.0, -1.0, 699.99, -699.99]
    worst = 0
    for x in xs:
        ep, em = _exp_pm(x, c, tab)
        for got, want in ((ep, math.exp(x)), (em, math.exp(-x))):
            worst = max(worst, abs(_bits(got) - _bits(want)))
    assert worst <= 1
    assert _exp_pm(0.0, c, tab) == (1.0, 1.0)
