"""Write ``exp_table.cuh``: the constants of the table-driven binary64 exp.

The table holds 2^(j/256) and 2^(-j/256) for j = 0..255, each the binary64
value nearest the exact one, computed here with Python's decimal module at 60
significant digits (independent of any libm).  ln 2 / 256 is split as L1 + L2
with L1 a multiple of 2^-40 (29 significant bits, so N * L1 is exact for
|N| < 2^24; the kernels use |N| < 2^18), and 256 / ln 2 is rounded to binary64.

Run: python gen_exp_table.py  (rewrites exp_table.cuh beside this file)
"""
import os
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def nearest_double(d):
    # float(Decimal) rounds to nearest binary64
    return float(d)


def main():
    ln2 = Decimal(2).ln()
    tab_p = [nearest_double(Decimal(2) ** (Decimal(j) / 256)) for j in range(256)]
    tab_m = [nearest_double(Decimal(2) ** (Decimal(-j) / 256)) for j in range(256)]
    l = ln2 / 256
    l1 = Fraction(int((l * (Decimal(2) ** 40)).to_integral_value()), 2 ** 40)
    l2 = nearest_double(l - Decimal(l1.numerator) / Decimal(l1.denominator))
    inv = nearest_double(Decimal(256) / ln2)
    lines = [
        "// Generated by gen_exp_table.py: constants of the table-driven binary64 exp",
        "// (Tang's method, 256 entries).  2^(j/256) and 2^(-j/256), j = 0..255, each",
        "// the binary64 value nearest the exact one; ln 2 / 256 = EXP_L1 + EXP_L2 with",
        "// EXP_L1 a multiple of 2^-40; EXP_INV = 256 / ln 2 rounded.",
        "#pragma once",
        "",
        "namespace ac {",
        "",
        "constexpr double EXP_INV = %s;" % float(inv).hex(),
        "constexpr double EXP_L1 = %s;" % float(l1).hex(),
        "constexpr double EXP_L2 = %s;" % float(l2).hex(),
        "",
        "// [0, 256): 2^(j/256); [256, 512): 2^(-j/256)",
        "__device__ const double EXP_TAB[512] = {",
    ]
    vals = tab_p + tab_m
    for i in range(0, 512, 3):
        lines.append("    " + ", ".join(v.hex() for v in vals[i:i + 3]) + ",")
    lines += ["};", "", "}  // namespace ac", ""]
    with open(os.path.join(HERE, "exp_table.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
