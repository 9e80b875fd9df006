"""Write ff_tables.h: constants of the double-float exponential in ff_math.h.

Table-driven exponential after P. T. P. Tang, "Table-driven implementation of
the exponential function in IEEE floating-point arithmetic", ACM TOMS 15 (1989):
exp(-x) = 2^(-k/64) exp(-r), x = k ln2/64 + r.  The 64 values 2^(-j/64) are
stored as unevaluated float pairs (hi + lo), and ln2/64 is split in three
floats (Cody-Waite) with an 11-bit leading part so that k * C1 is exact for
k < 2^13.  Values are computed here with 60-digit decimal arithmetic.
"""
import decimal
import os
import struct

decimal.getcontext().prec = 60
D = decimal.Decimal


def f32(v: D) -> float:
    return struct.unpack("f", struct.pack("f", float(v)))[0]


def split(v: D):
    hi = f32(v)
    lo = f32(v - D(hi))
    return hi, lo


def hexf(x: float) -> str:
    return float.hex(x) + "f" if x != 0.0 else "0.0f"


def main():
    ln2 = D(2).ln()
    c = ln2 / 64
    # C1: 11 significant bits
    e = c.adjusted()
    scale = D(2) ** (11 - 1 - int((c.ln() / ln2).to_integral_value(rounding=decimal.ROUND_FLOOR)))
    c1 = (c * scale).to_integral_value(rounding=decimal.ROUND_FLOOR) / scale
    c2 = D(f32(c - c1))
    c3 = D(f32(c - c1 - c2))
    assert float(c1) == f32(c1)
    lines = ["// Generated by gen_ff_tables.py: constants of the double-float exponential.",
             "#pragma once", "namespace mra {",
             "// ln2/64 = C1 + C2 + C3 (C1 has 11 significant bits)",
             "#define MRA_FF_C1 %s" % hexf(float(c1)),
             "#define MRA_FF_C2 %s" % hexf(float(c2)),
             "#define MRA_FF_C3 %s" % hexf(float(c3)),
             "#define MRA_FF_INV_C %s  // 64/ln2, only used to pick k" % hexf(f32(64 / ln2)),
             "// 2^(-j/64), j = 0..63, as hi + lo float pairs",
             "#define MRA_FF_EXP2_TABLE { \\"]
    for j in range(64):
        v = (-(D(j) / 64) * ln2).exp()
        hi, lo = split(v)
        lines.append("    {%s, %s}%s \\" % (hexf(hi), hexf(lo), "," if j < 63 else ""))
    lines += ["}", "} // namespace mra", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ff_tables.h")
    open(out, "w").write("\n".join(lines))
    print(out, float(c1), float(c2), float(c3))


if __name__ == "__main__":
    main()
