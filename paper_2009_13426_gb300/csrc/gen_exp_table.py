"""Generate csrc/exp_table.h: constants of the table-driven FP64 exponential.

Method (P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989):
exp(x) = 2^(n/32) * exp(r) with n = round(32 x / ln 2) and
r = x - n ln2/32, |r| <= ln2/64; 2^(n/32) = 2^(n >> 5) * T[n & 31] with
T[j] = 2^(j/32); exp(r) by its Taylor polynomial of degree 6 (remainder
below r^7/7! < 4e-18 on |r| <= ln2/64).

Every constant is computed here with 60-digit decimal arithmetic and rounded
to the nearest double: T[j], 32/ln2, the two-part split of ln2/32 (high part
with 38 significant bits so that n * high is exact for |n| < 2^15) and 1/k!.
Run: python gen_exp_table.py > exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def d_exp(x):
    """exp of a Decimal by its Taylor series (x small)."""
    s, t, k = Decimal(1), Decimal(1), 1
    while True:
        t = t * x / k
        if abs(t) < Decimal(10) ** -58:
            break
        s += t
        k += 1
    return s


def d_ln2():
    # ln 2 = 2 atanh(1/3) = 2 sum_{k>=0} 3^{-(2k+1)} / (2k+1)
    s, k = Decimal(0), 0
    while True:
        term = Decimal(1) / (Decimal(3) ** (2 * k + 1) * (2 * k + 1))
        if term < Decimal(10) ** -58:
            break
        s += term
        k += 1
    return 2 * s


def hexd(x):
    return float(x).hex()


def main():
    ln2 = d_ln2()
    L = ln2 / 32
    inv_l = 32 / ln2
    # high part of L with 38 significant bits
    f = float(L)
    m, e = __import__("math").frexp(f)
    scale = 2 ** 38
    hi = round(m * scale) / scale
    hi = __import__("math").ldexp(hi, e)
    lo = float(L - Decimal(hi))
    table = [float(d_exp(Decimal(j) * ln2 / 32)) for j in range(32)]
    fact = [float(Decimal(1) / Decimal(__import__("math").factorial(k))) for k in range(7)]
    out = []
    out.append("// Generated by gen_exp_table.py: constants of the table-driven FP64")
    out.append("// exponential (Tang's method), each computed with 60-digit decimal")
    out.append("// arithmetic and rounded to the nearest double.")
    out.append("#pragma once")
    out.append("namespace alb {")
    out.append("constexpr double EXPT_INV_L = %s;  // 32 / ln 2" % hexd(inv_l))
    out.append("constexpr double EXPT_L_HI = %s;   // ln2/32, 38 significant bits" % hexd(hi))
    out.append("constexpr double EXPT_L_LO = %s;   // ln2/32 - EXPT_L_HI" % hexd(lo))
    for k in range(2, 7):
        out.append("constexpr double EXPT_C%d = %s;  // 1/%d!" % (k, hexd(fact[k]), k))
    out.append("}  // namespace alb")
    out.append("// T[j] = 2^(j/32), j = 0..31, as an initializer list")
    out.append("#define ALB_EXPT_TABLE_VALUES \\")
    for j in range(0, 32, 2):
        tail = ", \\" if j < 30 else ""
        out.append("    %s, %s%s" % (hexd(table[j]), hexd(table[j + 1]), tail))
    print("\n".join(out))


if __name__ == "__main__":
    main()
