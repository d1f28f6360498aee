"""Generate csrc/exp_table.h: constants of the table-driven FP64 exponential.

Method (P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989), with a
table of N = 2^BITS = 256 entries:
exp(x) = 2^(n/N) * exp(r) with n = round(N x / ln 2) and
r = x - n ln2/N, |r| <= ln2/(2N); 2^(n/N) = 2^(n >> BITS) * T[n & (N-1)] with
T[j] = 2^(j/N); exp(r) by its Taylor polynomial of degree DEG = 4 (remainder
below r^5/5! < 4e-17 on |r| <= ln2/512).

A cheaper variant for residual evaluations that only need ~1e-13 relative
accuracy uses the same table with the reduction r = x - n L in one step
(L = ln2/N rounded to the nearest double; error |n| ulp(L)/2 < 1e-14 for
|x| < 700) and the Taylor polynomial of degree 3 (remainder below
r^4/4! < 1.4e-13 on |r| <= ln2/512).

Every constant is computed here with 60-digit decimal arithmetic and rounded
to the nearest double: T[j], N/ln2, the two-part split of ln2/N (high part
with 33 significant bits so that n * high is exact for |n| < 2^20) and 1/k!.
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


BITS = 8
N = 1 << BITS
DEG = 4
HI_BITS = 33


def main():
    ln2 = d_ln2()
    L = ln2 / N
    inv_l = N / ln2
    # high part of L with HI_BITS significant bits
    f = float(L)
    m, e = __import__("math").frexp(f)
    scale = 2 ** HI_BITS
    hi = round(m * scale) / scale
    hi = __import__("math").ldexp(hi, e)
    lo = float(L - Decimal(hi))
    table = [float(d_exp(Decimal(j) * ln2 / N)) for j in range(N)]
    fact = [float(Decimal(1) / Decimal(__import__("math").factorial(k))) for k in range(DEG + 1)]
    out = []
    out.append("// Generated by gen_exp_table.py: constants of the table-driven FP64")
    out.append("// exponential (Tang's method), each computed with 60-digit decimal")
    out.append("// arithmetic and rounded to the nearest double.")
    out.append("#pragma once")
    out.append("namespace alb {")
    out.append("constexpr int EXPT_BITS = %d;  // table of 2^EXPT_BITS entries" % BITS)
    out.append("constexpr int EXPT_N = %d;" % N)
    out.append("constexpr double EXPT_INV_L = %s;  // %d / ln 2" % (hexd(inv_l), N))
    out.append("constexpr double EXPT_L_HI = %s;   // ln2/%d, %d significant bits"
               % (hexd(hi), N, HI_BITS))
    out.append("constexpr double EXPT_L_LO = %s;   // ln2/%d - EXPT_L_HI" % (hexd(lo), N))
    out.append("constexpr double EXPT_L = %s;      // ln2/%d (one-step reduction)"
               % (hexd(L), N))
    for k in range(2, DEG + 1):
        out.append("constexpr double EXPT_C%d = %s;  // 1/%d!" % (k, hexd(fact[k]), k))
    out.append("}  // namespace alb")
    out.append("// T[j] = 2^(j/%d), j = 0..%d, as an initializer list" % (N, N - 1))
    out.append("#define ALB_EXPT_TABLE_VALUES \\")
    for j in range(0, N, 2):
        tail = ", \\" if j < N - 2 else ""
        out.append("    %s, %s%s" % (hexd(table[j]), hexd(table[j + 1]), tail))
    print("\n".join(out))


if __name__ == "__main__":
    main()
