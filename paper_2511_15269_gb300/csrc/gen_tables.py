"""Writes tables_gen.h: the constant tables of the evaluation kernels as
literal constexpr arrays, so that fully unrolled kernels carry every entry as
an instruction immediate.

Formulas (their derivation is in the header comment of expansion.cuh):
  quarter-turn Wigner elements d^n_{m,k}(pi/2) = 2^-n sqrt((n+m)!(n-m)!/((n+k)!(n-k)!))
      * sum_t (-1)^(m-k+t) C(n+k,t) C(n-k,n-m-t)   (exact integer sum),
  B = Y(-pi/2) Z(-pi/2), B^-1 = Z(pi/2) Y(pi/2) in the internal basis,
  axial M2L/M2M/L2L factors and the normalised regular-basis recursion constants.
Square roots of exact rationals are taken with math.sqrt of the correctly
rounded rational.
"""
import math
import os
import sys
from fractions import Fraction
from math import comb, factorial

MAXP = 10


def d_right(n, m, k):
    s = 0
    for t in range(0, 2 * n + 1):
        if n + k - t < 0 or n - m - t < 0 or m - k + t < 0:
            continue
        s += (-1) ** (m - k + t) * comb(n + k, t) * comb(n - k, n - m - t)
    norm = math.sqrt(float(Fraction(factorial(n + m) * factorial(n - m), factorial(n + k) * factorial(n - k))))
    return math.ldexp(norm * s, -n)


def y_right(n, sign, m, src):
    if (m >= 0) != (src >= 0):
        return 0.0
    am, k = abs(m), abs(src)
    d = (lambda a, b: d_right(n, a, b)) if sign > 0 else (lambda a, b: d_right(n, b, a))
    if k > 0:
        return d(am, k) + (1.0 if m >= 0 else -1.0) * (-1.0 if k % 2 else 1.0) * d(am, -k)
    return d(am, 0)


def z_right(sign, m, mc):
    if m == 0 or mc == 0:
        return 1.0 if (m == 0 and mc == 0) else 0.0
    q = (abs(m) * sign) % 4
    c = {0: 1.0, 2: -1.0}.get(q, 0.0)
    s = {1: 1.0, 3: -1.0}.get(q, 0.0)
    if m > 0:
        return c if mc == m else (-s if mc == -m else 0.0)
    return c if mc == m else (s if mc == -m else 0.0)


def tables():
    B, Bi = [], []
    for n in range(MAXP + 1):
        for i in range(2 * n + 1):
            for j in range(2 * n + 1):
                B.append(sum(y_right(n, -1, i - n, l) * z_right(-1, l, j - n) for l in range(-n, n + 1)))
                Bi.append(sum(z_right(1, i - n, l) * y_right(n, 1, l, j - n) for l in range(-n, n + 1)))
    m2l, m2m, l2l = [], [], []
    for n in range(MAXP + 1):
        for k in range(MAXP + 1):
            for m in range(MAXP + 1):
                a = b = c = 0.0
                if m <= n and m <= k:
                    r = Fraction(factorial(n + k) ** 2,
                                 factorial(n - m) * factorial(n + m) * factorial(k - m) * factorial(k + m))
                    a = (-1.0 if (k + m) % 2 else 1.0) * math.sqrt(float(r))
                if m <= k <= n:
                    b = math.sqrt(float(comb(n - m, k - m) * comb(n + m, k + m)))
                if m <= n <= k:
                    c = (-1.0 if (k - n) % 2 else 1.0) * math.sqrt(float(comb(k - m, n - m) * comb(k + m, n + m)))
                m2l.append(a)
                m2m.append(b)
                l2l.append(c)
    rdiag = [math.sqrt(float(Fraction(2 * n - 1, 2 * n))) if n >= 1 else 0.0 for n in range(MAXP + 1)]
    rsub = [math.sqrt(2 * n + 1) for n in range(MAXP + 1)]
    ra, rb = [], []
    for n in range(MAXP + 1):
        for m in range(MAXP + 1):
            if m + 2 <= n:
                nm = (n - m) * (n + m)
                ra.append((2 * n - 1) / math.sqrt(nm))
                rb.append(math.sqrt(float(Fraction((n - m - 1) * (n + m - 1), nm))))
            else:
                ra.append(0.0)
                rb.append(0.0)
    return dict(kB=B, kBi=Bi, kAxM2L=m2l, kAxM2M=m2m, kAxL2L=l2l, kRDiag=rdiag, kRSub=rsub, kRA=ra, kRB=rb)


def main(out):
    t = tables()
    lines = ["// Generated by gen_tables.py; do not edit.", "#pragma once", "namespace fmm {", "namespace gen {"]
    for name, vals in t.items():
        body = ",\n  ".join(", ".join(repr(float(v)) for v in vals[i:i + 6]) for i in range(0, len(vals), 6))
        lines.append("constexpr double %s[%d] = {\n  %s};" % (name, len(vals), body))
    lines += ["}  // namespace gen", "}  // namespace fmm", ""]
    tmp = out + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(lines))
    os.replace(tmp, out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables_gen.h"))
