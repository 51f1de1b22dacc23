"""Generates the FP64 tables of the adjoint's exponential integral E_1
(lbm_adjoint.cu, between the "BEGIN/END generated E_1 tables" markers).

  0 < x <= 1:  E_1(x) = -gamma - ln x - sum_{k=1}^{K} (-x)^k / (k k!)
               (the convergent series, Abramowitz & Stegun 5.1.11), K fixed
               so that the remainder is below 1e-20: the coefficients
               (-1)^k / (k k!) for Horner's rule;
  1 < x <= 32: R(x) = x e^x E_1(x), a smooth function between 0.59 and 0.97,
               as a Chebyshev series on each of [1,2], [2,4], [4,8], [8,16],
               [16,32] (the Chebyshev interpolant at the extrema nodes of the
               smallest degree whose error against R evaluated in 40-digit
               arithmetic stays below 2e-17 relative), summed by Clenshaw's
               recurrence;
  x > 32:      the library keeps its continued fraction (A&S 5.1.22).

Run once (needs mpmath, which this image carries with sympy):
    python paper_1603_08221_gb300/csrc/gen_e1_table.py
and paste the printed block.
"""
from __future__ import annotations

import math

import mpmath as mp

mp.mp.dps = 40
INTERVALS = [(1, 2), (2, 4), (4, 8), (8, 16), (16, 32)]


def R(x):
    x = mp.mpf(x)
    return x * mp.e**x * mp.expint(1, x)


def cheb_coeffs(f, a, b, n):
    """Coefficients c_0..c_n of the Chebyshev interpolant of f on [a, b] at
    the n + 1 extrema nodes cos(pi j / n)."""
    xs = [mp.cos(mp.pi * j / n) for j in range(n + 1)]
    fv = [f((b - a) / 2 * t + (b + a) / 2) for t in xs]
    c = []
    for k in range(n + 1):
        s = mp.mpf(0)
        for j in range(n + 1):
            w = mp.mpf(0.5) if j in (0, n) else mp.mpf(1)
            s += w * fv[j] * mp.cos(mp.pi * j * k / n)
        ck = 2 * s / n
        if k in (0, n):
            ck /= 2
        c.append(ck)
    return c


def clenshaw(c, t):
    b1 = b2 = 0.0
    for ck in reversed(c[1:]):
        b1, b2 = 2.0 * t * b1 - b2 + ck, b1
    return t * b1 - b2 + c[0]


def max_rel_err(c, a, b):
    cd = [float(x) for x in c]
    worst = 0.0
    for i in range(401):
        x = a + (b - a) * i / 400
        t = (2 * x - (a + b)) / (b - a)
        ref = R(x)
        worst = max(worst, abs(float((mp.mpf(clenshaw(cd, t)) - ref) / ref)))
    return worst


def main():
    K = next(k for k in range(1, 40) if 1.0 / (k * math.factorial(k)) < 1e-20) - 1
    print("// BEGIN generated E_1 tables (gen_e1_table.py)")
    print(f"constexpr int kE1SeriesTerms = {K};")
    print("__constant__ double kE1Series[kE1SeriesTerms] = {  // (-1)^k / (k k!), k = 1..")
    coef = [mp.mpf(-1) ** k / (k * mp.factorial(k)) for k in range(1, K + 1)]
    print("    " + ",\n    ".join(mp.nstr(c, 20) for c in coef) + "};")
    tables = []
    for a, b in INTERVALS:
        for n in range(6, 60):
            c = cheb_coeffs(R, a, b, n)
            err = max_rel_err(c, a, b)
            if err < 2e-16:
                # drop trailing coefficients below the FP64 resolution of R
                while abs(c[-1]) < 1e-18:
                    c.pop()
                tables.append((a, b, c, err))
                break
    deg = max(len(c) for _, _, c, _ in tables)
    print(f"constexpr int kE1ChebTerms = {deg};")
    print("__constant__ double kE1Cheb[5][kE1ChebTerms] = {  // x e^x E_1(x) on [1,2] .. [16,32]")
    for a, b, c, err in tables:
        cc = list(c) + [mp.mpf(0)] * (deg - len(c))
        print(f"    {{  // [{a}, {b}], max relative error {err:.1e}")
        print("     " + ",\n     ".join(mp.nstr(x, 20) for x in cc) + "},")
    print("};")
    print("// END generated E_1 tables")


if __name__ == "__main__":
    main()
