"""The FP64 exponential-integral tables of the adjoint kernels
(lbm_adjoint.cu, generated by csrc/gen_e1_table.py): the fixed-length series
for 0 < x <= 1 and the Chebyshev series of x e^x E_1(x) on [1, 32], read
from the source and evaluated here exactly as the device code does (Horner;
segment from the binary exponent of x, Clenshaw's recurrence), against
scipy's E_1 (no GPU needed)."""
import math
import os
import re

import numpy as np
import scipy.special

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1603_08221_gb300", "csrc", "lbm_adjoint.cu")
NUM = r"[-+]?[0-9.]+(?:e[-+]?[0-9]+)?"


def _tables():
    src = open(SRC).read()
    s = src[src.index("kE1Series[kE1SeriesTerms] = {"):]
    s = re.sub(r"//[^\n]*", "", s[s.index("{") + 1:s.index("};")])
    series = [float(v) for v in re.findall(NUM, s)]
    c = src[src.index("kE1Cheb[5][kE1ChebTerms] = {"):]
    c = re.sub(r"//[^\n]*", "", c[c.index("{") + 1:c.index("};")])
    cheb = [[float(v) for v in re.findall(NUM, r)] for r in c.split("}") if re.search(NUM, r)]
    return series, cheb


def _e1(x, series, cheb):
    if x <= 1.0:
        s = series[-1]
        for k in range(len(series) - 2, -1, -1):
            s = s * x + series[k]
        return -0.57721566490153286061 - math.log(x) - s * x
    _, e = math.frexp(x)
    seg = min(max(e - 1, 0), 4)
    lo = math.ldexp(1.0, seg)
    t = (x - lo) / lo * 2.0 - 1.0
    c = cheb[seg]
    b1 = b2 = 0.0
    for k in range(len(c) - 1, 0, -1):
        b1, b2 = 2.0 * t * b1 - b2 + c[k], b1
    return (t * b1 - b2 + c[0]) * math.exp(-x) / x


def test_e1_tables_against_scipy():
    series, cheb = _tables()
    assert len(series) == 20 and len(cheb) == 5 and all(len(c) == 20 for c in cheb)
    xs = np.concatenate([np.geomspace(1e-6, 1.0, 300), np.linspace(1.0, 32.0, 3001),
                         [1.0, 2.0, 4.0, 8.0, 16.0, 32.0, np.nextafter(1.0, 2.0)]])
    err = max(abs(_e1(float(x), series, cheb) / scipy.special.exp1(x) - 1.0) for x in xs)
    assert err < 4e-15
