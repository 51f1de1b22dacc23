"""The factored moment transforms of the FP64 adjoint kernels (mrt_fwd: m =
M v; mrt_tr: o = M^T d, in lbm_adjoint.cu), read from the source and
evaluated statement by statement in Python (fma(a, b, c) as a b + c), against
the matrix M of Eq. m as the paper prints it (tests/golden/mrt_matrix_M.txt).
No GPU needed."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1603_08221_gb300", "csrc", "lbm_adjoint.cu")
GOLDEN = os.path.join(ROOT, "tests", "golden", "mrt_matrix_M.txt")


def _matrix():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    return np.array(rows, dtype=float)


def _function(name):
    """The body of a device function of the source, as Python statements."""
    src = open(SRC).read()
    start = src.index(f"void {name}(")
    body = src[src.index("{", start) + 1:]
    depth, end = 1, 0
    for k, ch in enumerate(body):
        depth += ch == "{"
        depth -= ch == "}"
        if depth == 0:
            end = k
            break
    lines = []
    for stmt in re.sub(r"//[^\n]*", "", body[:end]).split(";"):
        stmt = " ".join(stmt.split())
        if not stmt:
            continue
        stmt = re.sub(r"^const double ", "", stmt)
        # "a = x, b = y" declarations become two statements
        parts = re.split(r",\s*(?=[A-Za-z_]\w*\s*=[^=])", stmt)
        lines.extend(parts)
    return "\n".join(lines)


def _run(name, vec_in, out_name):
    ns = {"fma": lambda a, b, c: a * b + c, out_name: [0.0] * 9,
          "v" if name == "mrt_fwd" else "d": list(vec_in)}
    exec(_function(name), ns)
    return np.array(ns[out_name])


def test_mrt_fwd_is_M():
    M = _matrix()
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.standard_normal(9)
        got = _run("mrt_fwd", v, "m")
        assert np.allclose(got, M @ v, rtol=0, atol=1e-13 * np.abs(v).sum()), (got, M @ v)
    for i in range(9):  # every column on its own
        e = np.zeros(9)
        e[i] = 1.0
        assert np.array_equal(_run("mrt_fwd", e, "m"), M[:, i])


def test_mrt_tr_is_M_transposed():
    M = _matrix()
    rng = np.random.default_rng(4)
    for _ in range(20):
        d = rng.standard_normal(9)
        got = _run("mrt_tr", d, "o")
        assert np.allclose(got, M.T @ d, rtol=0, atol=1e-13 * np.abs(d).sum()), (got, M.T @ d)
    for k in range(9):  # every row of M on its own
        e = np.zeros(9)
        e[k] = 1.0
        assert np.array_equal(_run("mrt_tr", e, "o"), M[k, :])


def test_inv_Mnorm_is_the_diagonal_of_M_M_transposed():
    """1/|M_k|^2 as the source tabulates it."""
    M = _matrix()
    src = open(SRC).read()
    s = src[src.index("inv_Mnorm(int k)"):]
    s = s[s.index("{", s.index("w[9]")) + 1:s.index("};")]
    w = [eval(t) for t in s.replace("\n", " ").split(",")]
    assert all(math.isclose(a, 1.0 / b, rel_tol=1e-15) for a, b in zip(w, (M * M).sum(axis=1)))
