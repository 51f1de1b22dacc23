"""The complex-step reference (oracle/complex_step.py): its real part is the
C oracle's time integration, and its derivatives agree with central
differences of the C oracle.  It then serves as the exact reference of the
GPU adjoint."""
import numpy as np
import pytest

import oracle
from oracle import complex_step as cs
from paper_1603_08221_gb300 import workloads

P = dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=2.0, Kn_out=0.2, N=8, N_x=40)
STEPS = 200


@pytest.fixture(scope="module")
def alpha():
    oracle.build()
    return np.minimum(workloads.random_accommodation(40, 1).reshape(2, 40), 1 - 1e-5)


def _c_oracle(p, al, steps):
    o = oracle.Oracle(p)
    o.init()
    o.set_accommodation_field(np.ascontiguousarray(al.ravel()))
    o.step(steps)
    f = o.get_post_state()
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
    return o.separation()["CL"], float((cx[:, None] * f[0, :, :, -2]).sum()), f


def test_real_part_is_the_c_oracle(alpha):
    CL, fl, _, _, F = cs.run(P, STEPS, alpha)
    CLo, flo, Fo = _c_oracle(P, alpha, STEPS)
    assert np.abs(F[..., 1:-1] - Fo[..., 1:-1]).max() < 1e-13 * np.abs(Fo).max()
    assert abs(CL - CLo) < 1e-13 and abs(fl - flo) < 1e-12 * abs(flo)


@pytest.mark.parametrize("what", ["theta", "Kn_out", "alpha"])
def test_derivatives_match_central_differences_of_the_c_oracle(alpha, what):
    h = 1e-6
    d_al = np.zeros_like(alpha)
    d_al[1, 17] = 1.0  # top wall, column 17
    kw = {"theta": dict(d_theta=1.0), "Kn_out": dict(d_kn=1.0),
          "alpha": dict(d_alpha=d_al)}[what]
    _, _, dCL, dfl, _ = cs.run(P, STEPS, alpha, **kw)
    pp, pm = dict(P), dict(P)
    ap, am = alpha, alpha
    if what == "alpha":
        ap, am = alpha + h * d_al, alpha - h * d_al
    else:
        pp[what] += h
        pm[what] -= h
    (cp, fp, _), (cm, fm, _) = _c_oracle(pp, ap, STEPS), _c_oracle(pm, am, STEPS)
    fd_cl, fd_fl = (cp - cm) / (2 * h), (fp - fm) / (2 * h)
    eps = np.finfo(float).eps
    assert abs(dCL - fd_cl) <= 1e-6 * abs(fd_cl) + 64 * eps / h
    assert abs(dfl - fd_fl) <= 1e-6 * abs(fd_fl) + 64 * eps * abs(fp) / h


def test_real_part_with_unequal_end_compositions():
    """C_l,in != C_l,out (as in Cases 4, 5, 9, 10 of Table 1) with an
    accommodation field, on a 120 x 10 channel at theta = 1.5 (shorter
    channels with unequal ends diverge in both): the restatement and the C
    oracle stay equal."""
    oracle.build()
    p = dict(P, C_l=0.5, C_l_out=0.3, theta=1.5, Kn_out=0.1, N=10, N_x=120)
    al = workloads.random_accommodation(120, seed=1, spread=0.05).reshape(2, 120)
    CL, fl, _, _, F = cs.run(p, 400, al)
    CLo, flo, Fo = _c_oracle(p, al, 400)
    assert np.isfinite(Fo).all()
    assert np.abs(F[..., 1:-1] - Fo[..., 1:-1]).max() < 1e-13 * np.abs(Fo).max()
    assert abs(CL - CLo) < 1e-13
