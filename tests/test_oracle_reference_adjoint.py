"""The reverse-mode reference (oracle/reference_adjoint.py, PyTorch CPU
autograd over a restatement of the time integration) against the
complex-step reference: two independent oracle-side derivatives."""
import numpy as np
import pytest

from oracle import complex_step as cs
from paper_1603_08221_gb300 import workloads

P = dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=2.0, Kn_out=0.2, N=8, N_x=40)
STEPS = 40


@pytest.mark.parametrize("objective,k", [("CL", 2), ("flux", 3)])
def test_reverse_mode_equals_complex_step(objective, k):
    torch = pytest.importorskip("torch")  # noqa: F841
    from oracle import reference_adjoint as ra
    al = np.minimum(workloads.random_accommodation(40, 1).reshape(2, 40), 1 - 1e-5)
    J, dth, dkn, dal = ra.gradient(P, STEPS, al, objective)
    CL, fl, _, _, _ = cs.run(P, STEPS, al)
    assert abs(J - (CL if objective == "CL" else fl)) < 1e-13 * max(1.0, abs(J))
    assert abs(dth / cs.run(P, STEPS, al, d_theta=1.0)[k] - 1) < 1e-10
    assert abs(dkn / cs.run(P, STEPS, al, d_kn=1.0)[k] - 1) < 1e-10
    v = np.random.default_rng(3).standard_normal(al.shape)
    assert abs((dal * v).sum() / cs.run(P, STEPS, al, d_alpha=v)[k] - 1) < 1e-10
