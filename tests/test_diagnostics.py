"""Host-side diagnostics: the separation rate and dimensionless time on
synthetic histories, and the Table 1 run list."""
import numpy as np
import pytest

from paper_1603_08221_gb300 import diagnostics, workloads


def test_separation_rate_is_the_steepest_rise():
    steps = np.arange(1, 11) * 100
    cl = 0.02 * (1 - np.exp(-steps / 300.0))
    # the first interval, from the uniform state CL = 0, is the steepest
    assert diagnostics.separation_rate(steps, cl) == pytest.approx(cl[0] / 100.0)
    ramp = np.concatenate([[0.0, 0.001], 0.001 + 0.004 * np.arange(1, 9)])
    assert diagnostics.separation_rate(steps, ramp) == pytest.approx(0.004 / 100.0)
    with pytest.raises(ValueError):
        diagnostics.separation_rate([100], [0.1])


def test_dimensionless_time():
    t = diagnostics.dimensionless_time([0, 700, 1400], u_c=0.02, H=20)
    assert np.allclose(t, [0.0, 0.7, 1.4])


def test_table1_runs():
    runs = dict(workloads.paper_table1())
    assert len(runs) == 4 + 2 * 20 + 4 * 2
    c4 = runs["case4_kn1_theta2"]
    assert (c4["C_l"], c4["C_l_out"], c4["m_a"]) == (0.7, 0.3, workloads.HE)
    c9 = runs["case9_kn0.3_theta2"]
    assert (c9["C_l"], c9["C_l_out"], c9["m_a"]) == (0.7, 0.3, workloads.NE)
    assert all(p["N"] * workloads.n_x(p) == 20 * 700 for p in runs.values())
