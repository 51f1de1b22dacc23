"""The seeded input generators: deterministic, in the stated ranges."""
from paper_1603_08221_gb300 import workloads


def test_sweep_instances_deterministic_and_in_range():
    a, b = workloads.sweep_instances(), workloads.sweep_instances()
    assert a == b and len(a) == 96
    for k, p in enumerate(a):
        assert p["m_a"] == (workloads.HE if k % 2 == 0 else workloads.NE)
        assert p["C_l"] == (0.1, 0.3, 0.5, 0.7, 0.9)[k % 5]
        assert 1.5 <= p["theta"] <= 5.0 and 0.01 <= p["Kn_out"] <= 1.0
        assert p["N"] in (16, 32, 64, 128) and p["L_over_H"] in (10.0, 20.0, 50.0)
    nodes = [p["N"] * workloads.n_x(p) for p in a]
    assert min(nodes) >= 2560 and max(nodes) <= 819200
    assert workloads.sweep_instances(seed=1) != a
