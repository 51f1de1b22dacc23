"""Pins against numbers the paper prints (tests/golden/, each file cites its
passage): the MRT transform of Eq. m, the cases of Table 1 and the fixed
constants.  The oracle's matrix and the workload definitions must agree."""
import os

import numpy as np

import oracle
from paper_1603_08221_gb300 import binding, workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_oracle_matrix_is_the_printed_M():
    oracle.build()
    M = np.array(_rows("mrt_matrix_M.txt"), dtype=float)
    assert M.shape == (9, 9)
    assert np.array_equal(oracle.matrix_M(), M)
    # and its inverse is the oracle's Gauss-Jordan inverse
    assert np.abs(oracle.matrix_Minv() @ M - np.eye(9)).max() < 1e-13


def test_table1_runs_are_the_printed_cases():
    printed = {}
    gas = {"He": workloads.HE, "Ne": workloads.NE}
    for case, g, cin, cout, kns, ths in _rows("table1_cases.txt"):
        for kn in kns.split(","):
            for th in ths.split(","):
                printed[(int(case), float(kn), float(th))] = (gas[g], float(cin), float(cout))
    runs = workloads.paper_table1()
    assert len(runs) == len(printed)
    for name, p in runs:
        case = int(name.split("_")[0][4:])
        key = (case, p["Kn_out"], p["theta"])
        assert printed[key] == (p["m_a"], p["C_l"], p["C_l_out"]), name
        assert p["m_b"] == workloads.AR and p["N"] * workloads.n_x(p) == 20 * 700


def test_constants():
    c = {k: float(v) for k, v in _rows("constants.txt")}
    # the workloads' masses (standard atomic weights) have the printed ratios
    assert round(workloads.AR / workloads.HE) == c["ratio_HeAr"]
    assert round(workloads.AR / workloads.NE) == c["ratio_NeAr"]
    d = binding.lbm_mix_default_params()
    assert (d.tau_rho, d.tau_e, d.tau_eps) == (c["tau_rho"], c["tau_e"], c["tau_eps"])
