"""Parametric sweeps: many independent channels advanced together through
replayed CUDA graphs, checked against lone runs of the same instances (the
same kernel, so the same numbers) and against the oracle.

The node-to-CTA schedule (rows per CTA) changes only the order of the FP64
column reductions that feed the end-column density correction (Eq. rho2).
Its factor is rounded to FP32, so a different summation order can move it by
one FP32 ulp: runs under different schedules agree to FP32 rounding noise
(1e-6 here, a tenth of the parity tolerance), not bitwise."""
import numpy as np
import pytest

import oracle
from paper_1603_08221_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5
RTOL_U = 1e-5
ATOL_U = 3e-8
RTOL_SCHED = 1e-6

# small, quickly converging channels of different shapes and gases
SMALL = [
    dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=1.5, Kn_out=0.3, N=8, N_x=48),
    dict(m_a=workloads.NE, m_b=workloads.AR, C_l=0.3, theta=2.0, Kn_out=0.5, N=16, N_x=40),
    dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.7, theta=1.8, Kn_out=1.0, N=8, N_x=100),
    dict(m_a=workloads.NE, m_b=workloads.AR, C_l=0.1, theta=1.5, Kn_out=0.2, N=24, N_x=70),
]


@pytest.fixture(scope="module", autouse=True)
def _libs():
    binding.load()
    oracle.build()


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _lone(p, tol, max_steps, check):
    g = binding.LbmMix(**p)
    g.init()
    st, steps, R = g.run_to_steady(tol, max_steps, check)
    return g, st, steps, R


def test_sweep_equals_lone_runs():
    sw = binding.LbmSweep(SMALL)
    sw.init()
    steps, R, status = sw.run_to_steady(1e-7, 40000, 500, autotune=False)
    assert sw.schedule()[0] == 0
    for k, p in enumerate(SMALL):
        g, st, n, r = _lone(p, 1e-7, 40000, 500)
        assert (status[k], steps[k]) == (st, n), k
        assert R[k] == r, k
        m, mg = sw.instance(k).moments(), g.moments()
        for key in m:
            assert np.array_equal(m[key], mg[key]), (k, key)
        assert sw.instance(k).separation()["CL"] == g.separation()["CL"]


def test_sweep_autotune_keeps_the_integration():
    sw = binding.LbmSweep(SMALL)
    sw.init()
    steps, R, status = sw.run_to_steady(1e-7, 40000, 500, autotune=True)
    policy, rows, ms = sw.schedule()
    assert 0 <= policy < binding.LBM_SWEEP_NPOLICY
    assert all(t > 0 for t in ms)
    assert all(r % 8 == 0 and r >= 8 for r in rows)
    for k, p in enumerate(SMALL):
        g, st, n, r = _lone(p, 1e-7, 40000, 500)
        assert status[k] == st and abs(steps[k] - n) <= 500, k
        m, mg = sw.instance(k).moments(), g.moments()
        if steps[k] == n:
            for key in ("rho_a", "rho_b"):
                assert _relerr(m[key], mg[key]) < RTOL_SCHED, (k, key)


def test_sweep_instances_against_oracle():
    sw = binding.LbmSweep(SMALL)
    sw.init()
    sw.step(300)
    for k, p in enumerate(SMALL):
        o = oracle.Oracle(p)
        o.init()
        o.step(300)
        mg, mo = sw.instance(k).moments(), o.moments()
        for key in ("rho_a", "rho_b"):
            assert _relerr(mg[key], mo[key]) < RTOL_RHO, (k, key)
        scale = max(np.abs(mo["ua_x"]).max(), np.abs(mo["ub_x"]).max())
        for key in ("ua_x", "ua_y", "ub_x", "ub_y"):
            assert np.abs(mg[key] - mo[key]).max() < RTOL_U * scale + ATOL_U, (k, key)


@pytest.mark.parametrize("rows", [8, 16, 24, 64])
def test_rows_per_block_changes_only_reduction_order(rows):
    p = workloads.preset("heli_argon_1280x64", N=64, N_x=200)
    ref = binding.LbmMix(**p)
    ref.init()
    ref.step(400)
    g = binding.LbmMix(**p)
    g.set_rows_per_block(rows)
    g.init()
    g.step(400)
    m, mr = g.moments(), ref.moments()
    for key in ("rho_a", "rho_b"):
        assert _relerr(m[key], mr[key]) < RTOL_SCHED, key
    scale = np.abs(mr["ua_x"]).max()
    for key in ("ua_x", "ub_x"):
        assert np.abs(m[key] - mr[key]).max() < 10 * RTOL_SCHED * scale, key
    assert abs(g.separation()["CL"] - ref.separation()["CL"]) < 1e-6


def test_sweep_reports_a_diverging_instance():
    """An unstable instance stops with LBM_ENONFINITE; the others go on."""
    unstable = workloads.sweep_instances()[42]
    sw = binding.LbmSweep([unstable, SMALL[0]])
    sw.init()
    steps, R, status = sw.run_to_steady(1e-7, 40000, 500)
    assert status[0] == binding.LBM_ENONFINITE and steps[0] <= 2000
    assert status[1] == binding.LBM_OK


def test_sweep_with_no_steps():
    sw = binding.LbmSweep(SMALL[:2])
    sw.init()
    steps, R, status = sw.run_to_steady(1e-7, 0, 500)
    assert steps == [0, 0] and status == [binding.LBM_ENOTCONVERGED] * 2
    with pytest.raises(binding.LbmError):
        sw.run_to_steady(1e-7, 1000, 501)  # odd check interval: no whole graphs



def _same_sequence(run, handles):
    """run_to_steady (run()), then on every handle a change of what captured
    sweep graphs bake in, then run_to_steady again; returns the outcomes."""
    out = [run()]
    for h in handles:
        h.step(1)  # odd: the buffer parity flips under any captured graph
    out.append(run())
    for h in handles:
        h.set_post_state(h.get_post_state())  # upload: parity reset to buffer 0
    out.append(run())
    for h in handles:
        h.set_rows_per_block(16)  # schedule: the row-block partials are reallocated
    out.append(run())
    for h in handles:
        h.rereference()  # the reference-density table swaps
    out.append(run())
    return out


def test_sweep_graphs_follow_state_changes():
    """A captured graph bakes in the buffer parity, schedule and reference
    table of the state it was captured from; calls on the borrowed handles
    that change them between run_to_steady calls must lead to a recapture,
    so that every instance still takes exactly the steps of a lone handle
    driven through the same calls (bitwise the same state)."""
    params = SMALL[:2]
    sw = binding.LbmSweep(params)
    sw.init()
    insts = [sw.instance(k) for k in range(len(params))]

    def run_sweep():
        return [tuple(v) for v in zip(*sw.run_to_steady(1e-12, 1000, 500, autotune=False))]
    swept = _same_sequence(run_sweep, insts)
    for k, p in enumerate(params):
        g = binding.LbmMix(**p)
        g.init()

        def run_lone(g=g):
            st, n, r = g.run_to_steady(1e-12, 1000, 500)
            return (n, r, st)
        lone = _same_sequence(run_lone, [g])
        assert [o[k] for o in swept] == lone, k
        m, mg = insts[k].moments(), g.moments()
        for key in m:
            assert np.array_equal(m[key], mg[key]), (k, key)
        assert insts[k].separation()["CL"] == g.separation()["CL"]
