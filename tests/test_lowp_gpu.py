"""Reduced-precision storage (BF16 / FP16 deviations, FP32 arithmetic, FP64
reductions) and re-referencing of the stored deviations.

Re-referencing is exact arithmetic up to one rounding of the storage type, so
with FP32 storage it is checked against the plain run at the parity
tolerances.  BF16 and FP16 storage round every stored deviation to 8 or 11
significant bits each step; their error against the FP32 run is bounded, not
small.  The bounds below are the errors measured on this hardware for the
Ne-Ar workload at 1/8 linear scale (2048 x 32, C_l = 0.5, theta = 2.5,
Kn_out = 0.5) with the library's default re-referencing (every 256 steps),
times two; the GPU path is deterministic (fixed-order reductions), so the
measurement repeats exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1603_08221_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5
RTOL_U = 1e-4
ATOL_U = 3e-8

SCALE_1_8 = dict(N=32, N_x=2048)

# measured error x 2 after 2000 steps, against the FP32 run
BOUNDS_2000 = {
    binding.LBM_BF16: dict(rho=5e-3, u=0.11, v=0.04, mdot=0.12, CL=3e-3),
    binding.LBM_FP16: dict(rho=2e-3, u=0.025, v=6e-3, mdot=1e-3, CL=1e-3),
}
# steady state (residual 1e-8 or the step cap): CL relative, mass flow relative
BOUNDS_STEADY = {
    binding.LBM_BF16: dict(CL=0.30, mdot=0.08),
    binding.LBM_FP16: dict(CL=0.30, mdot=0.01),
}


@pytest.fixture(scope="module", autouse=True)
def _libs():
    binding.load()
    oracle.build()


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _run(p, steps, **kw):
    g = binding.LbmMix(**p, **kw)
    g.init()
    g.step(steps)
    return g


def test_rereference_is_exact_with_fp32():
    """f before and after one re-reference agree to one FP32 rounding, and a
    run that re-references every 32 steps stays on the plain run."""
    p = workloads.preset("heli_argon_320x16")
    g = _run(p, 500, reref_every=0)
    f0 = g.get_post_state_f64()
    m0 = g.moments()
    g.rereference()
    f1 = g.get_post_state_f64()
    assert np.abs(f1 - f0).max() <= 2.0 ** -22 * np.abs(f0).max()
    # the moments of the current step stream the previous buffer, which must
    # follow the new reference too
    m1 = g.moments()
    for k in ("rho_a", "rho_b"):
        assert _relerr(m1[k], m0[k]) < 1e-6, k
    for k in ("ua_x", "ua_y", "ub_x", "ub_y"):
        assert np.abs(m1[k] - m0[k]).max() < 1e-6 * np.abs(m0["ua_x"]).max() + ATOL_U, k
    g.step(300)
    h = _run(p, 800, reref_every=32)
    mg, mh = g.moments(), h.moments()
    for k in ("rho_a", "rho_b"):
        assert _relerr(mh[k], mg[k]) < RTOL_RHO, k
    scale = max(np.abs(mg["ua_x"]).max(), np.abs(mg["ub_x"]).max())
    for k in ("ua_x", "ua_y", "ub_x", "ub_y"):
        assert np.abs(mh[k] - mg[k]).max() < RTOL_U * scale + ATOL_U, k


def test_rereference_against_oracle():
    """A re-referenced FP32 run is still the oracle's time integration."""
    p = workloads.preset("neon_argon_2048x32", N=16, N_x=200, theta=1.5)
    g = _run(p, 600, reref_every=50)
    o = oracle.Oracle(p)
    o.init()
    o.step(600)
    mg, mo = g.moments(), o.moments()
    for k in ("rho_a", "rho_b"):
        assert _relerr(mg[k], mo[k]) < RTOL_RHO, k
    scale = max(np.abs(mo["ua_x"]).max(), np.abs(mo["ub_x"]).max())
    for k in ("ua_x", "ua_y", "ub_x", "ub_y"):
        assert np.abs(mg[k] - mo[k]).max() < RTOL_U * scale + ATOL_U, k


@pytest.mark.parametrize("storage", [binding.LBM_BF16, binding.LBM_FP16])
def test_reduced_precision_error_bounds_2000_steps(storage):
    p = workloads.preset("neon_argon_16384x256", **SCALE_1_8)
    ref = _run(p, 2000)
    g = _run(p, 2000, storage=storage)
    m, mr = g.moments(), ref.moments()
    s, sr = g.separation(), ref.separation()
    b = BOUNDS_2000[storage]
    for k in ("rho_a", "rho_b"):
        assert np.isfinite(m[k]).all()
        assert _relerr(m[k], mr[k]) < b["rho"], (k, _relerr(m[k], mr[k]))
    scale = max(np.abs(mr["ua_x"]).max(), np.abs(mr["ub_x"]).max())
    for k in ("ua_x", "ub_x"):
        assert np.abs(m[k] - mr[k]).max() < b["u"] * scale, k
    for k in ("ua_y", "ub_y"):
        assert np.abs(m[k] - mr[k]).max() < b["v"] * scale, k
    for k in ("mdot_a", "mdot_b"):
        assert abs(s[k] / sr[k] - 1) < b["mdot"], k
    assert abs(s["CL"] - sr["CL"]) < b["CL"]


@pytest.mark.parametrize("storage", [binding.LBM_BF16, binding.LBM_FP16])
def test_reduced_precision_steady_state(storage):
    """Steady separation and mass flow of the 1/8-scale Ne-Ar channel against
    the FP32 steady state (BF16 stalls at a residual near 1e-7: the rounding
    noise floor, so its run stops at the step cap)."""
    p = workloads.preset("neon_argon_16384x256", **SCALE_1_8)
    ref = binding.LbmMix(**p)
    ref.init()
    assert ref.run_to_steady(1e-8, 400000, 1000)[0] == binding.LBM_OK
    g = binding.LbmMix(storage=storage, **p)
    g.init()
    st, _, _ = g.run_to_steady(1e-8, 200000, 1000)
    assert st in (binding.LBM_OK, binding.LBM_ENOTCONVERGED)
    s, sr = g.separation(), ref.separation()
    b = BOUNDS_STEADY[storage]
    assert abs(s["CL"] / sr["CL"] - 1) < b["CL"]
    for k in ("mdot_a", "mdot_b"):
        assert abs(s[k] / sr[k] - 1) < b["mdot"], k
