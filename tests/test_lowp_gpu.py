"""Reduced-precision storage (BF16 / FP16 deviations, FP32 arithmetic, FP64
reductions) against the FP64 oracle, and re-referencing of the stored
deviations.

The oracle references (tests/golden/lowp_*.txt, written by
make_lowp_reference.py from the oracle alone) are on copies of the Ne-Ar
reduced-precision workload (C_l = 0.5, theta = 2.5, Kn_out = 0.5, L/H = 64):
the 1/8 linear-scale copy (2048 x 32) after 2000 and 20000 steps, and the
1/16 copy (1024 x 16) at steady state (206 000 steps, residual 1e-9).

Error model.  16-bit storage rounds every stored deviation each step;
stochastic rounding (the default) makes each rounding error zero-mean and
independent of the last, so the error of a run is one draw of a random
process.  The oracle samples that process itself: run with its
post-collision deviations rounded to the same format by stochastic rounding
(its storage emulation, FP64 arithmetic otherwise), it differs from the
exact oracle by the "model" errors the fixtures record (two generator
seeds at 2000 steps, one otherwise).  The GPU's error is another draw of
the same process, on top of its FP32 arithmetic.  One draw says little
about a single quantity (at 20000 steps the one emulated BF16 run happens
to move mdot_b by 8e-7 and mdot_a by 1.3e-4), so the model's scale is taken
over the quantities one rounding process drives alike: the composition
(CL, C~_l, C_l(x), absolute), the two mass flows (relative) and the six
velocity profiles (relative to their columns' largest |u_x|).  Each
quantity is held to K_MODEL times its group's largest emulated error plus
the FP32 parity floor (1e-5 relative on velocities and mass flows, 1e-6
absolute on mole fractions and CL).  Round to nearest has no such model: the same rounding repeats every
step once the flow is steady and its bias accumulates; it is checked to be
far worse than stochastic rounding.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1603_08221_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5
RTOL_U = 1e-5
ATOL_U = 3e-8
K_MODEL = 3.0
# the error model's bound on CL at steady state, relative to CL: the
# emulated BF16 run of the 1024 x 16 fixture moves CL by 0.78 % (FP16: 0.49 %);
# K_MODEL times that is 2.3 %
BF16_STEADY_CL = 0.025
FLOOR = dict(CL=1e-6, Cl_tilde=1e-6, Cl_profile=1e-6, mdot=1e-5, u=1e-5)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STORAGE = {"bf16_sr": binding.LBM_BF16, "fp16_sr": binding.LBM_FP16}


@pytest.fixture(scope="module", autouse=True)
def _libs():
    binding.load()
    oracle.build()


def _golden(name):
    exact, model = {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            if w[0] == "exact":
                exact[(int(w[1]), w[2])] = np.array([float(v) for v in w[3:]])
            else:
                model[(w[1], int(w[2]), int(w[3]), w[4])] = np.array([float(v) for v in w[5:]])
    return exact, model


def _params(N):
    return dict(m_a=workloads.NE, m_b=workloads.AR, C_l=0.5, theta=2.5, Kn_out=0.5, N=N,
                L_over_H=64.0)


def _observe(g):
    """The quantities the fixtures hold, from a GPU handle."""
    s = g.separation()
    m = g.moments()
    nx = g.N_x
    rec = {"CL": s["CL"], "Cl_tilde": s["Cl_tilde"], "mdot_a": s["mdot_a"],
           "mdot_b": s["mdot_b"], "Cl_profile": s["Cl_profile"][::nx // 16]}
    for f in (0.25, 0.5, 0.75):
        x = int(f * nx)
        rec[f"ua_x@{f}"] = m["ua_x"][:, x]
        rec[f"ub_x@{f}"] = m["ub_x"][:, x]
    return rec


def _size(key, d, ref):
    """Error measure of a difference d in quantity `key` (ref: exact
    values): absolute for CL, C~_l and C_l(x); relative for the mass flows;
    relative to the largest |u_x| of the column for velocities."""
    d = np.abs(np.atleast_1d(d))
    if key.startswith("mdot"):
        return float(d.max() / abs(ref[0]))
    if key.startswith("u"):
        return float(d.max() / np.abs(ref).max())
    return float(d.max())


def _group(key):
    if key.startswith("mdot"):
        return "mdot"
    if key.startswith("u"):
        return "u"
    return "composition"


def _floor(key):
    if key.startswith("mdot"):
        return FLOOR["mdot"]
    if key.startswith("u"):
        return FLOOR["u"]
    return FLOOR[key]


def _check_against_model(fixture, N, steps_list, storage_name):
    exact, model = _golden(fixture)
    g = binding.LbmMix(storage=STORAGE[storage_name], **_params(N))
    g.init()
    done = 0
    report = {}
    for steps in steps_list:
        g.step(steps - done)
        done = steps
        obs = _observe(g)
        for key, val in obs.items():
            ref = exact[(steps, key)]
            err = _size(key, np.asarray(val) - ref, ref)
            emul = max(_size(k, d, exact[(steps, k)]) for (st, _, h, k), d in model.items()
                       if st == storage_name and h == steps and _group(k) == _group(key))
            bound = K_MODEL * emul + _floor(key)
            report[(steps, key)] = (err, emul)
            assert err <= bound, (storage_name, steps, key, err, emul)
    return report, exact


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


@pytest.mark.parametrize("storage", ["bf16_sr", "fp16_sr"])
def test_sixteen_bit_against_oracle_one_eighth_copy(storage):
    """BF16 / FP16 storage with stochastic rounding on the 2048 x 32 copy
    after 2000 and 20000 steps: CL, C~_l, mass flows, C_l(x) and the species
    velocity profiles at three columns against the FP64 oracle, within the
    error model."""
    _check_against_model("lowp_neon_argon_2048x32.txt", 32, (2000, 20000), storage)


@pytest.mark.parametrize("storage", ["bf16_sr", "fp16_sr"])
def test_sixteen_bit_steady_state_against_oracle(storage):
    """The 1024 x 16 copy at steady state (206 000 steps): every recorded
    quantity within the error model, and CL within the stated bound of the
    oracle's: 1 % for FP16, BF16_STEADY_CL (2.5 %) for BF16."""
    report, exact = _check_against_model("lowp_neon_argon_1024x16.txt", 16, (206000,), storage)
    err, _ = report[(206000, "CL")]
    cl = exact[(206000, "CL")][0]
    assert err <= (0.01 if storage == "fp16_sr" else BF16_STEADY_CL) * cl, (err, cl)


@pytest.mark.parametrize("storage", [binding.LBM_BF16, binding.LBM_FP16])
def test_round_to_nearest_is_biased(storage):
    """Round to nearest on the 2048 x 32 copy after 20000 steps: its CL
    error against the oracle is more than ten times the error-model bound of
    stochastic rounding (the repeated rounding of a steady flow acts like a
    small body force on the momentum the collision conserves)."""
    exact, model = _golden("lowp_neon_argon_2048x32.txt")
    name = "bf16_sr" if storage == binding.LBM_BF16 else "fp16_sr"
    g = _run(_params(32), 20000, storage=storage, rounding=binding.LBM_ROUND_NEAREST)
    ref = exact[(20000, "CL")]
    err = abs(g.separation()["CL"] - ref[0])
    emul = max(abs(d[0]) for (st, _, h, k), d in model.items()
               if st == name and h == 20000 and k == "CL")
    assert err > 10 * (K_MODEL * emul + FLOOR["CL"]), (err, emul)


@pytest.mark.parametrize("case", [
    dict(N=6, N_x=37, wall=binding.LBM_WALL_BSR),
    dict(N=9, N_x=45, r_form=binding.LBM_R_SECOND),
    dict(N=8, N_x=70, r_form=binding.LBM_R_SPECIES, lambda_pressure=1),
    dict(N=10, N_x=120, C_l_out=0.3),
])
def test_sixteen_bit_wall_variants_follow_fp32(case):
    """16-bit storage takes r and tau_q from a wall kernel of its own (the
    same function the FP32 step's prologue calls).  On small ragged channels
    with the BSR wall, the other readings of Eq. R and lambda_sigma, and
    unequal end compositions, FP16 storage stays within 1 % of the largest
    |u_x| of the FP32 run after 300 steps.  Wall terms taken from the wrong
    column or half would move the near-wall flow by several per cent; FP16's
    rounding moves it by 0.14 - 0.22 % here (GB300).  BF16, with 8x coarser
    rounding, moves it by 1.2 - 2.0 %, too close to such an error to test."""
    p = workloads.preset("heli_argon_320x16", theta=1.5, Kn_out=0.2, **case)
    g32 = _run(p, 300)
    g16 = _run(p, 300, storage=binding.LBM_FP16)
    m32, m16 = g32.moments(), g16.moments()
    scale = max(np.abs(m32["ua_x"]).max(), np.abs(m32["ub_x"]).max())
    assert scale > 0
    for k in ("ua_x", "ua_y", "ub_x", "ub_y"):
        assert np.abs(m16[k] - m32[k]).max() < 1e-2 * scale, k
    for k in ("rho_a", "rho_b"):
        assert _relerr(m16[k], m32[k]) < 1e-3, k
