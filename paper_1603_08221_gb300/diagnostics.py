"""Time-history diagnostics of the paper's Sec. 4, computed on the host from
quantities the CUDA library reduces: the separation degree CL(t) and C~_l(t)
(Eq. CL, Eq. Clline) at a fixed step interval, the separation rate V_s and
the dimensionless time of the figures."""
from __future__ import annotations

import numpy as np


def separation_history(sim, total_steps: int, every: int):
    """Steps `sim` (a binding.LbmMix) in blocks of `every` steps up to
    total_steps and returns (steps, CL, C~_l, Q_v at the outlet) after each
    block (the last step of every block reduces the diagnostics)."""
    steps, cl, ct, qv = [], [], [], []
    done = 0
    while done < total_steps:
        k = min(every, total_steps - done)
        sim.step(k)
        done += k
        s = sim.separation()
        steps.append(sim.steps)
        cl.append(s["CL"])
        ct.append(s["Cl_tilde"])
        qv.append(sim.volume_flow())
    return np.array(steps), np.array(cl), np.array(ct), np.array(qv)


def separation_rate(steps, cl) -> float:
    """V_s, the slope of CL(t) that Sec. 4.1 reads off the curves: taken as
    the largest forward difference dCL/dstep of the sampled history (the
    initial rise), per lattice time step."""
    steps = np.asarray(steps, dtype=float)
    cl = np.asarray(cl, dtype=float)
    if steps.size < 2:
        raise ValueError("need at least two samples")
    s = np.concatenate([[0.0], steps])
    c = np.concatenate([[0.0], cl])  # CL = 0 in the uniform initial state
    return float(np.max(np.diff(c) / np.diff(s)))


def dimensionless_time(steps, u_c: float, H: float):
    """t = n dt u_c / H of Sec. 4.1 (dt = 1; u_c is the caller's reference
    mixture velocity, which the paper takes from Case 2 at Kn_out = 0.3,
    theta = 2 without giving its definition)."""
    return np.asarray(steps, dtype=float) * u_c / H
