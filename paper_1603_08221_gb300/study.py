"""The paper's parametric study (Table 1, Sec. 4) on the GPU: every run of
Table 1 on the 20 x 700 lattice is advanced to a steady residual as one
graph-replayed sweep, then CL, C~_l (Eq. CL, Eq. Clline), the volume flow
Q_v at the outlet, the species mass flows and the separation rate V_s of
the CL(t) history are reported per run, one JSON line each.

    python -m paper_1603_08221_gb300.study [--tol 1e-8] [--max-steps 400000]
    python -m paper_1603_08221_gb300.study --walls   (DBB against BSR, Fig. 3 setting)
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import binding, diagnostics, workloads


def run(tol: float, max_steps: int, check_every: int, out=sys.stdout):
    runs = workloads.paper_table1()
    names = [n for n, _ in runs]
    sw = binding.LbmSweep([p for _, p in runs])
    sw.init()
    t0 = time.perf_counter()
    steps, R, status = sw.run_to_steady(tol, max_steps, check_every, autotune=True)
    wall = time.perf_counter() - t0
    rows = []
    for k, name in enumerate(names):
        sim = sw.instance(k)
        rec = binding.lbm_mix_history(sim.h, 4096)
        rec_steps = rec[:, 0] * check_every
        row = {"run": name, "status": status[k], "steps": steps[k], "residual": R[k]}
        if status[k] != binding.LBM_ENONFINITE:
            s = sim.separation()
            row.update(CL=s["CL"], Cl_tilde=s["Cl_tilde"], mdot_a=s["mdot_a"],
                       mdot_b=s["mdot_b"], Q_v=sim.volume_flow(), x_min=s["x_min"],
                       V_s=diagnostics.separation_rate(rec_steps, rec[:, 1]))
        rows.append(row)
        print(json.dumps(row), file=out, flush=True)
    print(json.dumps({"runs": len(names), "seconds": wall, "schedule": sw.schedule()[0]}),
          file=out, flush=True)
    return rows


def wall_comparison(tol: float, max_steps: int, check_every: int, out=sys.stdout):
    """The setting of the Method validation section (Fig. 3): He-Ar Case 2
    at Kn_out = 0.3, theta = 3 on the 20 x 700 lattice, run to a steady
    residual once with the diffuse bounce-back wall and once with the
    bounce-back / specular-reflection wall.  Reports the mixture velocity
    u_x = (rho_a u_a,x + rho_b u_b,x)/(rho_a + rho_b) across the channel at
    a quarter, half and three quarters of its length for both walls, and
    their largest difference relative to the DBB maximum."""
    base = dict(workloads.preset("paper_case2_700x20"), theta=3.0, Kn_out=0.3)
    walls = {"dbb": binding.LBM_WALL_DBB, "bsr": binding.LBM_WALL_BSR}
    sw = binding.LbmSweep([dict(base, wall=w) for w in walls.values()])
    sw.init()
    steps, R, status = sw.run_to_steady(tol, max_steps, check_every)
    prof = {}
    for k, name in enumerate(walls):
        m = sw.instance(k).moments()
        rho = m["rho_a"] + m["rho_b"]
        u = (m["rho_a"] * m["ua_x"] + m["rho_b"] * m["ub_x"]) / rho
        nx = u.shape[1]
        prof[name] = {f: u[:, int(f * nx)] for f in (0.25, 0.5, 0.75)}
        row = {"wall": name, "status": status[k], "steps": steps[k], "residual": R[k],
               "CL": sw.instance(k).separation()["CL"],
               "u_x": {str(f): [round(float(v), 8) for v in prof[name][f]] for f in prof[name]}}
        print(json.dumps(row), file=out, flush=True)
    diff = {str(f): float(np.abs(prof["bsr"][f] - prof["dbb"][f]).max() / np.abs(prof["dbb"][f]).max())
            for f in (0.25, 0.5, 0.75)}
    slip = {w: float(prof[w][0.5][0] / prof[w][0.5].max()) for w in walls}
    print(json.dumps({"max_rel_difference": diff, "wall_row_over_max_mid": slip}), file=out,
          flush=True)
    return prof


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--check-every", type=int, default=500)
    ap.add_argument("--walls", action="store_true",
                    help="compare the DBB and BSR walls in the Fig. 3 setting instead")
    a = ap.parse_args(argv)
    if a.walls:
        wall_comparison(a.tol, a.max_steps, a.check_every)
    else:
        run(a.tol, a.max_steps, a.check_every)
    return 0


if __name__ == "__main__":
    sys.exit(main())
