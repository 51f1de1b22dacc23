"""The paper's parametric study (Table 1, Sec. 4) on the GPU: every run of
Table 1 on the 20 x 700 lattice is advanced to a steady residual as one
graph-replayed sweep, then CL, C~_l (Eq. CL, Eq. Clline), the volume flow
Q_v at the outlet, the species mass flows and the separation rate V_s of
the CL(t) history are reported per run, one JSON line each.

    python -m paper_1603_08221_gb300.study [--tol 1e-8] [--max-steps 400000]
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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--check-every", type=int, default=500)
    a = ap.parse_args(argv)
    run(a.tol, a.max_steps, a.check_every)
    return 0


if __name__ == "__main__":
    sys.exit(main())
